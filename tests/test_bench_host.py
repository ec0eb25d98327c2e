"""Host-side logic of bench.py (no GPU): the reading of a per-step trace into the levels
that two-level steps expanded without storing, and the algorithmic bytes that follow."""
import importlib.util
import os
from types import SimpleNamespace

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_unstored_levels_from_trace():
    b = _bench()
    tc = np.array([0, 0, 0, 5, 7, 9, 4, 0], dtype=np.uint64)
    assert b.unstored_levels(tc, [5, 7, 9, 4]) == set()      # one level per step
    assert b.unstored_levels(tc, [5, 16, 4]) == {5}          # t=4 step also expanded t=5
    assert b.unstored_levels(tc, [12, 13]) == {4, 6}
    assert b.unstored_levels(tc, [3, 2, 7, 9, 4]) == set()   # chunked steps: not resolved
    assert b.unstored_levels(tc, [5, 7]) == set()            # incomplete trace


def test_algorithmic_bytes_counts_stored_levels():
    b = _bench()
    tc = np.array([0, 0, 0, 5, 7, 9, 4, 0], dtype=np.uint64)
    bitset = SimpleNamespace(tcount=tc, info=SimpleNamespace(mode=1))
    # 20-byte records: every stored path read once, every one after the triplets written once
    assert b.algorithmic_bytes(bitset, 60) == 20 * (2 * 25 - 5)
    assert b.algorithmic_bytes(bitset, 60, {5}) == 20 * (2 * 16 - 5)
    assert b.algorithmic_bytes(bitset, 100) == 28 * (2 * 25 - 5)
    csr = SimpleNamespace(tcount=tc, info=SimpleNamespace(mode=2))
    # u16 ids padded to 8: 16 bytes for t <= 8
    assert b.algorithmic_bytes(csr, 2000) == 16 * 2 * 25 - 16 * 5


def _run_bench(args, env_extra=None):
    import json
    import subprocess
    import sys
    env = dict(os.environ)
    env.update(env_extra or {})
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=env,
                         capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [x for x in out.stdout.splitlines() if x.startswith("{")]
    return [json.loads(x) for x in lines]


def test_reference_arm_json_line():
    # the reference arm times the CPU oracle: one JSON line with the contract's keys
    (line,) = _run_bench(["--impl", "reference", "--workload", "grid6", "--steps", "2", "--warmup", "1"])
    assert line["impl"] == "reference" and line["metric"] == "chordless cycles/s" and line["unit"] == "cycles/s"
    assert line["value"] > 0 and line["higher_is_better"] is True and line["steps"] == 2 and line["warmup"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"] and line["cpu_baseline"]["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "cycles/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"].startswith("grid 6x6")


def test_reference_arm_other_ranks_exit_quietly():
    # under torchrun only rank 0 runs the reference arm; the others exit 0 without output
    env = {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1", "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": "29561"}
    assert _run_bench(["--impl", "reference", "--workload", "grid6", "--steps", "1", "--warmup", "1"], env) == []
