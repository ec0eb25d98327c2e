"""Host-side logic of bench.py (no GPU): algorithmic bytes per stored path, the roofline
arithmetic, the exchange of per-rank results, and the reference arm's JSON line."""
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


def test_algorithmic_bytes_counts_every_stored_path():
    b = _bench()
    tc = np.array([0, 0, 0, 5, 7, 9, 4, 0], dtype=np.uint64)
    # bitset records: 16 bytes for one word (n <= 64), 32 for two, 48 for four; each stored
    # path written once and read once
    assert b.algorithmic_bytes(tc, 60, 1) == 2 * 16 * 25
    assert b.algorithmic_bytes(tc, 100, 1) == 2 * 32 * 25
    assert b.algorithmic_bytes(tc, 200, 1) == 2 * 48 * 25
    # CSR records: u16 ids padded to 8 (16 bytes up to 8 vertices, 32 up to 16)
    tc2 = np.zeros(12, dtype=np.uint64)
    tc2[3], tc2[8], tc2[9], tc2[11] = 5, 2, 3, 1
    assert b.algorithmic_bytes(tc2, 2000, 2) == 2 * (16 * 5 + 16 * 2 + 32 * 3 + 32 * 1)


def test_roofline_of_a_known_kernel():
    b = _bench()
    r = b.roofline("k", 2.0e9, 1.0, 1e6, "no_such_profile")
    peak, _ = b._peaks()
    assert abs(r["achieved"] - 2000.0) < 1e-9 and abs(r["frac"] - 2000.0 / peak) < 1e-12
    assert r["traffic"] is None and r["unit"] == "GB/s"


def test_sum_results_without_ranks_wraps_the_hash():
    b = _bench()
    h, hh = b.sum_results(np.array([0, 0, 0, 4], dtype=np.uint64), (1 << 64) + 5, None)
    assert h.tolist() == [0, 0, 0, 4] and hh == 5


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
    _check_reference_line(line)
    assert line["config"]["workload"].startswith("grid 6x6")


def test_reference_arm_batch_workload():
    # the default workload: a rotating sample of the batch's graphs per step
    (line,) = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "1", "--batch-count", "1024"])
    _check_reference_line(line)
    assert line["config"]["workload"].startswith("1024 graphs of the seeded batch mixture")


def _check_reference_line(line):
    assert line["impl"] == "reference" and line["metric"] == "chordless cycles/s" and line["unit"] == "cycles/s"
    assert line["value"] > 0 and line["higher_is_better"] is True and line["steps"] >= 1 and line["warmup"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"] and line["cpu_baseline"]["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "cycles/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    # under torchrun only rank 0 runs the reference arm; the others exit 0 without output
    env = {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1", "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": "29561"}
    assert _run_bench(["--impl", "reference", "--workload", "grid6", "--steps", "1", "--warmup", "1"], env) == []


def test_steps_for_clocks_spans_the_sampler():
    b = _bench()
    # a 0.9 ms step needs about 1667 steps for a 1.5 s region; long steps keep the count
    assert b.steps_for_clocks(10, 0.9) == 1667
    assert b.steps_for_clocks(20, 120.0) == 20
    assert b.steps_for_clocks(10, 1e-4) == 5000   # capped
    assert b.steps_for_clocks(7, 0.0) == 7         # no estimate: as asked


def test_engine_fingerprint_is_per_form(tmp_path, monkeypatch):
    # a capture stays valid while the code its kernel runs is unchanged: editing one
    # expansion form changes that form's fingerprint only
    import shutil
    b = _bench()
    root = tmp_path / "repo"
    csrc = root / "paper_1410_4876_gb300" / "csrc"
    shutil.copytree(os.path.join(ROOT, "paper_1410_4876_gb300", "csrc"), csrc)
    monkeypatch.setattr(b, "ROOT", str(root))
    kinds = ("engine_kernel<Multi,256>", "engine_kernel<Bitset1,256>", "engine_kernel<Csr16,256>")
    before = {k: b._engine_fingerprint(k) for k in kinds}
    assert len(set(before.values())) == 3
    with open(csrc / "cc_expand_multi.cuh", "a") as f:
        f.write("\n// a comment changes nothing\n")
    assert {k: b._engine_fingerprint(k) for k in kinds} == before
    with open(csrc / "cc_expand_multi.cuh", "a") as f:
        f.write("\nstatic_assert(true, \"\");\n")
    after = {k: b._engine_fingerprint(k) for k in kinds}
    assert after[kinds[0]] != before[kinds[0]]
    assert after[kinds[1]] == before[kinds[1]] and after[kinds[2]] == before[kinds[2]]
