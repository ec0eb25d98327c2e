"""Streamed cycle lists (cc_enumerate_stream): the cycles delivered round by round equal the
oracle's cycle list, for device list capacities from the documented minimum (many rounds)
up to one round, and the counts equal cc_enumerate's.  Table 1's count-only 8 x 10 grid
is listed in full and checked against its printed total."""
import numpy as np
import pytest

import oracle
from paper_1410_4876_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1410_4876_gb300 import cc as _cc
    _cc.load_library()
    return _cc


def _min_caps(g, L):
    d = int(np.diff(np.asarray(g.row_ptr)).max())
    m = len(g.col) // 2
    Lp = g.n if (L == 0 or L > g.n) else L
    return max(d - 1, (d - 1) * m // 2), max((d - 1) * (Lp + 1), 3 * ((d - 1) * m // 2))


def _stream(lg, L, caps):
    got = []

    def sink(starts, lengths, verts):
        for s, k in zip(starts.tolist(), lengths.tolist()):
            got.append(tuple(int(x) for x in verts[s:s + k]))

    r, rounds = lg.enumerate_stream(sink, L, *caps)
    return r, rounds, got


@pytest.mark.parametrize("g,L", [(I.grid(5, 5), 0), (I.wheel(12), 0), (I.gnp(40, 0.12, 3), 0),
                                 (I.complete(7), 0), (I.gnm(120, 135, 3), 0), (I.gnm(400, 800, 9), 9)],
                         ids=lambda x: x.name if hasattr(x, "name") else str(x))
def test_stream_equals_oracle(cc, g, L):
    ref = oracle.enumerate_cycles(g, max_len=L, cycles=True)
    minc, minv = _min_caps(g, L)
    with cc.Context(frontier_bytes=1 << 30) as ctx, ctx.load(g) as lg:
        rounds_seen = []
        for caps in [(minc, minv), (3 * minc + 5, 3 * minv + 7), (1 << 20, 1 << 24)]:
            r, rounds, got = _stream(lg, L, caps)
            rounds_seen.append(rounds)
            assert len(got) == ref.total
            assert sorted(got) == sorted(ref.cycles)
            assert r.hist.tolist() == ref.hist.tolist() and r.hash == ref.hash
            assert r.tcount.tolist() == ref.tcount.tolist()
        assert rounds_seen[-1] == 1
        if ref.total > minc:
            assert rounds_seen[0] > 1
        # capacities below the minimum are refused
        s = cc.cc_enumerate_stream(lg.handle, g.n, lambda *a: None, L, minc - 1 if minc > 1 else 0, minv)[0]
        assert s == cc.CC_ERR_ARG


def test_stream_sink_errors_propagate(cc):
    g = I.grid(4, 4)

    def sink(starts, lengths, verts):
        raise RuntimeError("sink failed")

    with cc.Context(frontier_bytes=1 << 28) as ctx, ctx.load(g) as lg:
        with pytest.raises(RuntimeError, match="sink failed"):
            lg.enumerate_stream(sink)
        # the context is still usable
        assert lg.enumerate().total == oracle.enumerate_cycles(g).total


def test_stream_table1_grid8x10(cc):
    # Table 1 counts the 8 x 10 grid's cycles without storing them; here every one is listed
    # (71,535,910 cycles) through 4 M-cycle device lists
    g = I.grid(8, 10)
    tot = [0, 0]
    lens = np.zeros(81, dtype=np.int64)

    def sink(starts, lengths, verts):
        tot[0] += len(lengths)
        tot[1] += int(lengths.sum(dtype=np.int64))
        lens[:] += np.bincount(lengths, minlength=81)[:81]

    with cc.Context(frontier_bytes=32 << 30) as ctx, ctx.load(g) as lg:
        r, rounds = lg.enumerate_stream(sink, 0, 4 << 20, 96 << 20)
        ref = lg.enumerate()
    assert tot[0] == 71535910 == r.total == ref.total
    assert lens.tolist() == r.hist.tolist()[:81] and tot[1] == sum(k * int(c) for k, c in enumerate(r.hist))
    assert r.hash == ref.hash and rounds > 1
