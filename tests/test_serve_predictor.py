"""The serving admission predictor (cc_serve_predict_bytes, pure host code: no GPU) against
the oracle.  Admission reserves, for each request, the bytes of its predicted peak
frontier; the level-synchronous peak of a graph is its two largest consecutive stored
levels (|T_t| + |T_{t+1}| records of 20 bytes), which the oracle gives exactly."""
import numpy as np

import oracle
from paper_1410_4876_gb300 import inputs as I


def _lib():
    from paper_1410_4876_gb300 import build, cc
    build.build()
    cc.load_library()
    return cc


def test_predictor_covers_the_oracle_peak():
    cc = _lib()
    graphs = I.mixture(40, 41)
    covered = 0
    for g in graphs:
        tc = oracle.enumerate_cycles(g).tcount.astype(np.int64)
        peak = int(max(tc[i] + tc[i + 1] for i in range(len(tc) - 1)))
        d = int(np.diff(np.asarray(g.row_ptr)).max())
        covered += cc.cc_serve_predict_bytes(g.n, len(g.col) // 2, d) >= 20 * peak + 4096
    # the predictor's margin is the 99th percentile of its fit residuals
    assert covered >= len(graphs) - 1


def test_predictor_shape():
    cc = _lib()
    assert cc.cc_serve_predict_bytes(3, 3, 2) == 4096  # too small to have paths to store
    # more vertices or a higher mean degree (same maximum degree) never predict less
    assert cc.cc_serve_predict_bytes(20, 40, 5) <= cc.cc_serve_predict_bytes(60, 120, 5)
    assert cc.cc_serve_predict_bytes(40, 60, 6) <= cc.cc_serve_predict_bytes(40, 100, 6)
    # bounded for any input
    assert cc.cc_serve_predict_bytes(64, 2016, 63) <= 10 ** 18
