"""Writes tests/golden/table1_grids.txt: the oracle's per-length histogram and cycle hash for
the largest synthetic rows of Table 1 (grids 6 x 10, 7 x 10 and 8 x 10).  Their totals are
the paper's; the histogram and hash are the oracle's (the paper prints neither), so the
GPU tests can compare the full result, not only the total.  Calls only the oracle (its
triplet split over host threads); run from the repository root:

    python tests/golden/make_table1_hashes.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1410_4876_gb300 import inputs as I  # noqa: E402

TABLE1_TOTALS = {(6, 10): 800139, (7, 10): 8136453, (8, 10): 71535910}  # Table 1, #clc (C3 = 0)


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "table1_grids.txt")
    lines = ["# k l total hash hist[4..L'] (nonzero tail trimmed); written by make_table1_hashes.py from the oracle",
             "# totals are Table 1's #clc; histogram and hash are the oracle's"]
    for (k, l), total in TABLE1_TOTALS.items():
        r = oracle.enumerate_parallel(I.grid(k, l))
        assert r.total == total, (k, l, r.total)
        h = [int(x) for x in r.hist]
        while h and h[-1] == 0:
            h.pop()
        lines.append(f"{k} {l} {r.total} {r.hash:#018x} " + " ".join(str(x) for x in h[4:]))
        print(lines[-1][:120], flush=True)
    open(out, "w").write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
