"""Writes the stored expected values in tests/golden/*.json.

Calls only ``oracle`` (the CPU oracle) and ``synthetic`` (the seeded inputs); no
value here comes from the CUDA path. Run from the repository root:

    python tests/golden/make_golden.py [clique|triangle|patterns ...]

Counts are exact integers. "elems" is E, the number of list elements the
bounded linear scans of the paper's nested loops consume (see gz_oracle.c).
Root ranges are vertex ids of the degree-reindexed graph (Sec. 6 orientation).
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
import synthetic as S  # noqa: E402
from synthetic.patterns import PATTERN_SET, adjacency  # noqa: E402


def _dump(name, rec):
    path = os.path.join(HERE, name)
    with open(path, "w") as f:
        json.dump(rec, f, indent=1)
    print("wrote", path, flush=True)


def _plan(name):
    a = adjacency(name)
    order, _ = O.choose_schedule(a)
    return a, [int(x) for x in order]


def triangle():
    g = S.er_triangle()
    a, order = _plan("triangle")
    c, e = O.count_nested(a, order, g)
    _dump("er_triangle.json", {"graph": g.name, "n": g.n, "nnz": g.nnz, "oriented": False,
                               "triangle": {"order": order, "count": c, "elems": e}})


K5_SAMPLES = [(0, 32), (2000, 2064), (60000, 62000), (700000, 720000)]


def clique():
    g = S.rmat_clique()
    go, _ = O.reindex(g)
    rec = {"graph": g.name, "n": g.n, "nnz": g.nnz, "oriented": True}
    a, order = _plan("k4")
    t = time.time()
    c, e = O.count_nested(a, order, go)
    rec["k4"] = {"order": order, "count": c, "elems": e, "oracle_s": round(time.time() - t, 1)}
    print("k4", rec["k4"], flush=True)
    a, order = _plan("k5")
    t = time.time()
    e = O.elems_nested(a, order, go)
    rec["k5"] = {"order": order, "elems": e, "oracle_elems_s": round(time.time() - t, 1),
                 "samples": [[lo, hi, O.count_nested(a, order, go, lo, hi)[0]] for lo, hi in K5_SAMPLES]}
    print("k5", rec["k5"], flush=True)
    _dump("clique_rmat20.json", rec)


# Root ranges (reindexed ids) of the arbitrary-pattern workload: a top hub block, two
# mid-degree blocks and a low-degree block. Each range is grown from width 1 by
# doubling while the oracle stays within a few seconds on it, so the sample costs
# the same order of CPU time whatever the pattern.
PATTERN_STARTS = [64, 20000, 300000, 1000000]
PATTERN_MAX_W = 4096


def patterns():
    g = S.rmat_patterns()
    go, _ = O.reindex(g)
    rec = {"graph": g.name, "n": g.n, "nnz": g.nnz, "oriented": True, "patterns": {}}
    for name in PATTERN_SET:
        a, order = _plan(name)
        t0 = time.time()
        samples = []
        for s in PATTERN_STARTS:
            w, last = 1, None
            while True:
                t = time.time()
                c = O.count_nested(a, order, go, s, s + w)[0]
                dt = time.time() - t
                last = [s, s + w, c]
                if dt > 4.0 or w >= PATTERN_MAX_W:
                    break
                w *= 2
            samples.append(last)
        rec["patterns"][name] = {"order": order, "samples": samples,
                                 "oracle_s": round(time.time() - t0, 1)}
        print(name, rec["patterns"][name], flush=True)
    _dump("patterns_rmat22.json", rec)


if __name__ == "__main__":
    which = sys.argv[1:] or ["triangle", "clique", "patterns"]
    for w in which:
        globals()[w]()
