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


def clique_k5_full():
    """The full K5 count of the k-clique workload (long: the oracle builds every
    last-loop set), merged into clique_rmat20.json."""
    g = S.rmat_clique()
    go, _ = O.reindex(g)
    path = os.path.join(HERE, "clique_rmat20.json")
    rec = json.load(open(path))
    assert rec["nnz"] == g.nnz
    a, order = _plan("k5")
    t = time.time()
    c, e = O.count_nested(a, order, go)
    rec["k5"]["count"] = c
    rec["k5"]["oracle_s"] = round(time.time() - t, 1)
    assert e == rec["k5"]["elems"]
    print("k5", c, rec["k5"]["oracle_s"], flush=True)
    _dump("clique_rmat20.json", rec)


# Root ranges (reindexed ids) of the arbitrary-pattern workload, from hub blocks
# down to low-degree blocks. Each range starts at width 1 and doubles while one
# oracle run stays under SAMPLE_S seconds; a run that passes ATTEMPT_S is
# stopped and the previous width kept (a start whose first root alone passes it
# is dropped), so every pattern's sample costs minutes of CPU at most. Each
# sample stores [lo, hi, count, E].
PATTERN_STARTS = [64, 1000, 20000, 100000, 300000, 1000000]
# the house costs the oracle minutes for one root of degree 40 on this graph
# (its only restriction is one pair), so its blocks start lower in degree
PATTERN_STARTS_BY_NAME = {"house": [600000, 800000, 1000000, 1300000, 1600000, 2000000]}
PATTERN_MAX_W = 4096
SAMPLE_S = 3.0
ATTEMPT_S = 90.0


class _Worker:
    """A spawned process that holds the reindexed graph and runs oracle counts,
    so one that runs past ATTEMPT_S can be stopped (OpenMP state does not
    survive a fork, hence spawn and a graph file instead of inheritance)."""

    def __init__(self, path):
        import multiprocessing as mp
        self.path = path
        self.ctx = mp.get_context("spawn")
        self._start()

    def _start(self):
        self.parent, child = self.ctx.Pipe()
        self.proc = self.ctx.Process(target=_worker_main, args=(child, self.path), daemon=True)
        self.proc.start()

    def count(self, a, order, lo, hi):
        self.parent.send((a, order, lo, hi))
        if self.parent.poll(ATTEMPT_S):
            return self.parent.recv()
        self.proc.kill()
        self.proc.join()
        self._start()
        return None

    def close(self):
        self.proc.kill()
        self.proc.join()


def _worker_main(conn, path):
    import numpy as np
    z = np.load(path)
    go = S.Csr(int(z["n"]), z["row_ptr"], z["col"], "reindexed")
    while True:
        a, order, lo, hi = conn.recv()
        c, e = O.count_nested(a, order, go, lo, hi)
        conn.send((int(c), int(e)))


def patterns(names=None):
    """Recomputes the samples of `names` (default: all five) and keeps the other
    patterns' stored records."""
    import numpy as np
    import tempfile
    g = S.rmat_patterns()
    go, _ = O.reindex(g)
    tmp = os.path.join(tempfile.mkdtemp(), "go.npz")
    np.savez(tmp, n=go.n, row_ptr=go.row_ptr, col=go.col)
    worker = _Worker(tmp)
    rec = {"graph": g.name, "n": g.n, "nnz": g.nnz, "oriented": True, "patterns": {}}
    path = os.path.join(HERE, "patterns_rmat22.json")
    if names and os.path.exists(path):
        old = json.load(open(path))
        if old.get("nnz") == g.nnz:
            rec["patterns"] = old["patterns"]
    for name in (names or PATTERN_SET):
        a, order = _plan(name)
        t0 = time.time()
        samples = []
        for s in PATTERN_STARTS_BY_NAME.get(name, PATTERN_STARTS):
            w, last = 1, None
            while w <= PATTERN_MAX_W:
                t = time.time()
                r = worker.count(a, order, s, s + w)
                dt = time.time() - t
                if r is None:
                    break
                last = [s, s + w, r[0], r[1]]
                if dt > SAMPLE_S:
                    break
                w *= 2
            if last is not None:
                samples.append(last)
        rec["patterns"][name] = {"order": order, "samples": samples,
                                 "oracle_s": round(time.time() - t0, 1)}
        print(name, rec["patterns"][name], flush=True)
    worker.close()
    os.remove(tmp)
    _dump("patterns_rmat22.json", rec)


if __name__ == "__main__":
    which = sys.argv[1:] or ["triangle", "clique", "patterns"]
    for w in which:
        if w.startswith("patterns:"):  # e.g. patterns:house
            patterns(w.split(":", 1)[1].split(","))
        else:
            globals()[w]()
