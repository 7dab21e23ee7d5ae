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


def clique_work():
    """The 32-bit word operations of the per-root bitset form of the K4 and K5
    loops on the k-clique workload (oracle.clique_bitset_work), merged into
    clique_rmat20.json; the walk's clique counts must equal the stored ones."""
    g = S.rmat_clique()
    go, _ = O.reindex(g)
    path = os.path.join(HERE, "clique_rmat20.json")
    rec = json.load(open(path))
    assert rec["nnz"] == g.nnz
    for name, k in (("k4", 4), ("k5", 5)):
        t = time.time()
        c, w = O.clique_bitset_work(k, go)
        assert c == rec[name]["count"], (name, c)
        rec[name]["bitset_words"] = w
        rec[name]["bitset_words_s"] = round(time.time() - t, 1)
        print(name, w, rec[name]["bitset_words_s"], flush=True)
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

    def __init__(self, path, attempt_s=None):
        import multiprocessing as mp
        self.path = path
        self.attempt_s = ATTEMPT_S if attempt_s is None else attempt_s
        self.ctx = mp.get_context("spawn")
        self._start()

    def _start(self):
        self.parent, child = self.ctx.Pipe()
        self.proc = self.ctx.Process(target=_worker_main, args=(child, self.path), daemon=True)
        self.proc.start()

    def count(self, a, order, lo, hi, timeout=None):
        self.parent.send((a, order, lo, hi))
        if self.parent.poll(self.attempt_s if timeout is None else timeout):
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


def _samples(worker, a, order, starts, n=None):
    """[lo, hi, count, E] per start: the width doubles from 1 while one oracle run
    stays under SAMPLE_S (a run past the worker's limit keeps the previous width)."""
    samples = []
    for s in starts:
        if n is not None and s >= n:
            continue
        w, last = 1, None
        while w <= PATTERN_MAX_W:
            hi = s + w if n is None else min(n, s + w)
            t = time.time()
            r = worker.count(a, order, s, hi)
            dt = time.time() - t
            if r is None:
                break
            last = [s, hi, r[0], r[1]]
            if dt > SAMPLE_S or (n is not None and hi >= n):
                break
            w *= 2
        if last is not None:
            samples.append(last)
    return samples


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
        samples = _samples(worker, a, order, PATTERN_STARTS_BY_NAME.get(name, PATTERN_STARTS))
        rec["patterns"][name] = {"order": order, "samples": samples,
                                 "oracle_s": round(time.time() - t0, 1)}
        print(name, rec["patterns"][name], flush=True)
    worker.close()
    os.remove(tmp)
    _dump("patterns_rmat22.json", rec)


# The batched workload: 64 queries over 16 R-MAT graphs (synthetic.patterns.
# batch_queries). Each distinct (graph, pattern) pair gets the oracle's full count
# when it finishes within BATCH_FULL_S on the host; otherwise root-range samples
# (reindexed ids) from hub blocks to low-degree blocks, as for R-MAT 22. The file
# is written after every pair, and a rerun keeps the pairs already stored.
BATCH_FULL_S = 1500.0
BATCH_SAMPLE_FRACS = [0.0, 0.001, 0.01, 0.05, 0.2, 0.5]


def _graph_worker(g, attempt_s):
    import numpy as np
    import tempfile
    go, _ = O.reindex(g)
    tmp = os.path.join(tempfile.mkdtemp(), "go.npz")
    np.savez(tmp, n=go.n, row_ptr=go.row_ptr, col=go.col)
    return _Worker(tmp, attempt_s), tmp


def batched():
    from synthetic.patterns import batch_queries
    table = batch_queries()
    path = os.path.join(HERE, "batched_table.json")
    rec = {"queries": [[gi, name] for gi, name in table], "oriented": True, "graphs": {},
           "results": {}}
    if os.path.exists(path):
        old = json.load(open(path))
        if old.get("queries") == rec["queries"]:
            rec["graphs"], rec["results"] = old["graphs"], old["results"]
    for gi in sorted({gi for gi, _ in table}):
        g = S.batch_graph(gi)
        names = sorted({n for gj, n in table if gj == gi})
        old = rec["graphs"].get(str(gi))
        if old and old["nnz"] == g.nnz and all(f"{gi}:{n}" in rec["results"] for n in names):
            continue
        rec["graphs"][str(gi)] = {"name": g.name, "n": g.n, "nnz": g.nnz}
        worker, tmp = _graph_worker(g, ATTEMPT_S)
        for name in names:
            key = f"{gi}:{name}"
            if key in rec["results"]:
                continue
            a, order = _plan(name)
            t = time.time()
            r = worker.count(a, order, 0, g.n, timeout=BATCH_FULL_S)
            if r is not None:
                res = {"order": order, "count": r[0], "elems": r[1],
                       "oracle_s": round(time.time() - t, 1)}
            else:
                starts = [int(f * g.n) for f in BATCH_SAMPLE_FRACS]
                res = {"order": order, "full_count_over_s": BATCH_FULL_S,
                       "samples": _samples(worker, a, order, starts, g.n),
                       "oracle_s": round(time.time() - t, 1)}
            rec["results"][key] = res
            print(key, g.name, res, flush=True)
            _dump("batched_table.json", rec)
        worker.close()
        os.remove(tmp)
    _dump("batched_table.json", rec)


# The served workload's graph, R-MAT 24 (ef 16, seed 24): full counts are out of
# reach for the oracle, so every pattern of the request mix gets root-range
# samples over the reindexed ids, hub blocks down to low-degree blocks.
SERVED_STARTS = [64, 2000, 50000, 400000, 2000000, 6000000]


def served():
    from synthetic.patterns import SERVED_PATTERNS
    g = S.rmat_served()
    worker, tmp = _graph_worker(g, ATTEMPT_S)
    rec = {"graph": g.name, "n": g.n, "nnz": g.nnz, "oriented": True, "patterns": {}}
    for name in SERVED_PATTERNS:
        a, order = _plan(name)
        t0 = time.time()
        rec["patterns"][name] = {"order": order, "samples": _samples(worker, a, order, SERVED_STARTS),
                                 "oracle_s": round(time.time() - t0, 1)}
        print(name, rec["patterns"][name], flush=True)
        _dump("served_rmat24.json", rec)
    worker.close()
    os.remove(tmp)


if __name__ == "__main__":
    which = sys.argv[1:] or ["triangle", "clique", "patterns"]
    for w in which:
        if w.startswith("patterns:"):  # e.g. patterns:house
            patterns(w.split(":", 1)[1].split(","))
        else:
            globals()[w]()
