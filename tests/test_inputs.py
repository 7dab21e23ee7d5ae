"""Host-side checks of the workload inputs: the seeded query table of the
batched workload and the synthetic graph recipes (no GPU, no oracle)."""
from collections import Counter

import numpy as np

import synthetic as S
from synthetic.patterns import (BATCH_MAX_SCALE, BATCH_PATTERNS, BATCH_SPARSE, SERVED_PATTERNS,
                                adjacency, batch_queries)


def test_batch_table_shape_and_placement():
    q = batch_queries()
    assert len(q) == 64
    assert Counter(g for g, _ in q) == {g: 4 for g in range(16)}
    per = Counter(p for _, p in q)
    assert set(per) == set(BATCH_PATTERNS) and min(per.values()) >= 4
    for g, p in q:
        assert S.BATCH_SCALES[g] <= BATCH_MAX_SCALE[p]
        if p in BATCH_SPARSE:
            assert S.BATCH_SCALES[g] <= 14
    assert q == batch_queries()  # seeded


def test_graph_recipes_are_simple_and_seeded():
    for g in [S.rmat(10, 8, 5), S.erdos_renyi(300, 0.05, 3), S.random_small(20, 0.3, 1)]:
        rp, col = g.row_ptr, g.col
        assert rp[0] == 0 and rp[-1] == g.nnz and (np.diff(rp) >= 0).all()
        for v in range(g.n):
            nb = col[rp[v]:rp[v + 1]]
            assert (np.diff(nb) > 0).all() and v not in nb  # sorted, no dups, no loops
        # symmetric
        src = np.repeat(np.arange(g.n), np.diff(rp))
        fwd = set(zip(src.tolist(), col.tolist()))
        assert all((b, a) in fwd for a, b in fwd)
    a, b = S.rmat(10, 8, 5), S.rmat(10, 8, 5)
    assert (a.col == b.col).all() and (a.row_ptr == b.row_ptr).all()


def test_served_patterns_are_named():
    for p in SERVED_PATTERNS:
        a = adjacency(p)
        assert (a == a.T).all()
