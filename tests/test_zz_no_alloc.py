"""gz_count_noalloc: counting for callers that cannot allocate device memory at
counting time (real-time loops that forbid allocator calls after start-up, host
applications whose own memory manager reserves the whole device). Its counts
must equal gz_count's exactly, on two calls in a row (the static scratch array
keeps the previous call's contents); it must make no allocation call (the
library's allocation counter stays put); and it must refuse plans whose scratch
exceeds the static maximum.

This file is collected last on purpose, and it also runs alone in a fresh
process: every graph it needs is prepared here.
"""
import numpy as np
import pytest

import synthetic as S

gz = pytest.importorskip("paper_1911_12877_gb300")
pytestmark = pytest.mark.gpu

PATTERNS = ["wedge", "triangle", "path4", "c4", "paw", "diamond", "k4", "house", "chordal5", "k5"]
NOALLOC_SCRATCH_BYTES = 32 << 20  # GZ_NOALLOC_SCRATCH_BYTES in include/gz.h


@pytest.mark.parametrize("oriented", [False, True])
def test_noalloc_matches_count_twice(oriented):
    g = S.rmat(12, 16, 77)
    G = gz.Graph.from_csr(g)
    if oriented:
        G.orient()
    for name in PATTERNS:
        p = gz.Plan(name)
        want = gz.count(p, G, orientation=oriented)  # also builds the views the plan needs
        a0 = gz.allocations()
        first = gz.count_noalloc(p, G, orientation=oriented)
        second = gz.count_noalloc(p, G, orientation=oriented)
        assert gz.allocations() == a0, (name, "gz_count_noalloc allocated")
        assert first == want and second == want, (name, oriented, want, first, second)


def test_noalloc_reduced_grid_nonzero_counts():
    # A hub adjacent to every vertex of R-MAT 12 makes the per-warp scratch of
    # these plans large enough that the static array holds fewer warps than a
    # full grid, so the call runs on a reduced grid; the counts are far from 0.
    g = S.rmat(12, 16, 79)
    hub = g.n
    src = np.repeat(np.arange(g.n, dtype=np.int32), np.diff(g.row_ptr))
    e = np.stack([src, g.col], 1)
    e = np.concatenate([e[e[:, 0] < e[:, 1]], np.stack([np.full(g.n, hub, np.int32),
                                                        np.arange(g.n, dtype=np.int32)], 1)])
    G = gz.Graph.from_csr(S.from_edges(g.n + 1, e, "rmat12_hub"), validate=gz.GZ_VALIDATE_SYMMETRIC)
    G.orient()
    for name in ["c4", "diamond", "paw", "house"]:
        p = gz.Plan(name)
        for ori in (False, True):
            want = gz.count(p, G, orientation=ori)
            assert gz.scratch_bytes(p, G, orientation=ori) > NOALLOC_SCRATCH_BYTES, (name, ori)
            a0 = gz.allocations()
            got = [gz.count_noalloc(p, G, orientation=ori) for _ in range(2)]
            assert gz.allocations() == a0, (name, ori, "gz_count_noalloc allocated")
            assert want > 0 and got == [want, want], (name, ori, want, got)


def test_noalloc_needs_prepared_views():
    G = gz.Graph.from_csr(S.rmat(10, 8, 78))
    with pytest.raises(gz.GzError) as e:
        gz.count_noalloc(gz.Plan("c4"), G, orientation=False)
    assert e.value.status == gz.GZ_EINVAL


def test_noalloc_rejects_scratch_beyond_the_static_maximum():
    # house keeps five full-degree sets per warp: a 2M-leaf star needs 40 MB each
    leaves = 2_000_000
    e = np.stack([np.zeros(leaves, dtype=np.int32), np.arange(1, leaves + 1, dtype=np.int32)], 1)
    G = gz.Graph.from_csr(S.from_edges(leaves + 1, e, "star2M"), validate=0).orient()
    with pytest.raises(gz.GzError) as err:
        gz.count_noalloc(gz.Plan("house"), G, orientation=True)
    assert err.value.status == gz.GZ_EOVERFLOW
    # a plan that fits still runs on the same graph: a star has no triangle
    assert gz.count_noalloc(gz.Plan("triangle"), G, orientation=True) == 0
