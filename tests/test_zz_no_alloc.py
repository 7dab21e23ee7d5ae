"""gz_count_noalloc: counting for callers that cannot allocate device memory at
counting time (stream capture, allocator-free real-time loops, hosts whose
memory manager owns the device). Its counts must equal gz_count's exactly, on
two calls in a row (the static scratch array keeps the previous call's
contents), and it must refuse plans whose scratch exceeds the static maximum.

This file is collected last on purpose, and it also runs alone in a fresh
process: every graph it needs is prepared here.
"""
import numpy as np
import pytest

import synthetic as S

gz = pytest.importorskip("paper_1911_12877_gb300")
pytestmark = pytest.mark.gpu

PATTERNS = ["wedge", "triangle", "path4", "c4", "paw", "diamond", "k4", "house", "chordal5", "k5"]


@pytest.mark.parametrize("oriented", [False, True])
def test_noalloc_matches_count_twice(oriented):
    g = S.rmat(12, 16, 77)
    G = gz.Graph.from_csr(g)
    if oriented:
        G.orient()
    for name in PATTERNS:
        p = gz.Plan(name)
        want = gz.count(p, G, orientation=oriented)  # also builds the views the plan needs
        first = gz.count_noalloc(p, G, orientation=oriented)
        second = gz.count_noalloc(p, G, orientation=oriented)
        assert first == want and second == want, (name, oriented, want, first, second)


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
