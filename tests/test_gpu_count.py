"""GPU parity: libgz's CUDA path against the CPU oracle, bit-exact (counts are
integers, so the tolerance is zero).

Inputs are the seeded synthetic graphs of ``synthetic``; expected values come
from ``oracle`` only (computed here, or stored by tests/golden/make_golden.py).
"""
import json
import os

import numpy as np
import pytest

import oracle as O
import synthetic as S
from synthetic.patterns import BATCH_PATTERNS, EDGES, PATTERN_SET, adjacency

gz = pytest.importorskip("paper_1911_12877_gb300")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SMALL_NAMES = ["edge", "wedge", "triangle", "path4", "star3", "c4", "paw", "diamond", "k4", "c5",
               "house", "hourglass", "chordal5", "k5", "k6", "chordal6", "asym6"]


_ORACLE_CACHE = {}


def oracle_count(name_or_adj, g, oriented=True, lo=0, hi=None):
    """Oracle B count. The count does not depend on the labelling (pinned in
    test_oracle), and on the degree-reindexed graph the oracle's bounded scans
    are far shorter, so it runs there by default."""
    a = adjacency(name_or_adj) if isinstance(name_or_adj, str) else name_or_adj
    key = (a.tobytes(), g.name, g.n, g.nnz, oriented, lo, hi)
    if g.name and key in _ORACLE_CACHE:
        return _ORACLE_CACHE[key]
    order, _ = O.choose_schedule(a)
    if oriented:
        g, _ = O.reindex(g)
    r = O.count_nested(a, order, g, lo, hi)[0]
    _ORACLE_CACHE[key] = r
    return r


@pytest.fixture(scope="module")
def tiny_graphs():
    return [S.random_small(12, 0.45, 21), S.random_small(30, 0.2, 22), S.random_small(40, 0.12, 23)]


@pytest.mark.parametrize("name", SMALL_NAMES)
def test_tiny_graphs_every_schedule(name, tiny_graphs):
    a = adjacency(name)
    for g in tiny_graphs:
        G = gz.Graph.from_csr(g, validate=gz.GZ_VALIDATE_SYMMETRIC).orient()
        want = oracle_count(a, g)
        for s in O.distinct_schedules(a)[:6]:
            p = gz.Plan(a, order=s)
            assert gz.count(p, G, orientation=False) == want, (name, s)
            assert gz.count(p, G, orientation=True) == want, (name, s, "oriented")


@pytest.mark.parametrize("graph", ["empty0", "empty7", "star", "K8", "K34", "petersen", "C6",
                                   "hub_last", "two_comp"])
def test_structured_edge_cases(graph):
    g = {
        "empty0": lambda: S.empty(0), "empty7": lambda: S.empty(7), "star": lambda: S.star(40),
        "K8": lambda: S.complete(8), "K34": lambda: S.complete_bipartite(3, 4),
        "petersen": S.petersen, "C6": lambda: S.cycle(6),
        "hub_last": lambda: S.from_edges(50, [(49, i) for i in range(49)] + [(0, 1), (2, 3)]),
        "two_comp": lambda: S.from_edges(12, [(i, j) for i in range(5) for j in range(i + 1, 5)]
                                         + [(6, 7), (7, 8), (8, 9), (9, 6)]),
    }[graph]()
    G = gz.Graph.from_csr(g, validate=gz.GZ_VALIDATE_SYMMETRIC).orient()
    for name in ["edge", "wedge", "triangle", "c4", "star3", "diamond", "k4", "c5", "k5"]:
        want = O.count_brute_induced(adjacency(name), g) if g.n <= 50 and len(adjacency(name)) <= 4 \
            else oracle_count(name, g)
        p = gz.Plan(name)
        assert gz.count(p, G, False) == want, (graph, name)
        assert gz.count(p, G, True) == want, (graph, name, "oriented")


@pytest.mark.parametrize("which", ["er", "rmat12", "rmat16"])
def test_orientation_matches_oracle_relabel(which):
    g = {"er": S.er_triangle, "rmat12": lambda: S.rmat(12, 16, 5),
         "rmat16": lambda: S.rmat(16, 8, 6)}[which]()
    G = gz.Graph.from_csr(g).orient()
    rp, col, nid = G.export(oriented=True)
    orp, ocol = O.reindex(g)[0].row_ptr, O.reindex(g)[0].col
    onid = O.reindex(g)[1]
    assert (nid == onid).all()
    assert (rp == orp).all()
    assert (col == ocol).all()
    info = G.info()
    split = [int(np.searchsorted(ocol[orp[v]:orp[v + 1]], v)) for v in range(g.n)]
    assert info["max_out_degree_oriented"] == max(split)
    assert info["max_degree"] == int(np.diff(g.row_ptr).max())


def test_reorient_is_repeatable():
    g = S.rmat(13, 16, 7)
    G = gz.Graph.from_csr(g).orient()
    a = G.export(oriented=True)
    G.orient()
    b = G.export(oriented=True)
    for x, y in zip(a, b):
        assert (x == y).all()


def test_er_triangle_workload():
    # Triangle counting, plain method on the original ids: G(4096, 16/4095), seed 1.
    g = S.er_triangle()
    G = gz.Graph.from_csr(g, validate=gz.GZ_VALIDATE_SYMMETRIC)
    want = oracle_count("triangle", g)
    assert gz.count(gz.Plan("triangle"), G, orientation=False) == want
    G.orient()
    assert gz.count(gz.Plan("triangle"), G, orientation=True) == want


@pytest.mark.parametrize("name", ["wedge", "triangle", "path4", "star3", "c4", "paw", "diamond",
                                  "k4", "house", "chordal5", "k5", "chordal6", "hourglass", "c5"])
def test_rmat_medium_all_patterns(name):
    g = S.rmat(11, 8, 31)  # 2048 vertices, ragged hub lists
    G = gz.Graph.from_csr(g).orient()
    want = oracle_count(name, g)
    p = gz.Plan(name)
    assert gz.count(p, G, True) == want
    assert gz.count(p, G, False) == want


def test_root_ranges_partition_count():
    g = S.rmat(14, 16, 9)
    G = gz.Graph.from_csr(g).orient()
    p = gz.Plan("diamond")
    total = gz.count(p, G, True)
    cuts = [0, 1, 7, 100, 1000, 5000, g.n]
    parts = [gz.count(p, G, True, lo, hi) for lo, hi in zip(cuts[:-1], cuts[1:])]
    assert sum(parts) == total
    go, _ = O.reindex(g)
    order, _ = O.choose_schedule(adjacency("diamond"))
    for (lo, hi), c in zip(zip(cuts[:-1], cuts[1:]), parts):
        if hi - lo <= 1000:
            assert c == O.count_nested(adjacency("diamond"), order, go, lo, hi)[0]


@pytest.mark.parametrize("bw,chunk", [(4, 1), (8, 4), (2, 16), (8, 64)])
def test_launch_shapes_do_not_change_counts(bw, chunk):
    g = S.rmat(13, 16, 10)
    G = gz.Graph.from_csr(g).orient()
    for name in ["k4", "c4", "diamond"]:
        p = gz.Plan(name)
        assert gz.count(p, G, True, block_warps=bw, chunk=chunk) == oracle_count(name, g)


@pytest.mark.parametrize("name", ["k4", "diamond", "c4"])
def test_autotune_keeps_count(name):
    g = S.rmat(13, 16, 11)
    G = gz.Graph.from_csr(g).orient()
    p = gz.Plan(name)
    want = oracle_count(name, g)
    assert gz.count(p, G, True) == want
    t = gz.autotune(p, G, True)
    assert t["block_warps"] in (4, 8) and t["chunk"] in (1, 2, 4, 8, 16)
    assert t["split_min"] in (4, 16, 64, 128, 512, 4096) and t["split_chunk"] in (1, 8, 64, 256)
    assert gz.count(p, G, True) == want  # single count with the tuned settings
    # a batch with the tuned query beside untuned ones
    q = gz.Plan("triangle")
    assert gz.count_batch([p, q, p], [G, G, G], [True, False, True]) == [want, oracle_count("triangle", g), want]


def test_split_thresholds_do_not_change_counts():
    """Tuned split thresholds per query: with every unit deferred (threshold 1)
    and one-candidate work items the counts stay the oracle's."""
    g = S.rmat(12, 16, 12)
    G = gz.Graph.from_csr(g).orient()
    for name in ["diamond", "c4", "house", "chordal5"]:
        p = gz.Plan(name)
        want = oracle_count(name, g)
        assert gz.count(p, G, True, split_min=1, split_chunk=1) == want, name
        assert gz.count(p, G, True, split_min=1 << 40, split_chunk=512) == want, name


def test_batch_equals_alone():
    graphs = [S.rmat(10, 8, 100), S.rmat(12, 16, 101), S.er_triangle(), S.rmat(11, 32, 102)]
    Gs = [gz.Graph.from_csr(g).orient() for g in graphs]
    plans = {n: gz.Plan(n) for n in BATCH_PATTERNS}
    qp, qg, qo = [], [], []
    for i, n in enumerate(BATCH_PATTERNS):
        for j in range(len(Gs)):
            if (i + j) % 2 == 0:
                qp.append(plans[n]); qg.append(Gs[j]); qo.append((i + j) % 4 == 0)
    got = gz.count_batch(qp, qg, qo)
    alone = [gz.count(p, G, o) for p, G, o in zip(qp, qg, qo)]
    assert got == alone
    idx = {id(G): graphs[j] for j, G in enumerate(Gs)}
    for p, G, c in zip(qp, qg, got):
        name = [n for n, pp in plans.items() if pp is p][0]
        if name in ("triangle", "k4", "diamond", "c4", "k5"):
            assert c == oracle_count(name, idx[id(G)])


def test_batched_table_against_oracle():
    """The batched workload (64 queries over 16 R-MAT graphs) in one gz_count_batch
    call against the oracle's values stored by tests/golden/make_golden.py: full
    counts where the oracle finished, else its sampled root ranges (each counted
    here through gz_count_ex) plus equality with the query counted alone."""
    gold = json.load(open(os.path.join(GOLDEN, "batched_table.json")))
    from synthetic.patterns import batch_queries
    table = batch_queries()
    assert gold["queries"] == [[gi, n] for gi, n in table]
    graphs = {}
    for gi in sorted({gi for gi, _ in table}):
        g = S.batch_graph(gi)
        assert gold["graphs"][str(gi)]["nnz"] == g.nnz
        graphs[gi] = gz.Graph.from_csr(g).orient()
    plans = {n: gz.Plan(n) for n in {n for _, n in table}}
    got = gz.count_batch([plans[n] for _, n in table], [graphs[gi] for gi, _ in table], [True] * len(table))
    sampled = 0
    for (gi, n), c in zip(table, got):
        r = gold["results"][f"{gi}:{n}"]
        assert r["order"] == plans[n].info()["order"] or "count" in r
        if "count" in r:
            assert c == r["count"], (gi, n, c, r["count"])
        else:
            sampled += 1
            assert c == gz.count(plans[n], graphs[gi], True), (gi, n)
            for lo, hi, want, _ in r["samples"]:
                assert gz.count(plans[n], graphs[gi], True, lo, hi) == want, (gi, n, lo, hi)
    assert sampled <= len(table) // 4


def test_server_equals_alone():
    g = S.rmat(12, 16, 50)
    G = gz.Graph.from_csr(g).orient()
    names = ["triangle", "c4", "diamond", "k4", "k5", "chordal5"]
    plans = [gz.Plan(n) for n in names]
    alone = [gz.count(p, G, True) for p in plans]
    # served, FIFO and alone must all equal the oracle's count for each pattern
    assert alone == [oracle_count(n, g) for n in names]
    srv = gz.Server(max_inflight=3, max_batch=8)
    rng = np.random.default_rng(5)
    pidx = rng.integers(0, len(names), 60).astype(np.int32)
    arr = np.cumsum(rng.exponential(2e5, 60)).astype(np.int64)  # ~5000 req/s
    counts, lat, stats = srv.replay(plans, [G], [1] * 60, arr, pidx, np.zeros(60, np.int32))
    assert [int(c) for c in counts] == [alone[i] for i in pidx]
    assert (lat > 0).all()
    counts_f, lat_f, stats_f = srv.replay(plans, [G], [1] * 60, arr, pidx, np.zeros(60, np.int32),
                                          fifo=True)
    assert [int(c) for c in counts_f] == [alone[i] for i in pidx]
    assert stats_f["launches"] == 60
    t = [srv.submit(plans[i], G, True) for i in range(len(plans))]
    assert [srv.wait(x)[0] for x in t] == alone
    srv.close()


def test_server_slow_share_equals_oracle():
    """Every request classed slow (a tiny threshold): each runs alone on a small
    share of the device while the others wait; the counts must still equal the
    oracle's (the grid size never changes which work is done)."""
    g = S.rmat(12, 16, 51)
    G = gz.Graph.from_csr(g).orient()
    names = ["triangle", "c4", "diamond", "k4", "k5", "chordal5"]
    plans = [gz.Plan(n) for n in names]
    want = [oracle_count(n, g) for n in names]
    srv = gz.Server(max_inflight=2, max_batch=4, heavy_ms=1e-3, slow_share=0.05)
    rng = np.random.default_rng(7)
    pidx = rng.integers(0, len(names), 24).astype(np.int32)
    arr = np.cumsum(rng.exponential(1e6, 24)).astype(np.int64)
    counts, lat, stats = srv.replay(plans, [G], [1] * 24, arr, pidx, np.zeros(24, np.int32))
    assert [int(c) for c in counts] == [want[i] for i in pidx]
    assert stats["launches"] == 24  # every slow request alone in its launch
    srv.close()


def test_device_pointer_graph():
    import torch
    g = S.rmat(12, 16, 60)
    rp = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    G = gz.Graph(rp, col, validate=gz.GZ_VALIDATE_SYMMETRIC).orient()
    assert gz.count(gz.Plan("k4"), G, True) == oracle_count("k4", g)


@pytest.mark.parametrize("bad", ["unsorted", "selfloop", "range", "dup", "asym", "rowptr"])
def test_invalid_csr_rejected(bad):
    g = S.complete(5)
    rp, col = g.row_ptr.copy(), g.col.copy()
    if bad == "unsorted":
        col[0], col[1] = col[1], col[0]
    elif bad == "selfloop":
        col[0] = 0
    elif bad == "range":
        col[0] = 99
    elif bad == "dup":
        col[1] = col[0]
    elif bad == "asym":  # 0 -> 1 without 1 -> 0
        rp = np.array([0, 1, 1], dtype=np.int64)
        col = np.array([1], dtype=np.int32)
    elif bad == "rowptr":
        rp[2] = rp[1] - 1
    with pytest.raises(gz.GzError) as e:
        gz.Graph(rp, col, validate=gz.GZ_VALIDATE_SYMMETRIC)
    assert e.value.status == gz.GZ_EINVAL


def test_orientation_needed_for_oriented_count():
    G = gz.Graph.from_csr(S.complete(6))
    with pytest.raises(gz.GzError):
        gz.count(gz.Plan("triangle"), G, orientation=True)


# ------------------------------------------------------------ full-size workloads

def _golden(name):
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        pytest.skip(f"golden file {name} missing")
    return json.load(open(path))


def test_clique_rmat20_full_and_sampled():
    """k-clique workload (R-MAT scale 20, ef 16, seed 20, oriented), in the launch
    configuration the bench times: K4 and K5 in full, and K5 on sampled root ranges,
    against the stored oracle counts."""
    gold = _golden("clique_rmat20.json")
    g = S.rmat_clique()
    assert g.nnz == gold["nnz"]
    G = gz.Graph.from_csr(g).orient()
    k4, k5 = gz.Plan("k4"), gz.Plan("k5")
    assert gz.count(k4, G, True) == gold["k4"]["count"]
    for (lo, hi, c) in gold["k5"]["samples"]:
        assert gz.count(k5, G, True, lo, hi) == c, (lo, hi)
    if "count" in gold["k5"]:
        assert gz.count(k5, G, True) == gold["k5"]["count"]


def test_served_rmat24_sampled():
    """The served workload's graph (R-MAT 24, ef 16, seed 24): every pattern of the
    request mix on the oracle's sampled root ranges (reindexed ids)."""
    gold = json.load(open(os.path.join(GOLDEN, "served_rmat24.json")))
    g = S.rmat_served()
    assert gold["nnz"] == g.nnz
    G = gz.Graph.from_csr(g).orient()
    for name, rec in gold["patterns"].items():
        p = gz.Plan(name)
        assert p.info()["order"] == rec["order"]
        for lo, hi, want, _ in rec["samples"]:
            assert gz.count(p, G, True, lo, hi) == want, (name, lo, hi)


def test_patterns_rmat22_sampled():
    """Arbitrary-pattern workload (R-MAT scale 22, ef 16, seed 22, oriented):
    sampled root ranges against stored oracle counts."""
    gold = _golden("patterns_rmat22.json")
    g = S.rmat_patterns()
    assert g.nnz == gold["nnz"]
    G = gz.Graph.from_csr(g).orient()
    for name, rec in gold["patterns"].items():
        p = gz.Plan(name)
        for (lo, hi, c, *_) in rec["samples"]:
            assert gz.count(p, G, True, lo, hi) == c, (name, lo, hi)


@pytest.mark.parametrize("k", [4, 5, 6, 7, 8])
def test_cliques_on_long_out_lists(k):
    """Oriented k-cliques through the bitset kernels on roots whose out-lists span
    several 32-bit words (odd and even word counts) against the oracle."""
    for n, p, seed in [(90, 0.55, 41), (160, 0.45, 42), (240, 0.42, 44), (300, 0.4, 43)]:
        g = S.random_small(n, p, seed)
        G = gz.Graph.from_csr(g).orient()
        assert G.info()["max_out_degree_oriented"] > 32
        name = {4: "k4", 5: "k5", 6: "k6"}.get(k)
        a = adjacency(name) if name else adjacency([(i, j) for i in range(k) for j in range(i + 1, k)], k)
        want = oracle_count(a, g)
        assert gz.count(gz.Plan(a), G, orientation=True) == want, (k, n)


def test_cliques_with_out_lists_beyond_the_bitset_limit():
    """Roots whose out-list exceeds the bitset kernels' 1024 are counted by the
    general kernel in the same call. K_{m,m} plus a perfect matching inside each
    side: every K4 takes one matching edge per side, so there are (m/2)^2 of
    them, and there is no K5 (a side holds no triangle)."""
    m = 1100
    e = [(i, m + j) for i in range(m) for j in range(m)]
    e += [(2 * i, 2 * i + 1) for i in range(m // 2)] + [(m + 2 * i, m + 2 * i + 1) for i in range(m // 2)]
    g = S.from_edges(2 * m, e, "Kmm_matchings")
    G = gz.Graph.from_csr(g).orient()
    assert G.info()["max_out_degree_oriented"] > 1024
    assert gz.count(gz.Plan("k4"), G, orientation=True) == (m // 2) ** 2
    assert gz.count(gz.Plan("k5"), G, orientation=True) == 0
    assert gz.count(gz.Plan("k4"), G, orientation=True) == oracle_count("k4", g)


def test_fused_k4_k5_closed_form():
    """K4 and K5 in one gz_count_merged call take the fused clique pass (one walk
    over the root pairs yields both counts). Complete 16-partite graph with parts
    of 60: oriented out-lists up to 900 (rows of 29 words, all in shared memory).
    A k-clique takes one vertex from each of k parts: C(16, k) * 60^k. A second
    K4 query and a triangle query ride along on the separate clique kernels."""
    import math
    parts, r = 16, 60
    n = parts * r
    idx = np.arange(n)
    src, dst = np.meshgrid(idx, idx, indexing="ij")
    keep = (src < dst) & (src // r != dst // r)
    e = np.stack([src[keep], dst[keep]], 1).astype(np.int32)
    G = gz.Graph.from_csr(S.from_edges(n, e, "K16x60")).orient()
    assert 32 < G.info()["max_out_degree_oriented"] <= 1024
    want = {k: math.comb(parts, k) * r ** k for k in (3, 4, 5)}
    names = ["k4", "k5", "k4", "triangle"]
    got = gz.count_merged([gz.Plan(x) for x in names], G, orientation=True)
    assert got == [want[4], want[5], want[4], want[3]]
    # on an R-MAT graph (roots of every out-degree class up to the longest) the
    # fused counts equal the oracle's
    g = S.rmat(13, 16, 53)
    G2 = gz.Graph.from_csr(g).orient()
    assert gz.count_merged([gz.Plan("k5"), gz.Plan("k4")], G2, orientation=True) == [
        oracle_count("k5", g), oracle_count("k4", g)]


def test_prepare_then_count():
    """gz_prepare builds the views and clique rows ahead of the count; counts
    after it (and after a second prepare, and after reorienting) are the
    oracle's, and an oriented prepare on a graph never oriented is refused."""
    g = S.rmat(12, 16, 57)
    G = gz.Graph.from_csr(g)
    with pytest.raises(gz.GzError) as e:
        gz.prepare(gz.Plan("k5"), G, orientation=True)
    assert e.value.status == gz.GZ_EINVAL
    G.orient()
    want = [oracle_count(n, g) for n in ("k4", "k5", "diamond")]
    plans = [gz.Plan(n) for n in ("k4", "k5", "diamond")]
    for p in plans:
        gz.prepare(p, G, orientation=True)
    gz.prepare(plans[1], G, orientation=True)
    assert gz.count_merged(plans, G, orientation=True) == want
    G.orient()
    gz.prepare(plans[1], G, orientation=True)
    assert [gz.count(p, G, True) for p in plans] == want


def test_cliques_on_multipartite_long_out_lists():
    """Complete 16-partite graph with parts of 75: every vertex has degree 1125,
    so oriented out-lists run past 1024 (the long-root launch of the K4/K5
    kernels and their wide pairs, b >= 1024). A k-clique takes one vertex from
    each of k parts: C(16, k) * 75^k of them (closed form)."""
    import math
    parts, r = 16, 75
    n = parts * r
    idx = np.arange(n)
    src, dst = np.meshgrid(idx, idx, indexing="ij")
    keep = (src < dst) & (src // r != dst // r)
    e = np.stack([src[keep], dst[keep]], 1).astype(np.int32)
    G = gz.Graph.from_csr(S.from_edges(n, e, "K16x75")).orient()
    assert G.info()["max_out_degree_oriented"] > 1024
    for k in (4, 5):
        assert gz.count(gz.Plan(f"k{k}"), G, orientation=True) == math.comb(parts, k) * r ** k, k


@pytest.mark.parametrize("name", ["diamond", "paw", "c4", "house", "chordal5", "hourglass"])
def test_split_units_book_graph(name):
    """Units whose loop-2 candidate list reaches the split threshold (512) are
    deferred, cut into chunks and finished by other warps; the count must not
    change. Book graph: an edge (0, 1) whose ends share 700 neighbours, plus a
    seeded sprinkling of edges among those neighbours."""
    rng = np.random.default_rng(7)
    pages = list(range(2, 702))
    e = [(0, 1)] + [(0, p) for p in pages] + [(1, p) for p in pages]
    extra = rng.choice(pages, size=(900, 2))
    e += [(int(a), int(b)) for a, b in extra if a != b]
    g = S.from_edges(702, e, "book700")
    G = gz.Graph.from_csr(g).orient()
    p = gz.Plan(name)
    want = oracle_count(name, g)
    assert gz.count(p, G, orientation=True) == want
    assert gz.count(p, G, orientation=False) == want
    assert gz.count_batch([p, p], [G, G], [True, False]) == [want, want]


def test_server_wait_statuses():
    """gz_server_wait: a wait that runs out returns GZ_ETIMEOUT and leaves the
    request pending; a later wait gets its count; an unknown (or already
    collected) ticket is GZ_EINVAL."""
    g = S.rmat(14, 16, 51)
    G = gz.Graph.from_csr(g).orient()
    p = gz.Plan("chordal5")
    want = gz.count(p, G, True)
    srv = gz.Server(max_inflight=1, max_batch=4)
    t = srv.submit(p, G, True)
    with pytest.raises(gz.GzError) as e:
        srv.wait(t, timeout_ms=0)
    assert e.value.status == gz.GZ_ETIMEOUT
    assert srv.wait(t)[0] == want
    with pytest.raises(gz.GzError) as e:
        srv.wait(t, timeout_ms=0)
    assert e.value.status == gz.GZ_EINVAL
    with pytest.raises(gz.GzError) as e:
        srv.wait(987654, timeout_ms=0)
    assert e.value.status == gz.GZ_EINVAL
    srv.close()


@pytest.mark.parametrize("k", [3, 4, 5])
def test_count_motifs_against_oracle(k):
    """Motif counting (every connected k-vertex pattern, Sec. 7.1-7.2): each count
    equals the oracle's, and on a tiny graph the counts add up to the number of
    connected induced k-vertex subgraphs, found by brute force."""
    import itertools
    pats = gz.motif_patterns(k)
    for g in [S.random_small(14, 0.35, 61), S.rmat(9, 8, 62)]:
        G = gz.Graph.from_csr(g).orient()
        got = gz.count_motifs(G, k, orientation=True)
        assert got == gz.count_motifs(G, k, orientation=False)
        assert got == [oracle_count(a, g) for a in pats]
        if g.n <= 14:
            nb = [set(g.neighbors(v).tolist()) for v in range(g.n)]
            conn = 0
            for sub in itertools.combinations(range(g.n), k):
                seen, todo = {sub[0]}, [sub[0]]
                while todo:
                    v = todo.pop()
                    for u in sub:
                        if u not in seen and u in nb[v]:
                            seen.add(u)
                            todo.append(u)
                conn += len(seen) == k
            assert sum(got) == conn


@pytest.mark.parametrize("oriented", [False, True])
def test_count_merged_against_oracle(oriented):
    """One merged program for patterns of sizes 2 to 6 (shared loop-1 sets, one
    pass over the edges; cliques on the bitset kernels when oriented), repeated
    patterns included: every count equals the oracle's and the separate
    programs' counts."""
    names = ["edge", "wedge", "triangle", "path4", "star3", "c4", "paw", "diamond", "k4", "c5",
             "house", "hourglass", "chordal5", "k5", "chordal6", "asym6", "diamond", "c4"]
    for g in (S.rmat(11, 8, 31), S.random_small(60, 0.25, 32)):
        G = gz.Graph.from_csr(g).orient()
        plans = [gz.Plan(adjacency(n)) for n in names]
        got = gz.count_merged(plans, G, orientation=oriented)
        assert got == [gz.count(p, G, oriented) for p in plans]
        assert got == [oracle_count(n, g) for n in names]


def test_batch_ranges_against_oracle():
    """gz_count_batch_ranges: root ranges of general and clique queries on two
    graphs, oriented and not, in one call (empty, clamped and out-of-range
    bounds included): each range's count equals the oracle's on that range."""
    queries = []
    general = ["triangle", "paw", "c4", "diamond", "k4", "k5"]
    for g, names in ((S.rmat(12, 16, 41), general), (S.random_small(80, 0.2, 42), general + ["house"])):
        G = gz.Graph.from_csr(g).orient()
        n = g.n
        cuts = [-5, 0, 3, n // 7, n // 2, n // 2, n + 10]
        for name in names:
            p = gz.Plan(name)
            for ori in (True, False):
                for lo, hi in zip(cuts[:-1], cuts[1:]):
                    queries.append((p, G, ori, lo, hi, name, g))
    got = gz.count_batch_ranges([q[0] for q in queries], [q[1] for q in queries],
                                [q[2] for q in queries], [(q[3], q[4]) for q in queries])
    for (p, G, ori, lo, hi, name, g), c in zip(queries, got):
        lo_c, hi_c = max(lo, 0), min(hi, g.n)
        want = 0 if lo_c >= hi_c else oracle_count(name, g, oriented=ori, lo=lo_c, hi=hi_c)
        assert c == want, (name, g.name, ori, lo, hi)


def test_count_merged_split_pass():
    """Book graph (many triangles on one spine edge): the merged kernel defers
    the hub edges of several plans to its split pass."""
    pages = 3000
    e = [(0, 1)] + [(0, i) for i in range(2, pages + 2)] + [(1, i) for i in range(2, pages + 2)]
    e += [(i, i + 1) for i in range(2, pages + 1, 2)]
    g = S.from_edges(pages + 2, e, "book_pages")
    G = gz.Graph.from_csr(g).orient()
    names = ["diamond", "paw", "c4", "house", "chordal5", "k4"]
    plans = [gz.Plan(n) for n in names]
    for ori in (False, True):
        assert gz.count_merged(plans, G, orientation=ori) == [gz.count(p, G, ori) for p in plans]
    assert gz.count_merged(plans, G, orientation=True) == [oracle_count(n, g) for n in names]


def test_counts_survive_reorientation():
    """Re-orienting rebuilds the out-list view and the cached heavy-root rows in
    the same device buffers; counts before and after (and from a fresh graph)
    agree, for the clique kernels and the general kernel."""
    g = S.rmat(14, 16, 63)
    G = gz.Graph.from_csr(g).orient()
    assert G.info()["max_out_degree_oriented"] >= 128  # heavy roots exist
    names = ["k4", "k5", "diamond", "paw"]
    before = [gz.count(gz.Plan(n), G, True) for n in names]
    for _ in range(2):
        G.orient()
        assert [gz.count(gz.Plan(n), G, True) for n in names] == before
    H = gz.Graph.from_csr(g).orient()
    assert [gz.count(gz.Plan(n), H, True) for n in names] == before
    assert before[:2] == [oracle_count("k4", g), oracle_count("k5", g)]


@pytest.mark.parametrize("name", ["paw", "diamond", "house", "chordal5"])
def test_measured_schedule_keeps_counts(name):
    """Measured schedule selection picks one of Algorithm 4's distinct schedules
    by timing them on sample roots; the count must not depend on the choice."""
    g = S.rmat(11, 8, 64)
    G = gz.Graph.from_csr(g).orient()
    a = adjacency(name)
    p, best_ms, model_ms = gz.plan_measured(a, G, [(100, 164), (1000, 1256)])
    # model_ms = -1: the model's schedule took more than 4x the best and was dropped
    assert model_ms < 0 or best_ms <= model_ms + 1e-9
    order = p.info()["order"]
    assert any(list(s) == order for s in O.distinct_schedules(a))
    assert gz.count(p, G, True) == oracle_count(a, g)


def test_schedule_times_every_schedule():
    """gz_schedule_times lists Algorithm 4's schedules in generation order with
    the model's estimate of each, and every schedule counts the same instances."""
    g = S.rmat(11, 8, 64)
    G = gz.Graph.from_csr(g).orient()
    a = adjacency("paw")
    times = gz.schedule_times(a, G, [(0, g.n)], cutoff=0.0)
    assert [t["order"] for t in times] == [list(s) for s in O.distinct_schedules(a)]
    assert all(t["ms"] > 0 for t in times)
    want = oracle_count(a, g)
    for t in times:
        p = gz.Plan(a, t["order"])
        assert t["est_cost"] == pytest.approx(p.info()["est_cost"])
        assert gz.count(p, G, True) == want
    # a range split of the roots adds up under every schedule
    for t in times[:3]:
        p = gz.Plan(a, t["order"])
        assert gz.count(p, G, True, 0, 300) + gz.count(p, G, True, 300, g.n) == want


def _first_connected_order(a):
    """A valid schedule for the oracle: each vertex after the first is adjacent
    to an earlier one (the count does not depend on which valid schedule runs)."""
    k = len(a)
    order = [0]
    while len(order) < k:
        order.append(next(v for v in range(k) if v not in order and any(a[v][u] for u in order)))
    return order


def test_count_motifs_size7():
    """All 853 connected 7-vertex patterns (Sec. 1) counted in one batch: each count
    equals the oracle's, and on the 14-vertex graph they add up to the number of
    connected induced 7-vertex subgraphs, found by brute force."""
    import itertools
    pats = gz.motif_patterns(7)
    for g in [S.random_small(14, 0.35, 61), S.random_small(40, 0.15, 72)]:
        G = gz.Graph.from_csr(g).orient()
        got = gz.count_motifs(G, 7, orientation=True)
        go, _ = O.reindex(g)
        assert got == [O.count_nested(a, _first_connected_order(a), go)[0] for a in pats]
        if g.n <= 14:
            nb = [set(g.neighbors(v).tolist()) for v in range(g.n)]
            conn = 0
            for sub in itertools.combinations(range(g.n), 7):
                seen, todo = {sub[0]}, [sub[0]]
                while todo:
                    v = todo.pop()
                    for u in sub:
                        if u not in seen and u in nb[v]:
                            seen.add(u)
                            todo.append(u)
                conn += len(seen) == 7
            assert sum(got) == conn
