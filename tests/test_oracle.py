"""Pins for the CPU oracle: values the paper prints, closed forms, identities,
brute force on tiny graphs, and planted mistakes that these pins must catch.

Nothing here calls the CUDA library. Every expected value comes from the paper
(cited by section) or from mathematics independent of the oracle's code.
"""
import itertools
import math

import numpy as np
import pytest

import oracle as O
import synthetic as S
from synthetic.patterns import EDGES, adjacency

SCHEDULE_TABLE = {
    # pattern: (|Aut|, valid schedules K, distinct schedules K/|Aut|)
    "wedge": (2, 4, 2), "triangle": (6, 6, 1), "path4": (2, 8, 4), "star3": (6, 12, 2),
    "c4": (8, 16, 2), "paw": (2, 14, 7), "diamond": (4, 20, 5), "k4": (24, 24, 1),
    "house": (2, 60, 30), "chordal5": (12, 108, 9), "c5": (10, 40, 4), "k5": (120, 120, 1),
    "k6": (720, 720, 1), "chordal6": (48, 672, 14),
}
SMALL = ["wedge", "triangle", "path4", "star3", "c4", "paw", "diamond", "k4", "c5", "house",
         "hourglass", "chordal5", "k5", "asym6"]


# ------------------------------------------------------------------ planner pins

def test_aut_sizes_from_paper():
    # Sec. 2.2: a rectangle instance has 8 mappings.
    assert len(O.automorphisms(adjacency("c4"))) == 8
    # Sec. 1 / Sec. 7.2: AutoMine finds each size-7 chordal cycle 120 times after
    # halving by root symmetry, so |Aut(K7 - e)| = 240.
    assert len(O.automorphisms(adjacency("chordal7"))) == 240
    # Sec. 7.2: the best case for the pentagon is 5x = |Aut(C5)| / 2.
    assert len(O.automorphisms(adjacency("c5"))) == 10


@pytest.mark.parametrize("n", [3, 4, 5, 6])
def test_aut_closed_forms(n):
    clique = adjacency([(i, j) for i in range(n) for j in range(i + 1, n)], n)
    assert len(O.automorphisms(clique)) == math.factorial(n)
    cyc = adjacency([(i, (i + 1) % n) for i in range(n)], n)
    assert len(O.automorphisms(cyc)) == (2 * n if n > 2 else 2)
    if n >= 3:
        kme = adjacency([(i, j) for i in range(n) for j in range(i + 1, n) if (i, j) != (0, 1)], n)
        assert len(O.automorphisms(kme)) == 2 * math.factorial(n - 2)


def test_automorphisms_preserve_structure():
    for name in SMALL:
        a = adjacency(name)
        for x in O.automorphisms(a):
            assert sorted(x) == list(range(len(a)))
            assert (a[np.ix_(x, x)] == a).all()


@pytest.mark.parametrize("name", sorted(SCHEDULE_TABLE))
def test_schedule_counts(name):
    a = adjacency(name)
    aut, K, D = SCHEDULE_TABLE[name]
    assert len(O.automorphisms(a)) == aut
    valid = O.valid_schedules_brute(a)
    assert len(valid) == K
    # Sec. 5.3 / Theorem 3: Algorithm 4 returns exactly K / |Aut| schedules ...
    dist = O.distinct_schedules(a)
    assert len(dist) == D == K // aut
    # ... every one valid, no two equivalent, and every valid schedule equivalent to one.
    auts = O.automorphisms(a)
    vset = {tuple(s) for s in valid}
    canon = set()
    for s in dist:
        assert tuple(s) in vset
        orbit = {tuple(int(x[v]) for v in s) for x in auts}
        assert not (orbit & canon)
        canon |= orbit
    assert canon == vset


@pytest.mark.parametrize("n", [3, 4, 5, 6])
def test_path_and_clique_schedule_counts(n):
    path = adjacency([(i, i + 1) for i in range(n - 1)], n)
    assert len(O.valid_schedules_brute(path)) == 2 ** (n - 1)
    assert len(O.distinct_schedules(path)) == 2 ** (n - 2)
    # Sec. 5.2: all n! orders of a clique are valid and (Sec. 5.3) all equivalent.
    clique = adjacency([(i, j) for i in range(n) for j in range(i + 1, n)], n)
    assert len(O.valid_schedules_brute(clique)) == math.factorial(n)
    assert len(O.distinct_schedules(clique)) == 1


def test_tailed_triangle_equivalence():
    # Sec. 5.3: (A,B,C,D) and (A,B,D,C) are equivalent for the tailed triangle
    # (A = tail end, B = its degree-3 neighbour, C and D the other triangle vertices).
    a = adjacency("paw")  # edges 01 12 02 23: tail 3, centre 2
    A, B, C, D = 3, 2, 0, 1
    s1, s2 = (A, B, C, D), (A, B, D, C)
    auts = O.automorphisms(a)
    assert any(tuple(int(x[v]) for v in s1) == s2 for x in auts)
    dist = {tuple(map(int, s)) for s in O.distinct_schedules(a)}
    assert len(dist & {s1, s2}) == 1


def test_rectangle_partial_order():
    # Sec. 4.2: schedule (A,B,C,D) of the rectangle with B, C the neighbours of A
    # gives {(A,B), (A,C), (A,D), (B,C)}; Theorem 2 keeps one bound per vertex.
    A, B, C, D = 0, 1, 2, 3
    rect = adjacency([(A, B), (A, C), (B, D), (C, D)], 4)
    bp, L = O.restrictions(rect, [A, B, C, D])
    assert set(L) == {(A, B), (A, C), (A, D), (B, C)}
    assert list(bp) == [-1, 0, 1, 0]  # B < A, C < B, D < A


def test_restriction_probability_is_inverse_multiplicity():
    # Appendix: over the whole schedule prod 1/z_i = 1/|Aut|; rectangle = 1/4 * 1/2.
    A, B, C, D = 0, 1, 2, 3
    rect = adjacency([(A, B), (A, C), (B, D), (C, D)], 4)
    bp, _ = O.restrictions(rect, [A, B, C, D])
    assert O.restriction_probability(bp, 3) == pytest.approx(1 / 8)
    for name in SMALL:
        a = adjacency(name)
        aut = len(O.automorphisms(a))
        for s in O.distinct_schedules(a):
            bp, _ = O.restrictions(a, s)
            assert O.restriction_probability(bp, len(a) - 1) == pytest.approx(1.0 / aut)


def test_theorem2_bound_parents_precede():
    # Theorem 2 proof: a relation (S[a], S[b]) always has a < b.
    for name in SMALL:
        a = adjacency(name)
        for s in O.distinct_schedules(a):
            bp, L = O.restrictions(a, s)
            pos = {int(v): i for i, v in enumerate(s)}
            for (u, w) in L:
                assert pos[u] < pos[w]
            for i, p in enumerate(bp):
                assert p < i


def test_cost_model_prefers_triangle_first_for_tailed_triangle():
    # Sec. 5.1: [C,D,B,A] runs its innermost loop once per triangle, [A,B,C,D]
    # once per wedge; the model must rank the triangle-first schedule cheaper.
    a = adjacency("paw")
    A, B, C, D = 3, 2, 0, 1
    assert O.cost(a, [C, D, B, A]) < O.cost(a, [A, B, C, D])
    best, c = O.choose_schedule(a)
    assert c == pytest.approx(min(O.cost(a, s) for s in O.distinct_schedules(a)))


def _paw_costs_by_hand():
    """The Sec. 5.4 model for the two tailed-triangle schedules of Sec. 5.1, written
    out by hand in exact rationals (n = 1000 vertices, p = 5/999 from Sec. 7.3).

    Labels: C = 0, D = 1 (the triangle corners without the tail), B = 2 (the
    corner with the tail), A = 3 (the tail). Aut = {id, (C D)}, so each schedule
    keeps one restriction id(D) < id(C).

    [C, D, B, A]: loop iterations n; n p (D ~ C); n p^2 (B ~ C, D);
    n p (1-p)^2 (A ~ B only). The restriction binds D under C from loop 1 on,
    so loops 1..3 pass it with probability 1/2 (Appendix: prod 1/z_i, z_C = 2).

    [A, B, C, D]: loop iterations n; n p (B ~ A); n p (1-p) (C ~ B, not A);
    n p^2 (1-p) (D ~ B, C, not A). The restriction binds D under C in loop 3
    only, passed with probability 1/2.

    Cost = sum over loops of (product of iterations down to that loop) x the
    restriction pass probability of that loop."""
    from fractions import Fraction as Fr
    n, p = Fr(1000), Fr(5, 999)
    q = 1 - p
    h = Fr(1, 2)
    l1, l2, l3 = n * p, n * p ** 2, n * p * q ** 2
    cdba = n + n * l1 * h + n * l1 * l2 * h + n * l1 * l2 * l3 * h
    m1, m2, m3 = n * p, n * p * q, n * p ** 2 * q
    abcd = n + n * m1 + n * m1 * m2 + n * m1 * m2 * m3 * h
    return float(cdba), float(abcd)


PAW_C, PAW_D, PAW_B, PAW_A = 0, 1, 2, 3


def test_cost_model_closed_form_tailed_triangle():
    a = adjacency("paw")
    cdba, abcd = _paw_costs_by_hand()
    s1, s2 = [PAW_C, PAW_D, PAW_B, PAW_A], [PAW_A, PAW_B, PAW_C, PAW_D]
    assert list(O.restrictions(a, s1)[0]) == [-1, 0, -1, -1]
    assert list(O.restrictions(a, s2)[0]) == [-1, -1, -1, 2]
    assert O.cost(a, s1) == pytest.approx(cdba, rel=1e-12)
    assert O.cost(a, s2) == pytest.approx(abcd, rel=1e-12)
    assert cdba < abcd  # Sec. 5.1: the triangle-first schedule is the better one


# ------------------------------------------------------------------ Oracle A closed forms

@pytest.mark.parametrize("k", [2, 3, 4, 5, 6])
def test_cliques_in_complete_graph(k):
    g = S.complete(8)
    a = adjacency([(i, j) for i in range(k) for j in range(i + 1, k)], k)
    assert O.count_brute_induced(a, g) == math.comb(8, k)
    order, _ = O.choose_schedule(a)
    assert O.count_nested(a, order, g)[0] == math.comb(8, k)


def test_closed_forms_structured_graphs():
    K7 = S.complete(7)
    for name in ["c4", "diamond", "paw", "wedge", "house", "chordal5"]:
        assert O.count_brute_induced(adjacency(name), K7) == 0
    assert O.count_brute_induced(adjacency("chordal5"), S.complete(5)) == 0
    P = S.petersen()  # girth 5: 12 five-cycles, all induced
    assert O.count_brute_induced(adjacency("c5"), P) == 12
    assert O.count_brute_induced(adjacency("triangle"), P) == 0
    assert O.count_brute_induced(adjacency("c4"), P) == 0
    assert O.count_brute_induced(adjacency("c5"), S.cycle(5)) == 1
    assert O.count_brute_induced(adjacency("c4"), S.cycle(4)) == 1
    assert O.count_brute_induced(adjacency("c4"), S.complete_bipartite(3, 4)) == 3 * 6
    st = S.star(7)
    assert O.count_brute_induced(adjacency("star3"), st) == math.comb(7, 3)
    assert O.count_brute_induced(adjacency("wedge"), st) == math.comb(7, 2)
    assert O.count_brute_induced(adjacency("triangle"), S.empty(9)) == 0


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_triangles_trace_formula(seed):
    g = S.random_small(12, 0.5, seed)
    A = np.zeros((g.n, g.n), dtype=np.int64)
    for v in range(g.n):
        A[v, g.neighbors(v)] = 1
    tri = int(np.trace(A @ A @ A)) // 6
    a = adjacency("triangle")
    assert O.count_brute_induced(a, g) == tri
    assert O.count_nested(a, [0, 1, 2], g)[0] == tri


def _nested(name, g):
    a = adjacency(name)
    order, _ = O.choose_schedule(a)
    return O.count_nested(a, order, g)[0]


@pytest.mark.parametrize("seed,n,p", [(5, 40, 0.25), (6, 60, 0.12)])
def test_induced_noninduced_identities(seed, n, p):
    g = S.random_small(n, p, seed)
    A = np.zeros((n, n), dtype=np.int64)
    for v in range(n):
        A[v, g.neighbors(v)] = 1
    d = A.sum(1)
    m = int(A.sum()) // 2
    A2 = A @ A
    c = {k: _nested(k, g) for k in ["wedge", "triangle", "c4", "diamond", "k4", "paw", "star3"]}
    tri = int(np.trace(A2 @ A)) // 6
    assert c["triangle"] == tri
    assert int((d * (d - 1) // 2).sum()) == c["wedge"] + 3 * c["triangle"]
    four_cycles = (int(np.trace(A2 @ A2)) - 4 * int((d * (d - 1) // 2).sum()) - 2 * m) // 8
    assert four_cycles == c["c4"] + c["diamond"] + 3 * c["k4"]
    te = A2[A > 0]  # triangles on each directed edge
    assert int((te * (te - 1) // 2).sum()) // 2 == c["diamond"] + 6 * c["k4"]
    assert int((d * (d - 1) * (d - 2) // 6).sum()) == c["star3"] + c["paw"] + 2 * c["diamond"] + 4 * c["k4"]
    s = 0
    for u in range(n):
        for v in range(u + 1, n):
            for w in range(v + 1, n):
                if A[u, v] and A[v, w] and A[u, w]:
                    s += d[u] + d[v] + d[w] - 6
    assert s == c["paw"] + 4 * c["diamond"] + 12 * c["k4"]


# ------------------------------------------------------------------ Oracle B vs A

GRAPHS = [(10, 0.45, 1), (11, 0.45, 2), (9, 0.7, 3), (12, 0.3, 4)]


@pytest.mark.parametrize("name", SMALL)
def test_nested_equals_brute_every_schedule(name):
    a = adjacency(name)
    aut = len(O.automorphisms(a))
    for (n, p, seed) in GRAPHS:
        g = S.random_small(n, p, seed)
        want = O.count_brute_induced(a, g)
        if len(a) <= 5 or n <= 10:
            # Theorem 1 invariant: restricted count times |Aut| = unrestricted count.
            assert O.count_brute_injective(a, g) == want * aut
        go, _ = O.reindex(g)
        for s in O.distinct_schedules(a)[:12]:
            assert O.count_nested(a, s, g)[0] == want
            assert O.count_nested(a, s, go)[0] == want


@pytest.mark.parametrize("name", ["wedge", "triangle", "c4", "paw", "diamond", "house", "k4",
                                  "chordal5", "asym6"])
def test_elems_match_brute_definition(name):
    a = adjacency(name)
    g = S.random_small(9, 0.5, 7)
    for s in O.distinct_schedules(a)[:6]:
        assert O.count_nested(a, s, g)[1] == O.elems_brute(a, s, g)


@pytest.mark.parametrize("name", ["edge", "wedge", "triangle", "c4", "paw", "house", "k4", "k5",
                                  "chordal5", "asym6"])
def test_elems_without_last_loop_equal_plain_elems(name):
    a = adjacency(name)
    for g in [S.random_small(12, 0.5, 3), S.rmat(8, 8, 4)]:
        for og in [g, O.reindex(g)[0]]:
            for s in O.distinct_schedules(a)[:4]:
                assert O.elems_nested(a, s, og) == O.count_nested(a, s, og)[1]
                assert O.elems_nested(a, s, og, 3, 40) == O.count_nested(a, s, og, 3, 40)[1]


def test_root_ranges_partition_the_count():
    a = adjacency("diamond")
    g = S.random_small(40, 0.3, 9)
    order, _ = O.choose_schedule(a)
    total = O.count_nested(a, order, g)
    parts = [O.count_nested(a, order, g, lo, lo + 7) for lo in range(0, 40, 7)]
    assert sum(p[0] for p in parts) == total[0]
    assert sum(p[1] for p in parts) == total[1]


# ------------------------------------------------------------------ orientation

@pytest.mark.parametrize("seed", [1, 2])
def test_reindex_orders_by_degree(seed):
    g = S.random_small(50, 0.15, seed)
    go, nid = O.reindex(g)
    assert sorted(nid.tolist()) == list(range(g.n))
    d_old = g.degrees()
    d_new = go.degrees()
    old_of = np.argsort(nid)
    assert (d_new == d_old[old_of]).all()
    for r in range(g.n - 1):  # degree descending, ties by original id ascending
        assert d_new[r] > d_new[r + 1] or (d_new[r] == d_new[r + 1] and old_of[r] < old_of[r + 1])
    for v in range(g.n):
        assert go.neighbors(nid[v]).tolist() == sorted(nid[g.neighbors(v)].tolist())


def test_orientation_hub_list_shrinks():
    # Sec. 6: on a star whose hub has the largest id, reindexing gives the hub
    # id 0, so every bound below it empties its list and E drops.
    g = S.from_edges(21, [(20, i) for i in range(20)], "star_hub_last")
    go, nid = O.reindex(g)
    assert nid[20] == 0
    a = adjacency("triangle")
    _, e_plain = O.count_nested(a, [0, 1, 2], g)
    _, e_or = O.count_nested(a, [0, 1, 2], go)
    assert e_or < e_plain


# ------------------------------------------------------------------ planted mistakes

def _pins_pass():
    try:
        test_aut_sizes_from_paper()
        test_rectangle_partial_order()
        test_restriction_probability_is_inverse_multiplicity()
        for name in ["c4", "house", "paw", "asym6", "wedge", "diamond"]:
            test_nested_equals_brute_every_schedule(name)
        for name in ["house", "triangle", "k4"]:
            test_elems_match_brute_definition(name)
        test_reindex_orders_by_degree(1)
        for k in SCHEDULE_TABLE:
            test_schedule_counts(k)
        test_cost_model_closed_form_tailed_triangle()
    except AssertionError:
        return False
    return True


@pytest.mark.parametrize("mutation", [m for m in O.MUTATIONS if m != "none"])
def test_planted_mistakes_are_caught(mutation):
    O.set_mutation(mutation)
    try:
        assert not _pins_pass(), f"mutation {mutation} slipped through the pins"
    finally:
        O.set_mutation("none")
    assert _pins_pass()


# ------------------------------------------------------------------ motif patterns

def test_motif_pattern_counts():
    # Sec. 7.2: 2 patterns on 3 vertices, 21 on 5; Sec. 1: 112 size-6 patterns
    assert [len(O.connected_patterns(k)) for k in (3, 5, 6)] == [2, 21, 112]
    # the connected graphs on 3 and 4 vertices are exactly the named ones
    for k, names in [(3, ["wedge", "triangle"]),
                     (4, ["path4", "star3", "c4", "paw", "diamond", "k4"])]:
        forms = {O.canonical_form(a) for a in O.connected_patterns(k)}
        assert forms == {O.canonical_form(adjacency(n)) for n in names}
        assert len(forms) == len(names)


def test_motif_patterns_are_connected_and_distinct():
    for k in (4, 5):
        pats = O.connected_patterns(k)
        forms = [O.canonical_form(a) for a in pats]
        assert len(set(forms)) == len(pats)
        for a in pats:
            assert (a == a.T).all() and not a.diagonal().any()
            assert len(O.automorphisms(a)) >= 1  # the oracle accepts it as a connected pattern


# ------------------------------------------------------------------ bitset work measure

def _bitset_work_brute(k, g):
    """Word operations of the per-root bitset clique walk, by plain enumeration:
    every chain of out-list indices a > b > ... (2 to k-2 of them, pairwise
    adjacent in the graph) builds one set whose last index lim bounds it, and
    that set spans ceil(lim / 32) words. Also counts the k-cliques."""
    words = cnt = 0
    for v in range(g.n):
        out = [int(u) for u in g.neighbors(v) if u < v]
        if len(out) < k - 1:
            continue
        nb = [set(int(x) for x in g.neighbors(u)) for u in out]

        def chains(ch):
            nonlocal words, cnt
            if len(ch) == k - 1:  # a k-clique: one bit of the last loop's set
                cnt += 1
                return
            if len(ch) >= 2:  # a chain of 2 .. k-2 indices builds one set
                words += (ch[-1] + 31) // 32
            for c in range(ch[-1]):
                if all(out[c] in nb[x] for x in ch):
                    chains(ch + [c])
        for a in range(len(out)):
            chains([a])
    return cnt, words


@pytest.mark.parametrize("k", [4, 5, 6])
def test_clique_bitset_work_matches_brute_definition(k):
    import math
    for g in (S.complete(40), S.random_small(70, 0.45, 31), S.rmat(8, 16, 3)):
        go, _ = O.reindex(g)
        cnt, words = O.clique_bitset_work(k, go)
        bc, bw = _bitset_work_brute(k, go)
        assert (cnt, words) == (bc, bw), (g.name, k)
        if g.name == "K40":
            assert cnt == math.comb(40, k)
