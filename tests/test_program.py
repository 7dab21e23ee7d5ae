"""CPU checks of the host planner and of the compiled nested-loop program.

The planner (libgz host C++) is compared with the oracle's independent planner,
and the compiled program, read back as text through gz_plan_describe, is
interpreted here in plain Python with the kernels' exact operand rules (views,
out-list classes, prefix bounds, exclusions). Its counts must equal the oracle's
on tiny graphs for every pattern and every distinct schedule. No GPU is needed.
"""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from synthetic.patterns import EDGES, adjacency

gz = pytest.importorskip("paper_1911_12877_gb300")

NAMES = ["edge", "wedge", "triangle", "path4", "star3", "c4", "paw", "diamond", "k4", "c5", "house",
         "hourglass", "chordal5", "k5", "k6", "chordal6", "asym6"]


def test_library_exports_every_declared_symbol():
    import re
    import os
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "gz.h")).read()
    declared = set(re.findall(r"^(?:gz_status|void|const char\*|uint64_t)\s+(gz_\w+)\(", hdr, re.M))
    assert declared == set(gz.EXPORTS)
    L = gz.lib()
    for name in declared:
        assert hasattr(L, name), name


@pytest.mark.parametrize("name", list(EDGES))
def test_planner_matches_oracle_planner(name):
    a = adjacency(name)
    info = gz.Plan(a).info()
    order, cost = O.choose_schedule(a)
    bp, _ = O.restrictions(a, order)
    assert info["order"] == list(order)
    assert info["bound_parent"] == list(bp)
    assert info["aut_size"] == len(O.automorphisms(a))
    assert info["est_cost"] == pytest.approx(cost, rel=1e-12)
    assert (gz.schedules(a) == O.distinct_schedules(a)).all()


def test_planner_cost_matches_hand_derived_model():
    # the library's Sec. 5.4 model against the closed forms written out by hand
    # (not the oracle's code) for the two Sec. 5.1 tailed-triangle schedules
    from test_oracle import PAW_A, PAW_B, PAW_C, PAW_D, _paw_costs_by_hand
    a = adjacency("paw")
    cdba, abcd = _paw_costs_by_hand()
    for order, want in (([PAW_C, PAW_D, PAW_B, PAW_A], cdba), ([PAW_A, PAW_B, PAW_C, PAW_D], abcd)):
        assert gz.Plan(a, order=order).info()["est_cost"] == pytest.approx(want, rel=1e-12)
    assert gz.Plan(a).info()["est_cost"] <= cdba


def test_named_patterns_match_inputs():
    for name in EDGES:
        if name == "asym6":
            continue
        assert (gz.pattern_named(name) == adjacency(name)).all(), name


def test_invalid_patterns_rejected():
    with pytest.raises(gz.GzError):
        gz.Plan(np.zeros((3, 3), dtype=np.uint8))  # disconnected
    bad = adjacency("triangle").copy()
    bad[0, 1] = 0  # asymmetric
    with pytest.raises(gz.GzError):
        gz.Plan(bad)
    with pytest.raises(gz.GzError):
        gz.Plan(np.ones((9, 9), dtype=np.uint8) - np.eye(9, dtype=np.uint8))  # k > 8
    with pytest.raises(gz.GzError):
        gz.Plan(adjacency("path4"), order=[0, 2, 1, 3])  # 2 not adjacent to 0
    with pytest.raises(gz.GzError):
        gz.pattern_named("no_such_pattern")


# ------------------------------------------------------------ program interpreter

def parse(desc):
    prog = {"ops": [], "cand": {}, "buf": {}}
    for line in desc.strip().splitlines():
        f = line.split()
        if f[0] == "unit":
            prog["unit_dag"] = int(f[1].split("=")[1])
            prog["flat"] = int(f[2].split("=")[1])
        elif f[0] == "op":
            kv = dict(x.split("=", 1) for x in f[1:])
            op = {k: int(v) for k, v in kv.items() if k != "rights"}
            op["rights"] = [tuple(map(int, r.split(":"))) for r in kv["rights"].split(",") if r]
            prog["ops"].append(op)
        elif f[0] == "cand":
            kv = {k: int(v) for k, v in (x.split("=") for x in f[1:])}
            prog["cand"][kv["d"]] = kv
        elif f[0] == "buf":
            prog["buf"][int(f[1])] = int(f[2].split("=")[1])
    return prog


class Interp:
    """Runs a compiled program the way the kernel does, one root edge at a time."""

    def __init__(self, prog, k, g, flat=False, heavy=None):
        self.p, self.k, self.g = prog, k, g
        self.flat = flat and prog["flat"] != 0 and k >= 4
        self.heavy = heavy  # None: the kernel's rule; True / False: force one path
        self.out = {v: [int(u) for u in g.neighbors(v) if u < v] for v in range(g.n)}
        self.full = {v: [int(u) for u in g.neighbors(v)] for v in range(g.n)}

    def lst(self, v, dag):
        return self.out[v] if dag else self.full[v]

    def run(self):
        k, p = self.k, self.p
        total = 0
        for e0 in range(self.g.n):
            units = self.lst(e0, p["unit_dag"])
            for i1, e1 in enumerate(units):
                emb = [None] * k
                itp = [0] * k
                emb[0], emb[1], itp[1] = e0, e1, i1
                bufs = {}
                if k == 2:
                    total += 1
                    continue
                total += self.level(1, emb, itp, bufs)
                if k > 3:
                    if self.flat and k == 4:
                        total += self.flat_last(emb, bufs)
                    else:
                        total += self.dfs(2, emb, itp, bufs)
        return total

    def flat_last(self, emb, bufs):
        """The kernel's flattened last loop over the candidates c of loop k-2."""
        k, p = self.k, self.p
        t = k - 2
        op = [o for o in p["ops"] if o["level"] == t][0]
        S = self.cands(t, emb, bufs)
        cex = p["cand"][t]["excl"] if t >= 2 else 0
        shape2 = p["flat"] == 2
        xm = op["excl"] & ~(1 << t)
        excl_self = op["excl"] >> t & 1
        bnd = op["bound"]
        if shape2:
            sdag = op["left_dag"]
        else:
            sdag = op["rights"][0][2]
            sub = bool(op["rights"][0][1])
            F = list(bufs[op["left_buf"]]) if op["left_buf"] >= 0 else \
                self.lst(emb[op["left_pos"]], op["left_dag"])
            if bnd >= 0 and bnd != t:
                F = [x for x in F if x < emb[bnd]]
        ex = lambda x: any((xm >> j & 1) and emb[j] == x for j in range(k))
        total = 0
        for idx, c in enumerate(S):
            if any((cex >> j & 1) and emb[j] == c for j in range(t)):
                continue
            beta = None if bnd < 0 else (c if bnd == t else emb[bnd])
            R = self.lst(c, sdag)
            if beta is not None and sdag != 2:
                R = [x for x in R if x < beta]
            if shape2:
                for x in R:
                    keep = all((x in set(self.lst(emb[pos], dag))) != bool(sb)
                               for pos, sb, dag in op["rights"])
                    total += keep and not ex(x)
                continue
            if bnd == t:
                Lc = idx if op["left_iter"] else sum(1 for x in F if x < c)
            else:
                Lc = len(F)
            if Lc == 0:
                continue
            heavy = len(R) > 8 * Lc + 32 if self.heavy is None else self.heavy
            if sub:
                total += Lc
                for j in range(k):
                    if (xm >> j & 1) or (j == t and excl_self):
                        e = c if j == t else emb[j]
                        if (beta is None or e < beta) and e in F[:Lc] and e not in R:
                            total -= 1
            stream, probe = (F[:Lc], set(R)) if heavy else (R, set(F))
            for x in stream:
                found = x in probe
                total += (found and not ex(x)) if not sub else -found
        return total

    def level(self, t, emb, itp, bufs):
        c = 0
        for op in self.p["ops"]:
            if op["level"] != t:
                continue
            bound = emb[op["bound"]] if op["bound"] >= 0 else None
            if op["left_buf"] >= 0:
                L = bufs[op["left_buf"]]
                if op["left_iter"]:
                    L = L[:itp[t]]
                elif bound is not None:
                    L = [x for x in L if x < bound]
            else:
                L = self.lst(emb[op["left_pos"]], op["left_dag"])
                if op["left_iter"]:
                    L = L[:itp[t]]
                elif bound is not None and op["left_dag"] != 2:
                    L = [x for x in L if x < bound]
            assert bound is None or all(x < bound for x in L)
            keep = []
            for x in L:
                ok = True
                for (pos, sub, dag) in op["rights"]:
                    f = x in set(self.lst(emb[pos], dag))
                    ok = ok and (f != bool(sub))
                if ok:
                    keep.append(x)
            if op["dst"] < 0:
                ex = [emb[j] for j in range(self.k) if op["excl"] >> j & 1]
                c += sum(1 for x in keep if x not in ex)
            else:
                bufs[op["dst"]] = keep
        return c

    def cands(self, d, emb, bufs):
        cd = self.p["cand"][d]
        if cd["buf"] >= 0:
            return list(bufs[cd["buf"]])
        L = self.lst(emb[cd["pos"]], cd["dag"])
        if cd["bound"] >= 0 and cd["dag"] != 2:
            L = [x for x in L if x < emb[cd["bound"]]]
        return L

    def dfs(self, d, emb, itp, bufs):
        c = 0
        cd = self.p["cand"][d]
        for pos, x in enumerate(self.cands(d, emb, bufs)):
            if any((cd["excl"] >> j & 1) and emb[j] == x for j in range(d)):
                continue
            emb[d], itp[d] = x, pos
            c += self.level(d, emb, itp, bufs)
            if self.flat and d == self.k - 3:
                c += self.flat_last(emb, dict(bufs))
            elif d < self.k - 2:
                c += self.dfs(d + 1, emb, itp, dict(bufs))
        return c


@pytest.mark.parametrize("name", NAMES)
def test_compiled_program_counts_every_schedule(name):
    a = adjacency(name)
    graphs = [S.random_small(9, 0.5, 11), S.random_small(10, 0.35, 12)]
    for g in graphs:
        want = O.count_brute_induced(a, g)
        go, _ = O.reindex(g)
        for s in O.distinct_schedules(a)[:10]:
            prog = parse(gz.Plan(a, order=s).describe())
            for flat, heavy in ((False, None), (True, None), (True, True), (True, False)):
                assert Interp(prog, len(a), g, flat, heavy).run() == want, (name, s, flat, heavy)
                assert Interp(prog, len(a), go, flat, heavy).run() == want, (name, s, flat, heavy, "or")


def test_clique_program_is_chain_of_out_list_intersections():
    # Orientation on cliques (Sec. 6): every loop reads whole out-lists and the
    # previous candidates below the current vertex; one buffer per loop.
    prog = parse(gz.Plan("k5").describe())
    assert prog["unit_dag"] == 1
    for op in prog["ops"]:
        assert op["left_iter"] == 1
        assert all(r[1] == 0 and r[2] == 2 for r in op["rights"])
    assert all(v == 1 for v in prog["buf"].values())


@pytest.mark.parametrize("k", [2, 3, 4, 5, 6])
def test_motif_patterns_match_oracle(k):
    """The library's motif patterns (host enumeration) are the oracle's, up to
    isomorphism, with no repeats."""
    mine = [O.canonical_form(a) for a in gz.motif_patterns(k)]
    assert len(mine) == len(set(mine))
    assert set(mine) == {O.canonical_form(a) for a in O.connected_patterns(k)}


def _connected(a) -> bool:
    k = len(a)
    seen, todo = {0}, [0]
    while todo:
        v = todo.pop()
        for u in range(k):
            if a[v][u] and u not in seen:
                seen.add(u)
                todo.append(u)
    return len(seen) == k


def test_motif_patterns_size7():
    """Sec. 1 puts the number of connected 7-vertex patterns at 853. The library's
    list has that many, each connected, no two isomorphic (the oracle's canonical
    form over all 7! relabellings), so it holds every class exactly once."""
    pats = gz.motif_patterns(7)
    assert len(pats) == 853
    for a in pats:
        assert (a == a.T).all() and not a.diagonal().any() and _connected(a)
    forms = {O.canonical_form(a) for a in pats}
    assert len(forms) == 853


def test_plan_every_size7_motif():
    """Every 7-vertex motif plans (Algorithm 4 schedules, Algorithm 1 + Theorem 2
    restrictions, Sec. 5.4 model) with a valid schedule and |Aut(P)| matching the
    oracle's."""
    pats = gz.motif_patterns(7)
    for idx, a in enumerate(pats):
        info = gz.Plan(a).info()
        assert sorted(info["order"]) == list(range(7))
        if idx % 40 == 0:
            assert info["aut_size"] == len(O.automorphisms(a))


def test_size7_motifs_planner_and_program_match_oracle():
    """A spread sample of the 853 size-7 motifs: the library's plan equals the
    oracle planner's (schedule, Theorem 2 bound parents, |Aut(P)|, Sec. 5.4 cost),
    and its compiled program, interpreted with the kernels' operand rules, counts
    what brute force over all 7-subsets counts (Sec. 2.1 definition)."""
    pats = gz.motif_patterns(7)
    # sparse, medium and dense, so that most sampled patterns occur in one of them
    graphs = [S.random_small(13, 0.3, 31), S.random_small(13, 0.5, 32), S.random_small(13, 0.7, 33)]
    for idx in range(0, len(pats), 17):
        a = pats[idx]
        info = gz.Plan(a).info()
        order, cost = O.choose_schedule(a)
        bp, _ = O.restrictions(a, order)
        assert info["order"] == list(order), idx
        assert info["bound_parent"] == list(bp), idx
        assert info["aut_size"] == len(O.automorphisms(a)), idx
        assert info["est_cost"] == pytest.approx(cost, rel=1e-12), idx
        prog = parse(gz.Plan(a).describe())
        for g in graphs:
            want = O.count_brute_induced(a, g)
            go, _ = O.reindex(g)
            for flat in (False, True):
                assert Interp(prog, 7, g, flat, None).run() == want, (idx, flat)
                assert Interp(prog, 7, go, flat, None).run() == want, (idx, flat, "oriented")
