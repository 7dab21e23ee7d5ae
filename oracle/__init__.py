"""CPU oracle for GraphZero pattern counting (arXiv 1911.12877).

TEST INFRASTRUCTURE. Only the tests, ``__graft_entry__.smoke()`` and the bench's
CPU-baseline / reference legs may import this package. The product path (the CUDA
library and its Python binding) never imports, links or runs it, and it shares no
code with the product.

The C source ``gz_oracle.c`` holds the plain implementations and cites the paper
passage each one follows. This module compiles it with gcc and exposes thin
ctypes wrappers. Patterns are k x k uint8 adjacency matrices; schedules are
label orders; graphs are ``synthetic.Csr``.
"""
from __future__ import annotations

import ctypes
import functools
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gz_oracle.c")
_LIB = os.path.join(_HERE, "libgz_oracle.so")

MUTATIONS = {
    "none": 0, "drop_red": 1, "no_bound": 2, "no_exclude": 3, "bound_le": 4,
    "alg1_nostab": 5, "thm2_first": 6, "aut_next_only": 7, "reindex_asc": 8, "e_full": 9,
    "cost_no_diff": 10, "cost_exp": 11, "cost_product": 12,
}


def build() -> str:
    """Compiles the oracle (gcc -O2, OpenMP); returns the library path."""
    if (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_u8p = ctypes.POINTER(ctypes.c_uint8)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u64p = ctypes.POINTER(ctypes.c_uint64)


@functools.lru_cache(maxsize=None)
def _lib():
    lib = ctypes.CDLL(build())
    I, L = ctypes.c_int, ctypes.c_int64
    lib.orc_set_mutation.argtypes = [I]
    lib.orc_threads.restype = I
    lib.orc_automorphisms.argtypes = [I, _u8p, _i32p, I]
    lib.orc_restrictions.argtypes = [I, _u8p, _i32p, _i32p, _i32p, I]
    lib.orc_valid_schedules_brute.argtypes = [I, _u8p, _i32p, I]
    lib.orc_distinct_schedules.argtypes = [I, _u8p, _i32p, I]
    lib.orc_restriction_probability.argtypes = [I, _i32p, I]
    lib.orc_restriction_probability.restype = ctypes.c_double
    lib.orc_cost.argtypes = [I, _u8p, _i32p]
    lib.orc_cost.restype = ctypes.c_double
    lib.orc_choose_schedule.argtypes = [I, _u8p, _i32p, ctypes.POINTER(ctypes.c_double)]
    lib.orc_count_brute_induced.argtypes = [I, _u8p, L, _i64p, _i32p, _u64p]
    lib.orc_count_brute_injective.argtypes = [I, _u8p, L, _i64p, _i32p, _u64p]
    lib.orc_count_nested.argtypes = [I, _u8p, _i32p, L, _i64p, _i32p, L, L, I, _u64p, _u64p]
    lib.orc_elems_nested.argtypes = [I, _u8p, _i32p, L, _i64p, _i32p, L, L, I, _u64p]
    lib.orc_elems_brute.argtypes = [I, _u8p, _i32p, L, _i64p, _i32p, _u64p]
    lib.orc_reindex.argtypes = [L, _i64p, _i32p, _i64p, _i32p, _i32p]
    lib.orc_connected_patterns.argtypes = [I, _u8p, I]
    lib.orc_clique_bitset_work.argtypes = [I, L, _i64p, _i32p, L, L, I, _u64p, _u64p]
    lib.orc_canonical_form.argtypes = [I, _u8p, _u8p]
    return lib


def _adj(adj):
    a = np.ascontiguousarray(np.asarray(adj, dtype=np.uint8))
    return a, a.shape[0], a.ctypes.data_as(_u8p)


def _order(order):
    o = np.ascontiguousarray(np.asarray(order, dtype=np.int32))
    return o, o.ctypes.data_as(_i32p)


def _csr(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    if col.size == 0:
        col = np.zeros(1, dtype=np.int32)
    return rp, col, rp.ctypes.data_as(_i64p), col.ctypes.data_as(_i32p)


def _check(rc, what):
    if rc < 0:
        raise ValueError(f"oracle {what} failed with code {rc}")
    return rc


def set_mutation(name: str) -> None:
    _lib().orc_set_mutation(MUTATIONS[name])


def threads() -> int:
    return _lib().orc_threads()


def automorphisms(adj) -> np.ndarray:
    a, k, ap = _adj(adj)
    n = _check(_lib().orc_automorphisms(k, ap, None, 0), "automorphisms")
    out = np.zeros((n, k), dtype=np.int32)
    _lib().orc_automorphisms(k, ap, out.ctypes.data_as(_i32p), n)
    return out


def restrictions(adj, order):
    """(bp, L): bp[i] = schedule position bounding position i (-1 none); L = label pairs."""
    a, k, ap = _adj(adj)
    o, op = _order(order)
    bp = np.zeros(k, dtype=np.int32)
    pairs = np.zeros((64, 2), dtype=np.int32)
    n = _check(_lib().orc_restrictions(k, ap, op, bp.ctypes.data_as(_i32p),
                                       pairs.ctypes.data_as(_i32p), 64), "restrictions")
    return bp, [tuple(map(int, p)) for p in pairs[:n]]


def _schedules(fn, adj):
    a, k, ap = _adj(adj)
    n = _check(fn(k, ap, None, 0), "schedules")
    out = np.zeros((max(n, 1), k), dtype=np.int32)
    fn(k, ap, out.ctypes.data_as(_i32p), n)
    return out[:n]


def valid_schedules_brute(adj) -> np.ndarray:
    return _schedules(_lib().orc_valid_schedules_brute, adj)


def distinct_schedules(adj) -> np.ndarray:
    return _schedules(_lib().orc_distinct_schedules, adj)


def restriction_probability(bp, d: int) -> float:
    b = np.ascontiguousarray(np.asarray(bp, dtype=np.int32))
    return _lib().orc_restriction_probability(b.shape[0], b.ctypes.data_as(_i32p), d)


def cost(adj, order) -> float:
    a, k, ap = _adj(adj)
    o, op = _order(order)
    return _lib().orc_cost(k, ap, op)


def choose_schedule(adj):
    a, k, ap = _adj(adj)
    out = np.zeros(k, dtype=np.int32)
    c = ctypes.c_double()
    _check(_lib().orc_choose_schedule(k, ap, out.ctypes.data_as(_i32p), ctypes.byref(c)), "choose")
    return out, c.value


def count_brute_induced(adj, g) -> int:
    a, k, ap = _adj(adj)
    rp, col, rpp, colp = _csr(g)
    out = ctypes.c_uint64()
    _check(_lib().orc_count_brute_induced(k, ap, g.n, rpp, colp, ctypes.byref(out)), "brute")
    return out.value


def count_brute_injective(adj, g) -> int:
    a, k, ap = _adj(adj)
    rp, col, rpp, colp = _csr(g)
    out = ctypes.c_uint64()
    _check(_lib().orc_count_brute_injective(k, ap, g.n, rpp, colp, ctypes.byref(out)), "injective")
    return out.value


def count_nested(adj, order, g, root_lo: int = 0, root_hi: int | None = None,
                 nthreads: int = 0):
    """Oracle B: (count, E) for roots in [root_lo, root_hi)."""
    a, k, ap = _adj(adj)
    o, op = _order(order)
    rp, col, rpp, colp = _csr(g)
    cnt, el = ctypes.c_uint64(), ctypes.c_uint64()
    hi = g.n if root_hi is None else root_hi
    _check(_lib().orc_count_nested(k, ap, op, g.n, rpp, colp, root_lo, hi, nthreads,
                                   ctypes.byref(cnt), ctypes.byref(el)), "nested")
    return cnt.value, el.value


def elems_nested(adj, order, g, root_lo: int = 0, root_hi: int | None = None,
                 nthreads: int = 0) -> int:
    """E of Oracle B for roots in [root_lo, root_hi), without building the last loop's sets."""
    a, k, ap = _adj(adj)
    o, op = _order(order)
    rp, col, rpp, colp = _csr(g)
    el = ctypes.c_uint64()
    hi = g.n if root_hi is None else root_hi
    _check(_lib().orc_elems_nested(k, ap, op, g.n, rpp, colp, root_lo, hi, nthreads,
                                   ctypes.byref(el)), "elems_nested")
    return el.value


def elems_brute(adj, order, g) -> int:
    a, k, ap = _adj(adj)
    o, op = _order(order)
    rp, col, rpp, colp = _csr(g)
    out = ctypes.c_uint64()
    _check(_lib().orc_elems_brute(k, ap, op, g.n, rpp, colp, ctypes.byref(out)), "elems")
    return out.value


def reindex(g):
    """Sec. 6 orientation relabelling: returns (relabelled Csr, new_id[old])."""
    from synthetic import Csr  # input container only
    rp, col, rpp, colp = _csr(g)
    rp2 = np.zeros(g.n + 1, dtype=np.int64)
    col2 = np.zeros(max(g.nnz, 1), dtype=np.int32)
    nid = np.zeros(max(g.n, 1), dtype=np.int32)
    _check(_lib().orc_reindex(g.n, rpp, colp, rp2.ctypes.data_as(_i64p),
                              col2.ctypes.data_as(_i32p), nid.ctypes.data_as(_i32p)), "reindex")
    return Csr(g.n, rp2, col2[:g.nnz], g.name + "_oriented"), nid[:g.n]


def clique_bitset_work(k: int, g, root_lo: int = 0, root_hi: int | None = None,
                       nthreads: int = 0):
    """(count, words): the k-clique count found by the per-root bitset walk on the
    reindexed graph g, and its 32-bit word operations (see gz_oracle.c). A work
    measure for bitset kernels, not part of the method."""
    rp, col, rpp, colp = _csr(g)
    cnt, words = ctypes.c_uint64(), ctypes.c_uint64()
    hi = g.n if root_hi is None else root_hi
    _check(_lib().orc_clique_bitset_work(k, g.n, rpp, colp, root_lo, hi, nthreads, ctypes.byref(cnt),
                                         ctypes.byref(words)), "clique_bitset_work")
    return cnt.value, words.value


def connected_patterns(k: int) -> list:
    """Every connected k-vertex graph up to isomorphism (motif patterns, Sec. 7.1),
    each in canonical form, by brute force over edge subsets and relabellings."""
    n = _check(_lib().orc_connected_patterns(k, None, 0), "connected_patterns")
    out = np.zeros(n * k * k, dtype=np.uint8)
    _lib().orc_connected_patterns(k, out.ctypes.data_as(_u8p), n)
    return [out[i * k * k:(i + 1) * k * k].reshape(k, k).copy() for i in range(n)]


def canonical_form(adj) -> bytes:
    """Canonical form of a small graph: the largest adjacency string over all relabellings."""
    a, k, ap = _adj(adj)
    out = np.zeros(k * k, dtype=np.uint8)
    _check(_lib().orc_canonical_form(k, ap, out.ctypes.data_as(_u8p)), "canonical_form")
    return out.tobytes()
