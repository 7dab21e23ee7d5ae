"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module only builds graphs. It holds none of the counting method's arithmetic:
no patterns, no restrictions, no orientation, no set operations. Graphs come back as
``Csr(n, row_ptr int64[n+1], col int32[nnz])`` with sorted, deduplicated, symmetric
lists and no self-loops.

Workload recipes (the paper's datasets are not available, so these stand in for them):

* ``er_triangle()``: Erdos-Renyi G(4096, 16/4095), seed 1 (average degree 16).
* ``rmat(scale, ef, seed)``: R-MAT with (a, b, c, d) = (0.57, 0.19, 0.19, 0.05),
  ef * 2^scale samples, seeded random relabel, then symmetrise / dedup / sort.
"""
from __future__ import annotations

import ctypes
import functools
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gz_synth.c")
_LIB = os.path.join(_HERE, "libgz_synth.so")

RMAT_ABCD = (0.57, 0.19, 0.19, 0.05)


@dataclass(frozen=True)
class Csr:
    n: int
    row_ptr: np.ndarray  # int64 [n+1]
    col: np.ndarray  # int32 [nnz]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    @property
    def m(self) -> int:
        """Undirected edge count."""
        return self.nnz // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def neighbors(self, v: int) -> np.ndarray:
        return self.col[self.row_ptr[v]:self.row_ptr[v + 1]]


def build() -> str:
    """Compiles the generator library (gcc, OpenMP); returns its path."""
    if (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


@functools.lru_cache(maxsize=None)
def _lib():
    lib = ctypes.CDLL(build())
    i64p = ctypes.POINTER(ctypes.c_int64)
    i32p = ctypes.POINTER(ctypes.c_int32)
    out = [ctypes.POINTER(i64p), ctypes.POINTER(i32p), i64p]
    lib.gzs_erdos_renyi.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_uint64] + out
    lib.gzs_rmat.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                             ctypes.c_double, ctypes.c_uint64] + out
    lib.gzs_from_edges.argtypes = [ctypes.c_int64, ctypes.c_int64, i32p, i32p] + out
    lib.gzs_free.argtypes = [ctypes.c_void_p]
    lib.gzs_threads.restype = ctypes.c_int
    return lib


def _take(n, fn, *args, name="") -> Csr:
    lib = _lib()
    rp = ctypes.POINTER(ctypes.c_int64)()
    cp = ctypes.POINTER(ctypes.c_int32)()
    nnz = ctypes.c_int64()
    rc = fn(*args, ctypes.byref(rp), ctypes.byref(cp), ctypes.byref(nnz))
    if rc != 0:
        raise RuntimeError(f"synthetic generator failed with code {rc}")
    try:
        row_ptr = np.ctypeslib.as_array(rp, shape=(n + 1,)).copy()
        col = (np.ctypeslib.as_array(cp, shape=(nnz.value,)).copy() if nnz.value > 0
               else np.zeros(0, dtype=np.int32))
    finally:
        lib.gzs_free(ctypes.cast(rp, ctypes.c_void_p))
        lib.gzs_free(ctypes.cast(cp, ctypes.c_void_p))
    return Csr(n, row_ptr, col, name)


@functools.lru_cache(maxsize=8)
def erdos_renyi(n: int, p: float, seed: int) -> Csr:
    return _take(n, _lib().gzs_erdos_renyi, n, p, seed, name=f"er_n{n}_p{p:.6g}_s{seed}")


@functools.lru_cache(maxsize=4)
def rmat(scale: int, ef: int, seed: int) -> Csr:
    a, b, c, _ = RMAT_ABCD
    return _take(1 << scale, _lib().gzs_rmat, scale, ef, a, b, c, seed,
                 name=f"rmat_s{scale}_ef{ef}_seed{seed}")


def from_edges(n: int, edges, name: str = "") -> Csr:
    e = np.asarray(edges, dtype=np.int32).reshape(-1, 2)
    s = np.ascontiguousarray(e[:, 0])
    d = np.ascontiguousarray(e[:, 1])
    i32p = ctypes.POINTER(ctypes.c_int32)
    return _take(n, _lib().gzs_from_edges, n, e.shape[0], s.ctypes.data_as(i32p),
                 d.ctypes.data_as(i32p), name=name)


# --- workload presets -------------------------------------------------------------

def er_triangle() -> Csr:
    """Triangle workload: G(4096, 16/4095), seed 1, average degree 16."""
    return erdos_renyi(4096, 16.0 / 4095.0, 1)


def rmat_clique() -> Csr:
    """k-clique workload: R-MAT scale 20, edge factor 16, seed 20."""
    return rmat(20, 16, 20)


def rmat_patterns() -> Csr:
    """Arbitrary-pattern workload: R-MAT scale 22, edge factor 16, seed 22."""
    return rmat(22, 16, 22)


def rmat_served() -> Csr:
    """Served workload: R-MAT scale 24, edge factor 16, seed 24."""
    return rmat(24, 16, 24)


BATCH_SCALES = [10, 11, 12, 13, 14, 15, 16, 17, 18, 19, 20, 21, 12, 14, 16, 18]
BATCH_EFS = [8, 16, 24, 32]


def batch_graph(i: int) -> Csr:
    """Graph i (0..15) of the batched workload: scales 10..21 then 12,14,16,18; ef cycles 8..32."""
    return rmat(BATCH_SCALES[i], BATCH_EFS[i % 4], 100 + i)


# --- small structured graphs (edge cases and closed forms) ----------------------------

def complete(n: int) -> Csr:
    return from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)], f"K{n}")


def cycle(n: int) -> Csr:
    return from_edges(n, [(i, (i + 1) % n) for i in range(n)], f"C{n}")


def star(leaves: int) -> Csr:
    return from_edges(leaves + 1, [(0, i) for i in range(1, leaves + 1)], f"star{leaves}")


def complete_bipartite(a: int, b: int) -> Csr:
    return from_edges(a + b, [(i, a + j) for i in range(a) for j in range(b)], f"K{a},{b}")


def petersen() -> Csr:
    outer = [(i, (i + 1) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    return from_edges(10, outer + spokes + inner, "petersen")


def empty(n: int) -> Csr:
    return from_edges(n, [], f"empty{n}")


def random_small(n: int, p: float, seed: int) -> Csr:
    """Tiny G(n, p) through the same counter-based generator (for brute-force checks)."""
    return erdos_renyi(n, p, seed)
