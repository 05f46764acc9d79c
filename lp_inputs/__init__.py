"""Seeded synthetic inputs for the link-prediction tests and benchmark.

Shared by the CPU oracle side and the CUDA side; it generates graphs and the
hold-out split only and holds none of the link-prediction arithmetic.  The C
core (``gen.c``) is compiled on first use into ``_lpgen.so`` next to this file.

Graph recipes (stand-ins for the paper's web / social / road inputs, Section
5.1.3 and Table 1, which are not available here):

* ``rmat``: R-MAT samples with (a, b, c) = (0.57, 0.19, 0.19), symmetrised,
  self-loops and duplicates removed, vertex ids permuted with a seeded
  permutation so that hubs are not concentrated at low ids.
* ``chung_lu``: expected-degree weights w_i ~ (i + i0)^(-1/(gamma-1)) with
  mean degree ``mean_deg``, i0 set so the largest weight is ``dmax``; exactly
  round(n * mean_deg / 2) distinct undirected edges; ids permuted.
* ``grid``: rows x cols 4-neighbour lattice, row-major ids.
* ``holdout``: removes floor(frac * |E|) undirected edges chosen uniformly
  without replacement (Section 5.1.4), returning the observed graph and the
  held-out pairs (u < v).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "_lpgen.so")
_lock = threading.Lock()
_lib = None

_i32p = ctypes.POINTER(ctypes.c_int32)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile gen.c into _lpgen.so (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            lib.lpi_rng_u64.restype = ctypes.c_uint64
            lib.lpi_rng_u64.argtypes = [ctypes.c_uint64] * 3
            lib.lpi_rmat_edges.restype = None
            lib.lpi_rmat_edges.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                           _i32p, _i32p]
            lib.lpi_chung_lu_i0.restype = ctypes.c_double
            lib.lpi_chung_lu_i0.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double]
            lib.lpi_chung_lu_edges.restype = ctypes.c_int64
            lib.lpi_chung_lu_edges.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_int64, ctypes.c_uint64, _i32p, _i32p]
            lib.lpi_grid_edges.restype = ctypes.c_int64
            lib.lpi_grid_edges.argtypes = [ctypes.c_int32, ctypes.c_int32, _i32p, _i32p]
            lib.lpi_permutation.restype = None
            lib.lpi_permutation.argtypes = [ctypes.c_int32, ctypes.c_uint64, _i32p]
            lib.lpi_build_csr.restype = ctypes.c_int64
            lib.lpi_build_csr.argtypes = [ctypes.c_int32, ctypes.c_int64, _i32p, _i32p, _i32p,
                                          _i32p, _i32p, _i32p]
            lib.lpi_holdout.restype = ctypes.c_int64
            lib.lpi_holdout.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_int64,
                                        ctypes.c_uint64, _u8p, _i32p, _i32p]
            lib.lpi_filter_csr.restype = ctypes.c_int64
            lib.lpi_filter_csr.argtypes = [ctypes.c_int32, _i32p, _i32p, _u8p, _i32p, _i32p]
            _lib = lib
    return _lib


def _p(a: np.ndarray, t=_i32p):
    return a.ctypes.data_as(t) if a is not None else None


@dataclass
class Graph:
    """Symmetric CSR: ``off`` int32[n+1], ``idx`` int32[off[n]], sorted lists."""
    n: int
    off: np.ndarray
    idx: np.ndarray
    name: str = ""

    @property
    def arcs(self) -> int:
        return int(self.off[-1])

    @property
    def edges(self) -> int:
        return int(self.off[-1]) // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.off).astype(np.int64)


@dataclass
class Split:
    """Observed graph plus the held-out undirected pairs (u < v)."""
    observed: Graph
    hu: np.ndarray
    hv: np.ndarray


def rng_u64(seed: int, stream: int, i: int) -> int:
    return int(_load().lpi_rng_u64(seed, stream, i))


def from_edges(n: int, u, v, perm=None, name: str = "") -> Graph:
    """Symmetric, self-loop-free, deduplicated CSR from edge samples."""
    lib = _load()
    u = np.ascontiguousarray(u, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.int32)
    if u.size and (u.min() < 0 or v.min() < 0 or u.max() >= n or v.max() >= n):
        raise ValueError("endpoint out of range")
    perm = None if perm is None else np.ascontiguousarray(perm, dtype=np.int32)
    off = np.zeros(n + 1, dtype=np.int32)
    m = u.size
    scratch = np.empty(max(2 * m, 1), dtype=np.int32)
    a = lib.lpi_build_csr(n, m, _p(u), _p(v), _p(perm) if perm is not None else None,
                          _p(off), None, _p(scratch))
    if a < 0:
        raise MemoryError("CSR build failed (too many arcs)")
    idx = np.empty(max(a, 1), dtype=np.int32)
    a2 = lib.lpi_build_csr(n, m, _p(u), _p(v), _p(perm) if perm is not None else None,
                           _p(off), _p(idx), _p(scratch))
    assert a2 == a
    return Graph(n, off, idx[:a].copy() if a else np.zeros(0, np.int32), name)


def permutation(n: int, seed: int) -> np.ndarray:
    perm = np.empty(n, dtype=np.int32)
    _load().lpi_permutation(n, seed, _p(perm))
    return perm


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = 1, permute: bool = True) -> Graph:
    n = 1 << scale
    m = edge_factor * n
    u = np.empty(m, dtype=np.int32)
    v = np.empty(m, dtype=np.int32)
    _load().lpi_rmat_edges(scale, m, a, b, c, seed, _p(u), _p(v))
    perm = permutation(n, seed ^ 0x5EED) if permute else None
    return from_edges(n, u, v, perm, name=f"rmat{scale}_ef{edge_factor}_s{seed}")


def chung_lu(n: int, mean_deg: float, gamma: float, dmax: float = 0.0, seed: int = 42,
             permute: bool = True) -> Graph:
    lib = _load()
    i0 = lib.lpi_chung_lu_i0(n, gamma, mean_deg, float(dmax))
    m_target = int(round(n * mean_deg / 2.0))
    u = np.empty(max(m_target, 1), dtype=np.int32)
    v = np.empty(max(m_target, 1), dtype=np.int32)
    got = lib.lpi_chung_lu_edges(n, gamma, i0, m_target, seed, _p(u), _p(v))
    if got < 0:
        raise MemoryError("Chung-Lu generation failed")
    perm = permutation(n, seed ^ 0x5EED) if permute else None
    return from_edges(n, u[:got], v[:got], perm, name=f"chunglu{n}_d{mean_deg}_g{gamma}_s{seed}")


def grid(rows: int, cols: int) -> Graph:
    m = rows * (cols - 1) + cols * (rows - 1)
    u = np.empty(max(m, 1), dtype=np.int32)
    v = np.empty(max(m, 1), dtype=np.int32)
    got = _load().lpi_grid_edges(rows, cols, _p(u), _p(v))
    return from_edges(rows * cols, u[:got], v[:got], None, name=f"grid{rows}x{cols}")


def gnp(n: int, p: float, seed: int) -> Graph:
    """Erdos-Renyi G(n, p) for tiny brute-force cases (pair (i, j) kept when
    its draw is below p)."""
    us, vs = [], []
    k = 0
    for i in range(n):
        for j in range(i + 1, n):
            if (rng_u64(seed, 5, k) >> 11) * (1.0 / 9007199254740992.0) < p:
                us.append(i)
                vs.append(j)
            k += 1
    return from_edges(n, np.array(us, np.int32), np.array(vs, np.int32), name=f"gnp{n}_{p}_{seed}")


def holdout(g: Graph, frac: float = 0.1, seed: int = 43) -> Split:
    """Remove floor(frac * |E|) undirected edges chosen uniformly at random."""
    lib = _load()
    k = int(np.floor(frac * g.edges))
    held = np.zeros(max(g.arcs, 1), dtype=np.uint8)
    hu = np.empty(max(k, 1), dtype=np.int32)
    hv = np.empty(max(k, 1), dtype=np.int32)
    got = lib.lpi_holdout(g.n, _p(g.off), _p(g.idx), k, seed, _p(held, _u8p), _p(hu), _p(hv))
    if got < 0:
        raise MemoryError("hold-out failed")
    off2 = np.zeros(g.n + 1, dtype=np.int32)
    idx2 = np.empty(max(g.arcs - 2 * got, 1), dtype=np.int32)
    w = lib.lpi_filter_csr(g.n, _p(g.off), _p(g.idx), _p(held, _u8p), _p(off2), _p(idx2))
    assert w == g.arcs - 2 * got
    obs = Graph(g.n, off2, idx2[:w].copy(), name=g.name + f"_obs{frac}_s{seed}")
    return Split(obs, hu[:got].copy(), hv[:got].copy())


# ---------------------------------------------------------------- recipes --
# Workload recipes: the shapes of the benchmarked configurations.

def cfg_chung_lu_2k(seed: int = 42) -> Graph:
    """Chung-Lu, 2,000 vertices, mean degree 20 (~20,000 undirected edges),
    exponent 2.1, largest expected degree 400."""
    return chung_lu(2000, 20.0, 2.1, dmax=400.0, seed=seed)


def cfg_rmat20(seed: int = 1) -> Graph:
    """R-MAT scale 20, edge factor 16, (0.57, 0.19, 0.19)."""
    return rmat(20, 16, seed=seed)


def cfg_chung_lu_4m(seed: int = 7) -> Graph:
    """Chung-Lu, 4,194,304 vertices, mean degree 30.5, exponent 2.3,
    largest expected degree 100,000."""
    return chung_lu(1 << 22, 30.5, 2.3, dmax=100000.0, seed=seed)


def cfg_grid2048() -> Graph:
    return grid(2048, 2048)


def cfg_rmat24(seed: int = 1) -> Graph:
    return rmat(24, 16, seed=seed)
