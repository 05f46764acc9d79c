"""CPU oracle for neighbourhood-based link prediction -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it and
shares no code with it.  The C core (``lp_oracle.c``) follows Algorithm 1 of
the paper in FP64; this module compiles it and wraps it with ctypes, and adds
the prediction-quality measures of Section 3.2 (Eq. 10-12).

Every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle.py`` (brute force over all pairs with exact rationals,
hand-worked closed forms, invariants); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lp_oracle.c")
_LIB = os.path.join(_HERE, "_lp_oracle.so")
_lock = threading.Lock()
_lib = None

MEASURES = ["CN", "JC", "SI", "SC", "HP", "HD", "LHN", "AA", "RA"]
COUNT_MEASURES = MEASURES[:7]

LINK_DTYPE = np.dtype([("u", np.int32), ("v", np.int32), ("cn", np.int64),
                       ("num", np.uint64), ("den", np.uint64), ("value", np.float64)],
                      align=True)

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False, extra_flags=()) -> str:
    """Compile lp_oracle.c (gcc, OpenMP) into _lp_oracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11",
                               *extra_flags, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _bind(lib):
    lib.lpo_predict.restype = ctypes.c_int
    lib.lpo_predict.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_int, ctypes.c_int64,
                                ctypes.c_int64, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                                ctypes.c_int64, _i64p]
    lib.lpo_predict_sources.restype = ctypes.c_int
    lib.lpo_predict_sources.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_int,
                                        ctypes.c_int64, _i32p, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_double, ctypes.c_int, ctypes.c_void_p, _i32p]
    lib.lpo_pair.restype = ctypes.c_int
    lib.lpo_pair.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_int, ctypes.c_int64,
                             ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, _i32p]
    lib.lpo_work.restype = None
    lib.lpo_work.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_int64, ctypes.c_int,
                             _i64p, _i64p]
    lib.lpo_better.restype = ctypes.c_int
    lib.lpo_better.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.lpo_sizeof_link.restype = ctypes.c_int
    assert lib.lpo_sizeof_link() == LINK_DTYPE.itemsize
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(ctypes.CDLL(_LIB))
    return _lib


def load_variant(path: str):
    """Bind a separately compiled copy of the oracle (used by the tests that
    check that planted mistakes are caught)."""
    return _bind(ctypes.CDLL(path))


def _measure_id(measure) -> int:
    if isinstance(measure, str):
        return MEASURES.index(measure.upper())
    return int(measure)


def _cap(cap) -> int:
    return -1 if cap is None or cap < 0 or cap == float("inf") else int(cap)


def _csr(off, idx):
    off = np.ascontiguousarray(off, dtype=np.int32)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    if idx.size == 0:
        idx = np.zeros(1, dtype=np.int32)
    return off, idx


def predict(n, off, idx, measure, cap=None, k=0, threshold=0.0, nthreads=0, lib=None):
    """Global mode (Algorithm 1): top-k pairs u < v (k = 0: all), sorted by
    (score desc, u asc, v asc).  cap None/inf/negative = IBase."""
    lib = lib or _load()
    off, idx = _csr(off, idx)
    m = _measure_id(measure)
    c = _cap(cap)
    cnt = ctypes.c_int64(0)
    if k > 0:
        out = np.zeros(k, dtype=LINK_DTYPE)
        rc = lib.lpo_predict(n, off.ctypes.data_as(_i32p), idx.ctypes.data_as(_i32p), m, c, k,
                             float(threshold), nthreads, out.ctypes.data, k, ctypes.byref(cnt))
        if rc != 0:
            raise RuntimeError(f"lpo_predict failed ({rc})")
        return out[: cnt.value].copy()
    # unbounded: size the output by a first call
    rc = lib.lpo_predict(n, off.ctypes.data_as(_i32p), idx.ctypes.data_as(_i32p), m, c, 0,
                         float(threshold), nthreads, None, 0, ctypes.byref(cnt))
    if rc != 0:
        raise RuntimeError(f"lpo_predict failed ({rc})")
    total = cnt.value
    out = np.zeros(max(total, 1), dtype=LINK_DTYPE)
    rc = lib.lpo_predict(n, off.ctypes.data_as(_i32p), idx.ctypes.data_as(_i32p), m, c, 0,
                         float(threshold), nthreads, out.ctypes.data, total, ctypes.byref(cnt))
    if rc != 0:
        raise RuntimeError(f"lpo_predict failed ({rc})")
    return out[:total].copy()


def predict_sources(n, off, idx, measure, sources, k, cap=None, threshold=0.0, nthreads=0,
                    lib=None):
    """Per-source mode: returns (links[n_src, k], counts[n_src])."""
    lib = lib or _load()
    off, idx = _csr(off, idx)
    src = np.ascontiguousarray(sources, dtype=np.int32)
    ns = src.size
    out = np.zeros(max(ns * k, 1), dtype=LINK_DTYPE)
    counts = np.zeros(max(ns, 1), dtype=np.int32)
    rc = lib.lpo_predict_sources(n, off.ctypes.data_as(_i32p), idx.ctypes.data_as(_i32p),
                                 _measure_id(measure), _cap(cap),
                                 src.ctypes.data_as(_i32p) if ns else None, ns, k,
                                 float(threshold), nthreads, out.ctypes.data,
                                 counts.ctypes.data_as(_i32p))
    if rc != 0:
        raise RuntimeError(f"lpo_predict_sources failed ({rc})")
    return out[: ns * k].reshape(ns, k), counts[:ns].copy()


def pair(n, off, idx, measure, u, v, cap=None, lib=None):
    """Score of one pair from the definitions; returns (link, adjacent)."""
    lib = lib or _load()
    off, idx = _csr(off, idx)
    out = np.zeros(1, dtype=LINK_DTYPE)
    adj = ctypes.c_int32(0)
    rc = lib.lpo_pair(n, off.ctypes.data_as(_i32p), idx.ctypes.data_as(_i32p),
                      _measure_id(measure), _cap(cap), int(u), int(v), out.ctypes.data,
                      ctypes.byref(adj))
    if rc != 0:
        raise ValueError("bad pair")
    return out[0], bool(adj.value)


def work(n, off, idx, cap=None, mode=0, lib=None):
    """(wedges, kept arcs): wedges a-b-c with |Gamma_b| <= cap and c > a
    (mode 0) or c != a (mode 1)."""
    lib = lib or _load()
    off, idx = _csr(off, idx)
    w = ctypes.c_int64(0)
    ka = ctypes.c_int64(0)
    lib.lpo_work(n, off.ctypes.data_as(_i32p), idx.ctypes.data_as(_i32p), _cap(cap), mode,
                 ctypes.byref(w), ctypes.byref(ka))
    return w.value, ka.value


def better(x, y, lib=None) -> bool:
    """True if link x ranks strictly before link y in the total order."""
    lib = lib or _load()
    a = np.array([x], dtype=LINK_DTYPE)
    b = np.array([y], dtype=LINK_DTYPE)
    return bool(lib.lpo_better(a.ctypes.data, b.ctypes.data))


# ------------------------------------------------- prediction quality ------

def _pair_keys(u, v):
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    lo = np.minimum(u, v)
    hi = np.maximum(u, v)
    return (lo << 32) | hi


def quality(pred_u, pred_v, held_u, held_v):
    """Precision (Eq. 10), recall (Eq. 11) and F1 (Eq. 12) of predicted pairs
    against the held-out edges E^U, as unordered pairs."""
    p = np.unique(_pair_keys(pred_u, pred_v))
    h = np.unique(_pair_keys(held_u, held_v))
    hit = np.intersect1d(p, h, assume_unique=True).size
    precision = hit / p.size if p.size else 0.0
    recall = hit / h.size if h.size else 0.0
    f1 = 2 * precision * recall / (precision + recall) if precision + recall > 0 else 0.0
    return {"hits": int(hit), "precision": precision, "recall": recall, "f1": f1}
