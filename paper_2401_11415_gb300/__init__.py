"""Python binding of liblp (GPU neighbourhood-based link prediction, sm_103a).

Argument marshalling only: every step of the computation runs in the CUDA
library ``liblp.so`` built from ``csrc/`` (see ``_build.py``).  The names
mirror the C ABI in ``include/lp.h``.  There is no CPU fallback: every call
into the library fails loudly (ImportError) when it has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblp.so")

MEASURES = ["CN", "JC", "SI", "SC", "HP", "HD", "LHN", "AA", "RA"]
LP_CN, LP_JC, LP_SI, LP_SC, LP_HP, LP_HD, LP_LHN, LP_AA, LP_RA = range(9)
LP_CAP_NONE = -1
LP_MAX_TOPK_PER_SOURCE = 64
LP_VALIDATE_FULL = 1

STATUS = {0: "LP_OK", 1: "LP_EINVAL", 2: "LP_ENOMEM", 3: "LP_ECUDA", 4: "LP_ETRUNC",
          5: "LP_ETIMEOUT", 6: "LP_EBUSY", 7: "LP_EINTERNAL"}
LP_OK, LP_EINVAL, LP_ENOMEM, LP_ECUDA, LP_ETRUNC, LP_ETIMEOUT, LP_EBUSY, LP_EINTERNAL = range(8)

LINK_DTYPE = np.dtype([("u", np.int32), ("v", np.int32), ("score", np.float32),
                       ("cn", np.int32)])


class LPError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class lp_stats(ctypes.Structure):
    _fields_ = [("wedges", ctypes.c_int64), ("kept_arcs", ctypes.c_int64),
                ("scanned_arcs", ctypes.c_int64), ("candidates", ctypes.c_int64),
                ("admitted", ctypes.c_int64), ("warp_sources", ctypes.c_int32),
                ("cta_items", ctypes.c_int32), ("dense_items", ctypes.c_int32),
                ("splits", ctypes.c_int32), ("compactions", ctypes.c_int32),
                ("launches", ctypes.c_int32), ("ms_estimate", ctypes.c_float),
                ("ms_scan", ctypes.c_float), ("ms_select", ctypes.c_float),
                ("ms_total", ctypes.c_float), ("tier_wedges", ctypes.c_int64 * 4),
                ("tier_arcs", ctypes.c_int64 * 4), ("tier_kept", ctypes.c_int64 * 4),
                ("tier_launches", ctypes.c_int32 * 4), ("tier_ms", ctypes.c_float * 4),
                ("phase_cycles", ctypes.c_int64 * 6), ("ms_expand", ctypes.c_float),
                ("exp_units", ctypes.c_int32), ("exp_batches", ctypes.c_int32),
                ("exp_items", ctypes.c_int64), ("exp_dense_units", ctypes.c_int64)]


class lp_serve_opts(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("max_batch_sources", ctypes.c_int32),
                ("max_pending", ctypes.c_int32), ("max_k", ctypes.c_int32),
                ("paused", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("idle_polls", ctypes.c_int32), ("defer_wedges", ctypes.c_int32)]


class lp_serve_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("batched_sources", ctypes.c_int64),
                ("max_batch_requests", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("deferred_sources", ctypes.c_int64)]


_i32p = ctypes.POINTER(ctypes.c_int32)
_vp = ctypes.c_void_p
_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"liblp.so is not built ({LIB_PATH}); run "
                          "paper_2401_11415_gb300._build.build() first")
    lib = ctypes.CDLL(LIB_PATH)
    st = ctypes.c_int
    lib.lp_graph_create.restype = st
    lib.lp_graph_create.argtypes = [ctypes.c_int32, _vp, _vp, ctypes.c_uint32,
                                    ctypes.POINTER(_vp)]
    lib.lp_graph_destroy.restype = st
    lib.lp_graph_destroy.argtypes = [_vp]
    lib.lp_graph_info.restype = st
    lib.lp_graph_info.argtypes = [_vp, _i32p, ctypes.POINTER(ctypes.c_int64), _i32p]
    lib.lp_predict.restype = st
    lib.lp_predict.argtypes = [_vp, ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                               _vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
    lib.lp_predict_dev.restype = st
    lib.lp_predict_dev.argtypes = lib.lp_predict.argtypes
    lib.lp_batch_create.restype = st
    lib.lp_batch_create.argtypes = [ctypes.c_int32, _vp, _vp, _vp, ctypes.c_uint32,
                                    ctypes.POINTER(_vp)]
    lib.lp_batch_destroy.restype = st
    lib.lp_batch_destroy.argtypes = [_vp]
    lib.lp_batch_info.restype = st
    lib.lp_batch_info.argtypes = [_vp, _i32p, _i32p, _vp]
    lib.lp_batch_graph.restype = _vp
    lib.lp_batch_graph.argtypes = [_vp]
    lib.lp_batch_predict_all.restype = st
    lib.lp_batch_predict_all.argtypes = [_vp, ctypes.c_int, ctypes.c_int32, ctypes.c_int32, _vp,
                                         _vp]
    lib.lp_batch_autotune.restype = st
    lib.lp_batch_autotune.argtypes = [_vp, ctypes.c_int, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_int32, _vp, _vp, ctypes.POINTER(ctypes.c_float),
                                      ctypes.POINTER(ctypes.c_float)]
    lib.lp_batch_get_option.restype = ctypes.c_int64
    lib.lp_batch_get_option.argtypes = [_vp, ctypes.c_int]
    lib.lp_predict_range.restype = st
    lib.lp_predict_range.argtypes = [_vp, ctypes.c_int, ctypes.c_int32, ctypes.c_int64,
                                     ctypes.c_double, ctypes.c_int32, ctypes.c_int32, _vp,
                                     ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
    lib.lp_merge_links.restype = st
    lib.lp_merge_links.argtypes = [_vp, ctypes.c_int, ctypes.c_int32, _vp, ctypes.c_int64,
                                   ctypes.c_int64, _vp, ctypes.c_int64,
                                   ctypes.POINTER(ctypes.c_int64)]
    lib.lp_predict_sources.restype = st
    lib.lp_predict_sources.argtypes = [_vp, ctypes.c_int, ctypes.c_int32, _vp, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_double, _vp, _vp]
    lib.lp_predict_sources_dev.restype = st
    lib.lp_predict_sources_dev.argtypes = lib.lp_predict_sources.argtypes
    lib.lp_predict_sources_static.restype = st
    lib.lp_predict_sources_static.argtypes = lib.lp_predict_sources.argtypes
    lib.lp_serve_open.restype = st
    lib.lp_serve_open.argtypes = [_vp, ctypes.POINTER(lp_serve_opts), ctypes.POINTER(_vp)]
    lib.lp_serve_submit.restype = st
    lib.lp_serve_submit.argtypes = [_vp, _vp, ctypes.c_int32, ctypes.c_int, ctypes.c_int32,
                                    ctypes.c_int32, ctypes.POINTER(ctypes.c_uint64)]
    lib.lp_serve_wait.restype = st
    lib.lp_serve_wait.argtypes = [_vp, ctypes.c_uint64, ctypes.c_int64, _vp, _vp]
    lib.lp_serve_poll.restype = st
    lib.lp_serve_poll.argtypes = [_vp, ctypes.c_uint64, _i32p]
    lib.lp_serve_resume.restype = st
    lib.lp_serve_resume.argtypes = [_vp]
    lib.lp_serve_get_stats.restype = st
    lib.lp_serve_get_stats.argtypes = [_vp, ctypes.POINTER(lp_serve_stats)]
    lib.lp_serve_close.restype = st
    lib.lp_serve_close.argtypes = [_vp]
    lib.lp_last_stats.restype = st
    lib.lp_last_stats.argtypes = [ctypes.POINTER(lp_stats)]
    lib.lp_set_timing.restype = None
    lib.lp_set_timing.argtypes = [ctypes.c_int]
    lib.lp_graph_stream.restype = _vp
    lib.lp_graph_stream.argtypes = [_vp]
    lib.lp_last_error.restype = ctypes.c_char_p
    lib.lp_last_error.argtypes = []
    lib.lp_set_option.restype = st
    lib.lp_set_option.argtypes = [ctypes.c_int, ctypes.c_int64]
    lib.lp_get_option.restype = ctypes.c_int64
    lib.lp_get_option.argtypes = [ctypes.c_int]
    lib.lp_version.restype = ctypes.c_char_p
    lib.lp_version.argtypes = []
    _lib = lib
    return lib


def lib():
    """The loaded ctypes library."""
    return _load()


def _check(status: int, allow=()):
    if status != LP_OK and status not in allow:
        raise LPError(status, lp_last_error())
    return status


def _measure(m) -> int:
    return MEASURES.index(m.upper()) if isinstance(m, str) else int(m)


def _cap(cap) -> int:
    if cap is None or cap == float("inf") or cap < 0:
        return LP_CAP_NONE
    return int(min(cap, 2**31 - 1))


def _ptr(x):
    """Host numpy array or torch tensor (host or device) -> address."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return int(x)


# ------------------------------------------------------------ C ABI names --

def lp_last_error() -> str:
    return _load().lp_last_error().decode()


def lp_version() -> str:
    return _load().lp_version().decode()


def lp_set_timing(enable: bool) -> None:
    _load().lp_set_timing(1 if enable else 0)


def lp_graph_create(n: int, offsets, indices, flags: int = 0):
    off = np.ascontiguousarray(offsets, dtype=np.int32)
    idx = np.ascontiguousarray(indices, dtype=np.int32)
    if off.size != n + 1:
        raise ValueError("offsets must have n + 1 entries")
    h = _vp()
    _check(_load().lp_graph_create(n, off.ctypes.data, idx.ctypes.data if idx.size else None,
                                   flags, ctypes.byref(h)))
    return h


def lp_graph_destroy(h) -> None:
    if h:
        _load().lp_graph_destroy(h)


def lp_graph_info(h):
    n = ctypes.c_int32()
    a = ctypes.c_int64()
    d = ctypes.c_int32()
    _check(_load().lp_graph_info(h, ctypes.byref(n), ctypes.byref(a), ctypes.byref(d)))
    return n.value, a.value, d.value


def lp_graph_stream(h) -> int:
    return _load().lp_graph_stream(h) or 0


def lp_predict(h, measure, degree_cap=None, k: int = 0, threshold: float = 0.0,
               out_cap: int | None = None):
    """Global mode; returns a numpy array of LINK_DTYPE (host buffers)."""
    lib = _load()
    cnt = ctypes.c_int64(0)
    m, c = _measure(measure), _cap(degree_cap)
    if out_cap is None:
        out_cap = k if k > 0 else 0
    out = np.zeros(max(out_cap, 1), dtype=LINK_DTYPE)
    st = lib.lp_predict(h, m, c, k, threshold, out.ctypes.data, out_cap, ctypes.byref(cnt))
    if st == LP_ETRUNC and out_cap == 0 and k == 0:
        out = np.zeros(max(cnt.value, 1), dtype=LINK_DTYPE)
        st = lib.lp_predict(h, m, c, k, threshold, out.ctypes.data, cnt.value, ctypes.byref(cnt))
    _check(st)
    return out[: cnt.value].copy()


def lp_predict_range(h, measure, degree_cap, k: int, src_begin: int, src_end: int,
                     threshold: float = 0.0):
    """Global mode over the sources [src_begin, src_end) (host buffers)."""
    cnt = ctypes.c_int64(0)
    out = np.zeros(max(k, 1), dtype=LINK_DTYPE)
    _check(_load().lp_predict_range(h, _measure(measure), _cap(degree_cap), k, threshold,
                                    src_begin, src_end, out.ctypes.data, k, ctypes.byref(cnt)))
    return out[: cnt.value].copy()


def lp_merge_links(h, measure, degree_cap, links, k: int) -> np.ndarray:
    """The best k of the given global-mode links (an array of LINK_DTYPE, any
    order) under the library's exact order (host buffers)."""
    src = np.ascontiguousarray(links, dtype=LINK_DTYPE)
    cnt = ctypes.c_int64(0)
    cap_out = min(k, src.size) if k > 0 else src.size
    out = np.zeros(max(cap_out, 1), dtype=LINK_DTYPE)
    _check(_load().lp_merge_links(h, _measure(measure), _cap(degree_cap),
                                  src.ctypes.data if src.size else None, src.size, k,
                                  out.ctypes.data, cap_out, ctypes.byref(cnt)))
    return out[: cnt.value].copy()


def lp_predict_dev(h, measure, degree_cap, k: int, threshold: float, d_out, out_cap: int) -> int:
    """Global mode into a device buffer (torch tensor or address); returns the
    number of links found."""
    cnt = ctypes.c_int64(0)
    _check(_load().lp_predict_dev(h, _measure(measure), _cap(degree_cap), k, threshold,
                                  _ptr(d_out), out_cap, ctypes.byref(cnt)))
    return cnt.value


def lp_predict_sources(h, measure, sources, k: int, degree_cap=None, threshold: float = 0.0):
    """Per-source mode (host buffers); returns (links[n_src, k], counts[n_src])."""
    src = np.ascontiguousarray(sources, dtype=np.int32)
    ns = src.size
    out = np.zeros(max(ns * k, 1), dtype=LINK_DTYPE)
    counts = np.zeros(max(ns, 1), dtype=np.int32)
    _check(_load().lp_predict_sources(h, _measure(measure), _cap(degree_cap),
                                      src.ctypes.data if ns else None, ns, k, threshold,
                                      out.ctypes.data, counts.ctypes.data))
    return out[: ns * k].reshape(ns, k), counts[:ns].copy()


def lp_predict_sources_dev(h, measure, d_sources, n_src: int, k: int, degree_cap, threshold,
                           d_out, d_counts) -> None:
    _check(_load().lp_predict_sources_dev(h, _measure(measure), _cap(degree_cap),
                                          _ptr(d_sources), n_src, k, threshold, _ptr(d_out),
                                          _ptr(d_counts)))


def lp_predict_sources_static(h, measure, d_sources, n_src: int, k: int, degree_cap, threshold,
                              d_out, d_counts) -> None:
    """Per-source mode without allocation (device pointers; see include/lp.h)."""
    _check(_load().lp_predict_sources_static(h, _measure(measure), _cap(degree_cap),
                                             _ptr(d_sources), n_src, k, threshold, _ptr(d_out),
                                             _ptr(d_counts)))


LP_OPT_SELECT_BUFFER, LP_OPT_WARP_MAX_WEDGES, LP_OPT_CTA_MAX_WEDGES, LP_OPT_SPLIT_TARGET, \
    LP_OPT_SPLIT_LOGCAP, LP_OPT_MED_MAX_WEDGES, LP_OPT_ITEM_WEDGES, LP_OPT_PHASE_PROFILE, \
    LP_OPT_BIG_CTA_THREADS, LP_OPT_EXPAND, LP_OPT_EXPAND_BATCH, \
    LP_OPT_EXPAND_HASH_LOGCAP, LP_OPT_EXPAND_MIN_WEDGES = range(1, 14)


def lp_set_option(option: int, value: int) -> None:
    _check(_load().lp_set_option(option, value))


def lp_get_option(option: int) -> int:
    return int(_load().lp_get_option(option))


def lp_last_stats() -> dict:
    s = lp_stats()
    _check(_load().lp_last_stats(ctypes.byref(s)))
    out = {}
    for f, _ in lp_stats._fields_:
        v = getattr(s, f)
        out[f] = list(v) if hasattr(v, "__len__") else v
    return out


class Graph:
    """Owning wrapper of an lp_graph handle."""

    def __init__(self, n, offsets, indices, flags: int = 0):
        self.n = int(n)
        self.handle = lp_graph_create(self.n, offsets, indices, flags)

    @classmethod
    def from_csr(cls, g, flags: int = 0):
        return cls(g.n, g.off, g.idx, flags)

    def info(self):
        return lp_graph_info(self.handle)

    def predict(self, measure, degree_cap=None, k=0, threshold=0.0):
        return lp_predict(self.handle, measure, degree_cap, k, threshold)

    def predict_range(self, measure, degree_cap, k, src_begin, src_end, threshold=0.0):
        return lp_predict_range(self.handle, measure, degree_cap, k, src_begin, src_end,
                                threshold)

    def merge(self, measure, degree_cap, links, k):
        return lp_merge_links(self.handle, measure, degree_cap, links, k)

    def predict_sources(self, measure, sources, k, degree_cap=None, threshold=0.0):
        return lp_predict_sources(self.handle, measure, sources, k, degree_cap, threshold)

    @property
    def stream(self) -> int:
        return lp_graph_stream(self.handle)

    def close(self):
        if self.handle:
            lp_graph_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# -------------------------------------------------------- batched mode --

class Batch:
    """Many graphs packed into one block-diagonal graph (lp_batch_*): the
    per-source top-k of every vertex of every graph from one recorded launch
    sequence.  ``predict_all`` fills device buffers (torch tensors) and
    returns them with packed ids; ``bases[i]`` is graph i's first vertex."""

    def __init__(self, graphs, flags: int = 0):
        lib = _load()
        ng = len(graphs)
        self._keep = [(np.ascontiguousarray(g.off, dtype=np.int32),
                       np.ascontiguousarray(g.idx, dtype=np.int32)) for g in graphs]
        nv = np.array([g.n for g in graphs], dtype=np.int32)
        offs = (ctypes.c_void_p * ng)(*[o.ctypes.data for o, _ in self._keep])
        idxs = (ctypes.c_void_p * ng)(*[(i.ctypes.data if i.size else o.ctypes.data)
                                        for o, i in self._keep])
        h = _vp()
        _check(lib.lp_batch_create(ng, nv.ctypes.data, ctypes.cast(offs, _vp),
                                   ctypes.cast(idxs, _vp), flags, ctypes.byref(h)))
        self.handle = h
        self._keep = None
        ngr, nt = ctypes.c_int32(0), ctypes.c_int32(0)
        self.bases = np.zeros(ng + 1, dtype=np.int32)
        _check(lib.lp_batch_info(h, ctypes.byref(ngr), ctypes.byref(nt), self.bases.ctypes.data))
        self.n_graphs, self.n_total = ngr.value, nt.value
        self._out = None

    def close(self):
        if self.handle:
            _load().lp_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def graph_handle(self):
        return _load().lp_batch_graph(self.handle)

    def _buffers(self, k):
        import torch
        if self._out is None or self._out[2] != k:
            out = torch.empty((max(self.n_total, 1) * k * 16,), dtype=torch.uint8, device="cuda")
            cnt = torch.empty((max(self.n_total, 1),), dtype=torch.int32, device="cuda")
            self._out = (out, cnt, k)
        return self._out[0], self._out[1]

    def predict_all(self, measure, degree_cap=None, k: int = 10):
        """(links uint8 device tensor of n_total * k LINK_DTYPE rows, counts)."""
        out, cnt = self._buffers(k)
        _check(_load().lp_batch_predict_all(self.handle, _measure(measure), _cap(degree_cap), k,
                                            _ptr(out), _ptr(cnt)))
        return out, cnt

    def autotune(self, measure, degree_cap=None, k: int = 10, repeats: int = 2):
        """Tune the batch's binning options on this query; returns
        (default_ms, best_ms, {option: value})."""
        out, cnt = self._buffers(k)
        d, b = ctypes.c_float(0), ctypes.c_float(0)
        _check(_load().lp_batch_autotune(self.handle, _measure(measure), _cap(degree_cap), k,
                                         repeats, _ptr(out), _ptr(cnt), ctypes.byref(d),
                                         ctypes.byref(b)))
        names = {"warp_max": LP_OPT_WARP_MAX_WEDGES, "med_max": LP_OPT_MED_MAX_WEDGES,
                 "cta_max": LP_OPT_CTA_MAX_WEDGES, "item_wedges": LP_OPT_ITEM_WEDGES,
                 "big_threads": LP_OPT_BIG_CTA_THREADS}
        opts = {nm: int(_load().lp_batch_get_option(self.handle, o)) for nm, o in names.items()}
        return d.value, b.value, opts


# ------------------------------------------------------------- serving --

class Server:
    """lp_serve_* wrapper: continuous batching of per-source queries (mode 0:
    host worker threads running batches, the default; mode 1: a resident
    kernel)."""

    def __init__(self, graph, slots=0, max_batch_sources=0, max_pending=0, max_k=0,
                 paused=False, mode=0, idle_polls=0, defer_wedges=0):
        o = lp_serve_opts(slots, max_batch_sources, max_pending, max_k, 1 if paused else 0, mode,
                          idle_polls, defer_wedges)
        h = _vp()
        _check(_load().lp_serve_open(graph.handle if isinstance(graph, Graph) else graph,
                                     ctypes.byref(o), ctypes.byref(h)))
        self.handle = h
        self._sizes = {}

    def submit(self, sources, measure, k, degree_cap=None) -> int:
        src = np.ascontiguousarray(sources, dtype=np.int32)
        rid = ctypes.c_uint64()
        _check(_load().lp_serve_submit(self.handle, src.ctypes.data, src.size, _measure(measure),
                                       _cap(degree_cap), k, ctypes.byref(rid)))
        self._sizes[rid.value] = (src.size, k)
        return rid.value

    def wait(self, req_id: int, timeout_us: int = -1):
        n, k = self._sizes.get(req_id, (0, 1))
        out = np.zeros(max(n * k, 1), dtype=LINK_DTYPE)
        counts = np.zeros(max(n, 1), dtype=np.int32)
        st = _load().lp_serve_wait(self.handle, req_id, timeout_us, out.ctypes.data,
                                   counts.ctypes.data)
        if st != LP_ETIMEOUT:
            self._sizes.pop(req_id, None)
        _check(st)
        return out[: n * k].reshape(n, k), counts[:n].copy()

    def poll(self, req_id: int) -> bool:
        d = ctypes.c_int32()
        _check(_load().lp_serve_poll(self.handle, req_id, ctypes.byref(d)))
        return bool(d.value)

    def resume(self):
        _check(_load().lp_serve_resume(self.handle))

    def stats(self) -> dict:
        s = lp_serve_stats()
        _check(_load().lp_serve_get_stats(self.handle, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in lp_serve_stats._fields_}

    def close(self):
        if self.handle:
            _load().lp_serve_close(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

