"""Python binding of the B300 pattern-morphing library (libpm_b300.so).

Argument marshalling only: every step (graph preparation, morph selection,
plan compilation, matching, morph transform) runs inside the library, whose
C ABI is include/pm.h.  The library must be built (python
paper_2012_04553_b300/build.py); importing this package without it raises.
PyTorch supplies device memory (through pm_set_allocator) and streams.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# PM_DEBUG=1 selects the bounds-checked build (build.py --debug)
LIB_PATH = os.path.join(_HERE, "libpm_b300_debug.so" if os.environ.get("PM_DEBUG") == "1" else "libpm_b300.so")

PM_OK, PM_EINVAL, PM_ENOMEM, PM_ECUDA, PM_ETIMEOUT, PM_EOVERFLOW, PM_EUNSUPPORTED, PM_ECANCELLED = \
    0, -1, -2, -3, -4, -5, -6, -7
EDGE_INDUCED, VERTEX_INDUCED = 0, 1
OP_COUNT, OP_SUPPORT = 0, 1
MORPH_NONE, MORPH_NAIVE, MORPH_COST = 0, 1, 2
MAX_K = 8
PLANS_AUTO, PLANS_ROOTED, PLANS_FREE, PLANS_QUICK, PLANS_DECOMP = -1, 0, 1, 2, 3
LAUNCH_PER_PATTERN, LAUNCH_SINGLE = 0, 1


class PMError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = _lib.pm_strerror(status).decode()
        detail = _lib.pm_last_error().decode()
        super().__init__(f"{where}: {msg} ({status}){': ' + detail if detail else ''}")


class PMTimeout(PMError):
    pass


class c_pattern(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("edge_mask", ctypes.c_uint32),
                ("label", ctypes.c_int8 * MAX_K), ("induced", ctypes.c_int32)]


class c_graph_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("self_loops", ctypes.c_int64),
                ("duplicates", ctypes.c_int64), ("max_degree", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("labeled", ctypes.c_int32),
                ("device", ctypes.c_int32)]


class c_plan_info(ctypes.Structure):
    _fields_ = [("n_queries", ctypes.c_int32), ("n_matched", ctypes.c_int32),
                ("n_plans", ctypes.c_int32), ("op", ctypes.c_int32)]


class c_server_config(ctypes.Structure):
    _fields_ = [("workers_per_graph", ctypes.c_int32), ("max_batch_patterns", ctypes.c_int32),
                ("hbm_budget_bytes", ctypes.c_int64), ("batch_timeout_s", ctypes.c_double),
                ("batch_total_s", ctypes.c_double), ("mode", ctypes.c_int32), ("family", ctypes.c_int32),
                ("request_timeout_s", ctypes.c_double)]


class c_server_stats(ctypes.Structure):
    _fields_ = [(nm, ctypes.c_int64) for nm in (
        "requests_submitted", "requests_done", "batches", "patterns_done", "matched_alone",
        "matched_batched", "timeouts", "failures", "shed")]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p)


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python paper_2012_04553_b300/build.py`"
                          + (" --debug" if LIB_PATH.endswith("_debug.so") else ""))
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    sig = {
        "pm_set_allocator": [vp, vp, vp],
        "pm_load_graph": [i64, i64, vp, vp, vp, ctypes.c_int, vp, ctypes.POINTER(vp)],
        "pm_graph_get_info": [vp, ctypes.POINTER(c_graph_info)],
        "pm_graph_vertex_order": [vp, vp],
        "pm_prepare_csr": [i64, i64, vp, vp, vp, vp, vp, vp],
        "pm_plan": [vp, ctypes.POINTER(c_pattern), i32, ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp)],
        "pm_plan_get_info": [vp, ctypes.POINTER(c_plan_info)],
        "pm_plan_matched": [vp, ctypes.POINTER(c_pattern)],
        "pm_morph": [vp, vp, vp],
        "pm_count": [vp, vp, dbl, vp, vp],
        "pm_count_roots": [vp, vp, dbl, vp, i64, vp, vp],
        "pm_support": [vp, vp, dbl, ctypes.c_uint64, vp, vp, vp],
        "pm_plan_query_columns": [vp, vp],
        "pm_plan_export": [vp, i32, vp, i64],
        "pm_plan_select": [vp, i32],
        "pm_plan_set_launch": [vp, i32],
        "pm_count_each": [vp, vp, dbl, dbl, vp, vp],
        "pm_plan_autotune": [vp, vp, vp],
        "pm_count_c4_noalloc": [vp, vp, i64, vp, vp],
        "pm_plan_capture": [vp, vp, dbl],
        "pm_server_create": [vp, i32, ctypes.POINTER(c_server_config), ctypes.POINTER(vp)],
        "pm_server_submit": [vp, i32, ctypes.POINTER(c_pattern), i32, ctypes.POINTER(ctypes.c_uint64)],
        "pm_server_wait": [vp, ctypes.c_uint64, dbl, ctypes.POINTER(i32), vp, ctypes.POINTER(dbl),
                           ctypes.POINTER(ctypes.c_int), vp],
        "pm_server_get_stats": [vp, ctypes.POINTER(c_server_stats)],
        "pm_fsm": [vp, i32, ctypes.c_uint64, ctypes.c_int, vp, dbl, vp, vp, vp, i32, ctypes.POINTER(i32)],
        "pm_count_instrumented": [vp, vp, vp, vp],
        "pm_plan_last_kernel_ms": [vp, ctypes.POINTER(ctypes.c_float)],
        "pm_plan_pattern_ms": [vp, vp],
        "pm_plan_last_launches": [vp, vp],
        "pm_support_roots": [vp, vp, dbl, vp, i64, vp],
        "pm_domains_or": [vp, i32, i64, vp, vp],
        "pm_support_from_domains": [vp, vp, vp, ctypes.c_uint64, vp, vp],
        "pm_enumerate": [vp, vp, dbl, vp, vp, i64, ctypes.POINTER(i64)],
        "pm_plan_capture_each": [vp, vp, dbl, dbl],
        "pm_plan_pattern_bytes": [vp, vp],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.pm_free_graph.argtypes = [vp]
    lib.pm_free_graph.restype = None
    lib.pm_server_destroy.argtypes = [vp]
    lib.pm_server_destroy.restype = None
    lib.pm_free_plan.argtypes = [vp]
    lib.pm_free_plan.restype = None
    lib.pm_strerror.argtypes = [ctypes.c_int]
    lib.pm_strerror.restype = ctypes.c_char_p
    lib.pm_last_error.argtypes = []
    lib.pm_last_error.restype = ctypes.c_char_p
    return lib


_lib = _load()

# Exported symbols of the C ABI (include/pm.h).
ABI_SYMBOLS = [
    "pm_set_allocator", "pm_load_graph", "pm_graph_get_info", "pm_graph_vertex_order",
    "pm_free_graph", "pm_plan", "pm_plan_get_info", "pm_plan_matched", "pm_free_plan",
    "pm_morph", "pm_count", "pm_count_roots", "pm_support", "pm_strerror", "pm_last_error",
    "pm_plan_export", "pm_count_instrumented", "pm_plan_last_kernel_ms", "pm_plan_select",
    "pm_plan_autotune", "pm_count_c4_noalloc", "pm_fsm", "pm_plan_capture",
    "pm_server_create", "pm_server_submit", "pm_server_wait", "pm_server_get_stats",
    "pm_server_destroy", "pm_plan_set_launch", "pm_count_each", "pm_plan_query_columns",
    "pm_plan_pattern_ms", "pm_plan_last_launches", "pm_support_roots", "pm_domains_or",
    "pm_support_from_domains", "pm_enumerate", "pm_plan_capture_each", "pm_plan_pattern_bytes",
    "pm_prepare_csr",
]


def lib():
    return _lib


def _check(status, where):
    if status != PM_OK:
        raise (PMTimeout if status == PM_ETIMEOUT else PMError)(status, where)


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


_torch_alloc_refs = None


def use_torch_allocator():
    """Route the library's device allocations through torch's caching allocator."""
    global _torch_alloc_refs
    import torch

    def alloc(nbytes, device, _ctx):
        try:
            return torch.cuda.caching_allocator_alloc(nbytes, device)
        except Exception:
            return None

    def free(ptr, _nbytes, _device, _ctx):
        torch.cuda.caching_allocator_delete(ptr)

    refs = (_ALLOC_FN(alloc), _FREE_FN(free))
    _check(_lib.pm_set_allocator(ctypes.cast(refs[0], ctypes.c_void_p),
                                 ctypes.cast(refs[1], ctypes.c_void_p), None), "pm_set_allocator")
    _torch_alloc_refs = refs


def use_cuda_allocator():
    global _torch_alloc_refs
    _check(_lib.pm_set_allocator(None, None, None), "pm_set_allocator")
    _torch_alloc_refs = None


def fsm(graph, max_edges, threshold, mode=MORPH_NAIVE, stream=None, timeout_s=0.0, cap=1 << 16):
    """pm_fsm: every candidate of every level as (k, edge_mask, labels),
    with its MNI support and frequent flag."""
    while True:
        arr = (c_pattern * cap)()
        sup = np.zeros(cap, dtype=np.uint64)
        freq = np.zeros(cap, dtype=np.uint8)
        n = ctypes.c_int32()
        st = _lib.pm_fsm(graph.handle, int(max_edges), int(threshold), int(mode), _stream_handle(stream),
                         float(timeout_s), arr, _ptr(sup), _ptr(freq), int(cap), ctypes.byref(n))
        if st == PM_EOVERFLOW:
            cap = int(n.value)
            continue
        _check(st, "pm_fsm")
        pats = [(arr[i].k, arr[i].edge_mask, list(arr[i].label)[:arr[i].k]) for i in range(n.value)]
        return pats, [int(x) for x in sup[:n.value]], [bool(x) for x in freq[:n.value]]


def count_c4_noalloc(rowptr, col, n, out, stream=None):
    """pm_count_c4_noalloc: edge-induced 4-cycle count of a device CSR into
    `out` (2 device uint64 words), with no device allocation in the call.
    rowptr, col and out are CUDA tensors (int64, int32, 2 x int64) the caller
    owns; the call is asynchronous on the stream.  The tensors' types, device,
    layout and sizes are checked here (PMError with PM_EINVAL otherwise), so
    the kernel never reads past them; reading rowptr[n] costs one device to
    host copy."""
    n = int(n)
    bad = None
    for name, t, dt in (("rowptr", rowptr, "int64"), ("col", col, "int32"), ("out", out, "int64")):
        if not getattr(t, "is_cuda", False):
            bad = f"{name} must be a CUDA tensor"
        elif str(t.dtype) != f"torch.{dt}":
            bad = f"{name} must have dtype {dt}, not {t.dtype}"
        elif not t.is_contiguous():
            bad = f"{name} must be contiguous"
        if bad:
            break
    if bad is None:
        if not (rowptr.device == col.device == out.device):
            bad = "rowptr, col and out must be on one device"
        elif n < 1 or rowptr.numel() != n + 1:
            bad = f"rowptr must hold n + 1 = {n + 1} offsets (has {rowptr.numel()})"
        elif out.numel() < 2:
            bad = "out must hold 2 words"
        elif col.numel() < int(rowptr[-1].item()):
            bad = "col is shorter than rowptr[n]"
    if bad is not None:
        raise PMError(PM_EINVAL, f"count_c4_noalloc: {bad}")
    _check(_lib.pm_count_c4_noalloc(ctypes.c_void_p(rowptr.data_ptr()), ctypes.c_void_p(col.data_ptr()),
                                    int(n), ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)),
           "pm_count_c4_noalloc")


def domains_or(parts, stream=None):
    """OR of a stack of equally shaped device bitsets (parts[0] | parts[1] | ...),
    computed by the library (pm_domains_or)."""
    import torch
    parts = parts.contiguous()
    out = torch.empty(parts.shape[1:], dtype=parts.dtype, device=parts.device)
    words = out.numel()
    _check(_lib.pm_domains_or(parts.data_ptr(), int(parts.shape[0]), int(words), out.data_ptr(),
                              _stream_handle(stream)), "pm_domains_or")
    return out


def make_pattern(k, edge_mask, induced=EDGE_INDUCED, labels=None):
    p = c_pattern()
    p.k = k
    p.edge_mask = edge_mask
    for u in range(MAX_K):
        p.label[u] = -1 if labels is None or u >= k else int(labels[u])
    p.induced = induced
    return p


def _words_to_ints(words):
    w = np.asarray(words, dtype=np.uint64).reshape(-1, 2)
    return [int(lo) | (int(hi) << 64) for lo, hi in w]


def prepare_csr(n, src, dst):
    """pm_prepare_csr: the host half of graph loading alone, on no device.
    Returns (rowptr int64[n+1], col int32[rowptr[n]], new_id int32[n],
    lowdeg int64[n]): the degree-ordered CSR with sorted rows that
    pm_load_graph uploads, the internal id of each caller vertex, and per
    internal id its neighbours below it."""
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    n = int(n)
    rowptr = np.zeros(max(n, 0) + 1, dtype=np.int64)
    col = np.empty(max(1, 2 * len(src)), dtype=np.int32)
    new_id = np.empty(max(n, 0), dtype=np.int32)
    lowdeg = np.empty(max(n, 0), dtype=np.int64)
    _check(_lib.pm_prepare_csr(n, len(src), _ptr(src), _ptr(dst), _ptr(rowptr), _ptr(col), _ptr(new_id),
                               _ptr(lowdeg)), "pm_prepare_csr")
    return rowptr, col[:rowptr[-1]].copy(), new_id, lowdeg


class Graph:
    """A data graph resident on one GPU (pm_load_graph)."""

    def __init__(self, n, src, dst, labels=None, device=0, stream=None):
        src = np.ascontiguousarray(src, dtype=np.int32)
        dst = np.ascontiguousarray(dst, dtype=np.int32)
        lab = None if labels is None else np.ascontiguousarray(labels, dtype=np.uint8)
        h = ctypes.c_void_p()
        _check(_lib.pm_load_graph(int(n), len(src), _ptr(src), _ptr(dst), _ptr(lab), int(device),
                                  _stream_handle(stream), ctypes.byref(h)), "pm_load_graph")
        self._h = h

    @property
    def handle(self):
        return self._h

    def info(self):
        i = c_graph_info()
        _check(_lib.pm_graph_get_info(self._h, ctypes.byref(i)), "pm_graph_get_info")
        return {f: getattr(i, f) for f, _ in c_graph_info._fields_}

    def vertex_order(self):
        n = self.info()["n"]
        out = np.empty(n, dtype=np.int32)
        _check(_lib.pm_graph_vertex_order(self._h, _ptr(out)), "pm_graph_vertex_order")
        return out

    def free(self):
        if self._h:
            _lib.pm_free_graph(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Plan:
    """A planned query set (pm_plan): morph selection plus matching plans."""

    def __init__(self, graph, patterns, op=OP_COUNT, mode=MORPH_NAIVE):
        """graph may be None: the plan then only serves morph() / export_plans()."""
        arr = (c_pattern * len(patterns))(*patterns)
        h = ctypes.c_void_p()
        _check(_lib.pm_plan(None if graph is None else graph.handle, arr, len(patterns), op, mode,
                            ctypes.byref(h)), "pm_plan")
        self._h = h
        self.graph = graph      # keep the graph alive while the plan lives
        i = c_plan_info()
        _check(_lib.pm_plan_get_info(self._h, ctypes.byref(i)), "pm_plan_get_info")
        self.n_queries, self.n_matched, self.n_plans = i.n_queries, i.n_matched, i.n_plans

    def matched_patterns(self):
        arr = (c_pattern * self.n_matched)()
        _check(_lib.pm_plan_matched(self._h, arr), "pm_plan_matched")
        return [(p.k, p.edge_mask, p.induced, list(p.label)[:p.k]) for p in arr]

    def export_plans(self, family=PLANS_ROOTED):
        """The compiled plans of one family as a numpy structured array (pm_plan_export)."""
        level = np.dtype([("isect", "u1"), ("diff", "u1"), ("lt", "u1"), ("gt", "u1"),
                          ("neq", "u1"), ("label", "i1"), ("column", "u1"), ("vertex", "u1")])
        rec = np.dtype([("k", "<i4"), ("n_enum", "<i4"), ("tail", "<i4"), ("closed", "<i4"),
                        ("counter", "<i4"), ("dom_base", "<i4"), ("n_columns", "<i4"),
                        ("split", "<i4"), ("task_space", "<i4"), ("kind", "<i4"),
                        ("pair", "<i4"), ("pad", "<i4"),
                        ("lv", level, (8,))])
        out = np.zeros(self.n_plans if family == PLANS_ROOTED else self.n_matched, dtype=rec)
        _check(_lib.pm_plan_export(self._h, family, _ptr(out), out.nbytes), "pm_plan_export")
        return out

    def select(self, family):
        """Force a plan family for count()/support() (PLANS_AUTO = autotuned)."""
        _check(_lib.pm_plan_select(self._h, family), "pm_plan_select")

    def set_launch(self, mode):
        """LAUNCH_PER_PATTERN (default) or LAUNCH_SINGLE (one persistent launch)."""
        _check(_lib.pm_plan_set_launch(self._h, mode), "pm_plan_set_launch")

    def capture(self, stream=None, timeout_s=0.0):
        """Record this plan's pm_count as a CUDA graph; count() then replays it."""
        _check(_lib.pm_plan_capture(self._h, _stream_handle(stream), float(timeout_s)), "pm_plan_capture")

    def capture_each(self, timeout_per_pattern_s=0.0, timeout_total_s=0.0, stream=None):
        """Record count_each (deadlines fixed) as a CUDA graph replayed by count_each()."""
        _check(_lib.pm_plan_capture_each(self._h, _stream_handle(stream), float(timeout_per_pattern_s),
                                         float(timeout_total_s)), "pm_plan_capture_each")

    def autotune(self, stream=None):
        fam = np.zeros(self.n_matched, dtype=np.int32)
        _check(_lib.pm_plan_autotune(self._h, _stream_handle(stream), _ptr(fam)), "pm_plan_autotune")
        return [int(x) for x in fam]

    def morph(self, matched_counts):
        m = np.zeros(2 * self.n_matched, dtype=np.uint64)
        for j, v in enumerate(matched_counts):
            v %= 1 << 128
            m[2 * j], m[2 * j + 1] = v & ((1 << 64) - 1), v >> 64
        out = np.zeros(2 * self.n_queries, dtype=np.uint64)
        _check(_lib.pm_morph(self._h, _ptr(m), _ptr(out)), "pm_morph")
        return _words_to_ints(out)

    def count(self, stream=None, timeout_s=0.0, with_matched=False):
        out = np.zeros(2 * self.n_queries, dtype=np.uint64)
        mat = np.zeros(2 * self.n_matched, dtype=np.uint64)
        _check(_lib.pm_count(self._h, _stream_handle(stream), float(timeout_s), _ptr(out), _ptr(mat)),
               "pm_count")
        return (_words_to_ints(out), _words_to_ints(mat)) if with_matched else _words_to_ints(out)

    def last_kernel_ms(self):
        """Device time of the matching kernel of the last count/support call."""
        v = ctypes.c_float()
        _check(_lib.pm_plan_last_kernel_ms(self._h, ctypes.byref(v)), "pm_plan_last_kernel_ms")
        return float(v.value)

    def pattern_bytes(self):
        """Algorithmic bytes per matched pattern of the last count_instrumented()."""
        b = np.zeros(self.n_matched, dtype=np.uint64)
        _check(_lib.pm_plan_pattern_bytes(self._h, _ptr(b)), "pm_plan_pattern_bytes")
        return [int(x) for x in b]

    def last_launches(self):
        """Library kernels launched by the last count()."""
        v = np.zeros(1, dtype=np.int64)
        _check(_lib.pm_plan_last_launches(self._h, _ptr(v)), "pm_plan_last_launches")
        return int(v[0])

    def pattern_ms(self):
        """Device time of each matched pattern in the last count() (per-pattern launches)."""
        ms = np.zeros(self.n_matched, dtype=np.float32)
        _check(_lib.pm_plan_pattern_ms(self._h, _ptr(ms)), "pm_plan_pattern_ms")
        return [float(x) for x in ms]

    def count_each(self, timeout_per_pattern_s=0.0, timeout_total_s=0.0, stream=None):
        """(counts, statuses): a deadline per matched pattern, a status per query."""
        out = np.zeros(2 * self.n_queries, dtype=np.uint64)
        st = np.zeros(self.n_queries, dtype=np.int32)
        _check(_lib.pm_count_each(self._h, _stream_handle(stream), float(timeout_per_pattern_s),
                                  float(timeout_total_s), _ptr(out), _ptr(st)), "pm_count_each")
        return _words_to_ints(out), [int(x) for x in st]

    def count_instrumented(self, stream=None):
        """(counts, algorithmic bytes read by the matching) from an instrumented run."""
        out = np.zeros(2 * self.n_queries, dtype=np.uint64)
        b = np.zeros(1, dtype=np.uint64)
        _check(_lib.pm_count_instrumented(self._h, _stream_handle(stream), _ptr(out), _ptr(b)),
               "pm_count_instrumented")
        return _words_to_ints(out), int(b[0])

    def count_roots(self, roots, stream=None, timeout_s=0.0, with_matched=False):
        r = np.ascontiguousarray(roots, dtype=np.int32)
        out = np.zeros(2 * self.n_queries, dtype=np.uint64)
        mat = np.zeros(2 * self.n_matched, dtype=np.uint64)
        _check(_lib.pm_count_roots(self._h, _stream_handle(stream), float(timeout_s), _ptr(r), len(r),
                                   _ptr(out), _ptr(mat)), "pm_count_roots")
        return (_words_to_ints(out), _words_to_ints(mat)) if with_matched else _words_to_ints(out)

    def query_columns(self):
        """Per query, the MNI column of each of its k vertices."""
        cols = np.zeros(self.n_queries * MAX_K, dtype=np.int32)
        _check(_lib.pm_plan_query_columns(self._h, _ptr(cols)), "pm_plan_query_columns")
        return [[int(c) for c in cols[i * MAX_K:(i + 1) * MAX_K] if c >= 0] for i in range(self.n_queries)]

    def support(self, threshold=0, stream=None, timeout_s=0.0, domains=False):
        """MNI supports and frequent flags; with domains=True also the MNI
        columns, per query a list of device bitsets (torch int32 tensors of
        ceil(n / 32) words, bit v = caller vertex v), written by the library."""
        sup = np.zeros(self.n_queries, dtype=np.uint64)
        freq = np.zeros(self.n_queries, dtype=np.uint8)
        dom = None
        if domains:
            import torch
            cols = self.query_columns()
            total = sum(max(c) + 1 for c in cols)
            words = (self.graph.info()["n"] + 31) // 32
            dev = torch.device("cuda", self.graph.info()["device"])
            dom = torch.empty((total, words), dtype=torch.int32, device=dev)
        _check(_lib.pm_support(self._h, _stream_handle(stream), float(timeout_s), int(threshold),
                               _ptr(sup), _ptr(freq), dom.data_ptr() if dom is not None else None),
               "pm_support")
        out = [int(x) for x in sup], [bool(x) for x in freq]
        if not domains:
            return out
        per_query, at = [], 0
        for c in cols:
            per_query.append(dom[at:at + max(c) + 1])
            at += max(c) + 1
        return out + (per_query,)

    def enumerate(self, cap=1 << 20, stream=None, timeout_s=0.0):
        """Every occurrence of every query (pm_enumerate): a list of
        (query index, tuple of caller vertex ids indexed by query vertex)."""
        while True:
            tup = np.zeros((max(cap, 1), MAX_K), dtype=np.int32)
            qof = np.zeros(max(cap, 1), dtype=np.int32)
            n = ctypes.c_int64(0)
            st = _lib.pm_enumerate(self._h, _stream_handle(stream), float(timeout_s), _ptr(tup), _ptr(qof),
                                   int(cap), ctypes.byref(n))
            if st == PM_EOVERFLOW and n.value > cap:
                cap = int(n.value)
                continue
            _check(st, "pm_enumerate")
            return [(int(qof[r]), tuple(int(x) for x in tup[r] if x >= 0)) for r in range(n.value)]

    def _columns_tensor(self):
        import torch
        total = sum(max(c) + 1 for c in self.query_columns())
        info = self.graph.info()
        return torch.empty((total, (info["n"] + 31) // 32), dtype=torch.int32,
                           device=torch.device("cuda", info["device"]))

    def support_roots(self, roots, stream=None, timeout_s=0.0):
        """MNI columns (all queries, one row of ceil(n / 32) words each) over
        the matches whose highest-ranked vertex is among `roots` (caller ids)."""
        r = np.ascontiguousarray(roots, dtype=np.int32)
        out = self._columns_tensor()
        _check(_lib.pm_support_roots(self._h, _stream_handle(stream), float(timeout_s), _ptr(r), len(r),
                                     out.data_ptr()), "pm_support_roots")
        return out

    def support_from_domains(self, columns, threshold=0, stream=None):
        """(supports, frequent flags) from a complete set of MNI columns."""
        sup = np.zeros(self.n_queries, dtype=np.uint64)
        freq = np.zeros(self.n_queries, dtype=np.uint8)
        _check(_lib.pm_support_from_domains(self._h, columns.data_ptr(), _stream_handle(stream),
                                            int(threshold), _ptr(sup), _ptr(freq)),
               "pm_support_from_domains")
        return [int(x) for x in sup], [bool(x) for x in freq]

    def free(self):
        if self._h:
            _lib.pm_free_plan(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Server:
    """pm_server: continuous batching of count requests over loaded graphs."""

    def __init__(self, graphs, workers_per_graph=2, max_batch_patterns=256,
                 hbm_budget_bytes=64 << 30, batch_timeout_s=0.0, batch_total_s=0.0,
                 mode=MORPH_NAIVE, family=PLANS_AUTO, request_timeout_s=0.0):
        self.graphs = list(graphs)
        arr = (ctypes.c_void_p * len(self.graphs))(*[g.handle for g in self.graphs])
        cfg = c_server_config(workers_per_graph, max_batch_patterns, int(hbm_budget_bytes),
                              float(batch_timeout_s), float(batch_total_s), mode, family,
                              float(request_timeout_s))
        h = ctypes.c_void_p()
        _check(_lib.pm_server_create(arr, len(self.graphs), ctypes.byref(cfg), ctypes.byref(h)),
               "pm_server_create")
        self._h = h
        self._nq = {}

    def submit(self, graph, patterns):
        arr = (c_pattern * len(patterns))(*patterns)
        rid = ctypes.c_uint64()
        _check(_lib.pm_server_submit(self._h, int(graph), arr, len(patterns), ctypes.byref(rid)),
               "pm_server_submit")
        self._nq[rid.value] = len(patterns)
        return rid.value

    def wait(self, rid, timeout_s=-1.0, per_query=False):
        """(done, counts or None, latency_s, status); with per_query=True a
        fifth item, each query's own status."""
        nq = self._nq[rid]
        out = np.zeros(2 * nq, dtype=np.uint64)
        qst = np.zeros(nq, dtype=np.int32)
        done = ctypes.c_int32()
        lat = ctypes.c_double()
        st = ctypes.c_int()
        _check(_lib.pm_server_wait(self._h, ctypes.c_uint64(rid), float(timeout_s), ctypes.byref(done),
                                   _ptr(out), ctypes.byref(lat), ctypes.byref(st), _ptr(qst)),
               "pm_server_wait")
        if not done.value:
            return (False, None, None, None) + ((None,) if per_query else ())
        del self._nq[rid]
        res = (True, _words_to_ints(out), lat.value, st.value)
        return res + ([int(x) for x in qst],) if per_query else res

    def stats(self):
        s = c_server_stats()
        _check(_lib.pm_server_get_stats(self._h, ctypes.byref(s)), "pm_server_get_stats")
        return {f: getattr(s, f) for f, _ in c_server_stats._fields_}

    def close(self):
        if self._h:
            _lib.pm_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
