"""Thin ctypes binding of libgt.so (include/gt.h): argument marshalling only.

Every step of the transposition runs in the library's CUDA kernels; this
module converts torch tensors / numpy arrays into pointers and sizes.  If the
library has not been built, every call raises: there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgt.so")

GT_OK = 0
STATUS = {0: "GT_OK", 1: "GT_ERR_INVALID_ARG", 2: "GT_ERR_OUT_OF_RANGE", 3: "GT_ERR_BAD_ROW_PTR",
          4: "GT_ERR_NO_MEMORY", 5: "GT_ERR_CUDA", 6: "GT_ERR_TIMEOUT", 7: "GT_ERR_UNSUPPORTED"}
FLAG_AGGREGATE, FLAG_NO_GRAPH, FLAG_UNSORTED, FLAG_PARTITION_TIMES, FLAG_STEAL_TAILS = 1, 2, 4, 8, 16
METHOD_HLH = 0
METHOD_RADIX = 1


class GtError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        super().__init__(f"{what}: {STATUS.get(code, code)}")
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [("hdv_k", ctypes.c_uint32), ("table_log2", ctypes.c_uint32),
                ("block_threads", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32),
                ("warp_edges", ctypes.c_uint32), ("stage_edges", ctypes.c_uint32),
                ("sample_permille", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("method", ctypes.c_uint32), ("radix_tile", ctypes.c_uint32),
                ("seed", ctypes.c_uint64), ("batch_key_bits", ctypes.c_uint32),
                ("batch_edges_log2", ctypes.c_uint32), ("radix_digit_bits", ctypes.c_uint32),
                ("partition_bits", ctypes.c_uint32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}

    @classmethod
    def from_dict(cls, d):
        c = cls()
        for k, v in d.items():
            setattr(c, k, int(v))
        return c


class Stats(ctypes.Structure):
    _fields_ = [("hdv_selected", ctypes.c_uint32), ("partitions", ctypes.c_uint32),
                ("hdv_edges", ctypes.c_uint64), ("n_edges", ctypes.c_uint64),
                ("ldv_sorted_cols", ctypes.c_uint32), ("large_cols", ctypes.c_uint32),
                ("kernel_launches", ctypes.c_uint32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Timing(ctypes.Structure):
    _fields_ = [("calls", ctypes.c_uint32), ("sample_ms", ctypes.c_float), ("count_ms", ctypes.c_float),
                ("scan_ms", ctypes.c_float), ("scatter_ms", ctypes.c_float), ("sort_ms", ctypes.c_float),
                ("total_ms", ctypes.c_float), ("dominant_ms", ctypes.c_float),
                ("dominant_launches", ctypes.c_uint32), ("partition_ms", ctypes.c_float)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class HostTiming(ctypes.Structure):
    _fields_ = [("calls", ctypes.c_uint32), ("h2d_ms", ctypes.c_float), ("d2h_ms", ctypes.c_float),
                ("overlap_ms", ctypes.c_float), ("span_ms", ctypes.c_float)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class GraphDesc(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_uint32), ("n_cols", ctypes.c_uint32), ("n_edges", ctypes.c_uint64),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p), ("vals", ctypes.c_void_p),
                ("col_ptr", ctypes.c_void_p), ("row_idx", ctypes.c_void_p), ("vals_out", ctypes.c_void_p)]


class TuneEntry(ctypes.Structure):
    _fields_ = [("cfg", Config), ("ms", ctypes.c_float), ("score", ctypes.c_float), ("status", ctypes.c_int32)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("n_graphs", ctypes.c_uint32), ("sub_batches", ctypes.c_uint32), ("passes_max", ctypes.c_uint32),
                ("kernel_launches", ctypes.c_uint32), ("n_edges", ctypes.c_uint64),
                ("workspace_bytes", ctypes.c_uint64), ("slots", ctypes.c_uint32), ("key_bits", ctypes.c_uint32),
                ("sub_batch_edges", ctypes.c_uint64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class BatchLimits(ctypes.Structure):
    _fields_ = [("max_graphs", ctypes.c_uint32), ("max_cols", ctypes.c_uint32),
                ("max_graph_edges", ctypes.c_uint64), ("max_edges", ctypes.c_uint64),
                ("max_cols_total", ctypes.c_uint64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None

EXPORTS = ["gt_default_config", "gt_plan_create", "gt_plan_set_config", "gt_plan_get_config",
           "gt_transpose", "gt_transpose_sub", "gt_transpose_host", "gt_plan_status", "gt_plan_stats",
           "gt_plan_enable_timing", "gt_plan_timing", "gt_plan_workspace_bytes", "gt_plan_destroy",
           "gt_status_string", "gt_last_cuda_error", "gt_version", "gt_transpose_noalloc",
           "gt_batch_plan_create", "gt_transpose_batched", "gt_batch_plan_status", "gt_batch_plan_info",
           "gt_batch_plan_destroy", "gt_graph_features", "gt_tune_grid_config", "gt_tune_analytic",
           "gt_selector_param_count", "gt_selector_create", "gt_selector_get_params", "gt_selector_set_params",
           "gt_selector_forward", "gt_selector_backward", "gt_selector_adam_step", "gt_selector_destroy",
           "gt_plan_tune", "gt_plan_vertices", "gt_plan_edges", "gt_selector_in_range", "gt_transpose_host_async",
           "gt_plan_host_wait", "gt_plan_create_rect", "gt_transpose_sub_rect", "gt_plan_shape",
           "gt_graph_features_rect", "gt_plan_host_timing",
           "gt_batch_limits_from_descs", "gt_batch_plan_set_config", "gt_batch_plan_get_config",
           "gt_batch_tune_grid_config", "gt_batch_plan_tune", "gt_transpose_u64",
           "gt_plan_partition_times"]

N_FEATURES = 41
TUNE_GRID = 12
SEL_HIDDEN = 64
TUNE_ANALYTIC, TUNE_EXHAUSTIVE, TUNE_LEARNED = 0, 1, 2
BATCH_TUNE_GRID = 6


def load():
    """Loads libgt.so; raises if it was not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                           "(the CUDA library is required; there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
    lib.gt_default_config.argtypes = [ctypes.POINTER(Config), u32, u64]
    lib.gt_plan_create.argtypes = [ctypes.POINTER(P), u32, u64, ctypes.c_int, ctypes.POINTER(Config), P]
    lib.gt_plan_create_rect.argtypes = [ctypes.POINTER(P), u32, u32, u64, ctypes.c_int, ctypes.POINTER(Config), P]
    lib.gt_plan_create_rect.restype = ctypes.c_int
    lib.gt_plan_shape.argtypes = [P, ctypes.POINTER(u32), ctypes.POINTER(u32), ctypes.POINTER(u64)]
    lib.gt_plan_shape.restype = ctypes.c_int
    lib.gt_plan_set_config.argtypes = [P, ctypes.POINTER(Config)]
    lib.gt_plan_get_config.argtypes = [P, ctypes.POINTER(Config)]
    lib.gt_transpose.argtypes = [P, P, P, P, P, P, P, P]
    lib.gt_transpose_host.argtypes = [P, P, P, P, P, P, P, P]
    lib.gt_transpose_host_async.argtypes = [P, P, P, P, P, P, P, P]
    lib.gt_transpose_host_async.restype = ctypes.c_int
    lib.gt_plan_host_wait.argtypes = [P]
    lib.gt_plan_host_wait.restype = ctypes.c_int
    lib.gt_plan_host_timing.argtypes = [P, ctypes.POINTER(HostTiming)]
    lib.gt_plan_host_timing.restype = ctypes.c_int
    lib.gt_transpose_sub.argtypes = [P, u32, u64, P, P, P, P, P, P, P]
    lib.gt_transpose_sub.restype = ctypes.c_int
    lib.gt_transpose_sub_rect.argtypes = [P, u32, u32, u64, P, P, P, P, P, P, P]
    lib.gt_transpose_sub_rect.restype = ctypes.c_int
    lib.gt_plan_status.argtypes = [P]
    lib.gt_plan_stats.argtypes = [P, ctypes.POINTER(Stats)]
    lib.gt_transpose_noalloc.argtypes = [u32, u64, P, P, P, P, P, P, P]
    lib.gt_transpose_noalloc.restype = ctypes.c_int
    lib.gt_batch_plan_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(BatchLimits), ctypes.c_int,
                                         ctypes.POINTER(Config), P]
    lib.gt_transpose_batched.argtypes = [P, u32, P, P, P]
    lib.gt_batch_limits_from_descs.argtypes = [u32, ctypes.POINTER(GraphDesc), ctypes.POINTER(BatchLimits)]
    lib.gt_batch_plan_set_config.argtypes = [P, ctypes.POINTER(Config)]
    lib.gt_batch_plan_get_config.argtypes = [P, ctypes.POINTER(Config)]
    lib.gt_batch_tune_grid_config.argtypes = [u32, ctypes.POINTER(Config)]
    lib.gt_batch_plan_tune.argtypes = [P, u32, P, P, u32, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(u32), P]
    lib.gt_plan_partition_times.argtypes = [P, ctypes.POINTER(ctypes.c_float), u32, ctypes.POINTER(u32)]
    lib.gt_plan_partition_times.restype = ctypes.c_int
    lib.gt_transpose_u64.argtypes = [u64, u64, u64, P, P, P, P, P, P, P]
    lib.gt_transpose_u64.restype = ctypes.c_int
    for f in ["gt_batch_limits_from_descs", "gt_batch_plan_set_config", "gt_batch_plan_get_config",
              "gt_batch_tune_grid_config", "gt_batch_plan_tune", "gt_transpose_u64",
           "gt_plan_partition_times"]:
        getattr(lib, f).restype = ctypes.c_int
    lib.gt_batch_plan_status.argtypes = [P]
    lib.gt_batch_plan_info.argtypes = [P, ctypes.POINTER(BatchInfo)]
    lib.gt_batch_plan_destroy.argtypes = [P]
    lib.gt_batch_plan_destroy.restype = None
    for f in ["gt_batch_plan_create", "gt_transpose_batched", "gt_batch_plan_status", "gt_batch_plan_info"]:
        getattr(lib, f).restype = ctypes.c_int
    F = ctypes.c_float
    lib.gt_graph_features.argtypes = [u32, u64, ctypes.c_int, P, P, u64, P, P]
    lib.gt_graph_features_rect.argtypes = [u32, u32, u64, ctypes.c_int, P, P, u64, P, P]
    lib.gt_graph_features_rect.restype = ctypes.c_int
    lib.gt_tune_grid_config.argtypes = [u32, u32, u64, ctypes.POINTER(Config)]
    lib.gt_tune_analytic.argtypes = [P, u32, u64, ctypes.POINTER(u32)]
    lib.gt_selector_param_count.restype = u64
    lib.gt_selector_create.argtypes = [ctypes.POINTER(P), P, u64]
    lib.gt_selector_get_params.argtypes = [P, P]
    lib.gt_selector_set_params.argtypes = [P, P]
    lib.gt_selector_forward.argtypes = [P, P, u32, P, P]
    lib.gt_selector_backward.argtypes = [P, P, P, P, u32, P, P, P]
    lib.gt_selector_adam_step.argtypes = [P, F, F, F, F, F, P]
    lib.gt_selector_in_range.argtypes = [P, P, ctypes.POINTER(ctypes.c_int)]
    lib.gt_selector_destroy.argtypes = [P]
    lib.gt_selector_destroy.restype = None
    lib.gt_plan_tune.argtypes = [P, ctypes.c_int, P, P, P, P, P, P, P, u32, ctypes.POINTER(TuneEntry),
                                 ctypes.POINTER(u32), P]
    lib.gt_plan_vertices.argtypes = [P]
    lib.gt_plan_vertices.restype = u32
    lib.gt_plan_edges.argtypes = [P]
    lib.gt_plan_edges.restype = u64
    for f in ["gt_graph_features", "gt_tune_grid_config", "gt_tune_analytic", "gt_selector_create",
              "gt_selector_get_params", "gt_selector_set_params", "gt_selector_forward", "gt_selector_backward",
              "gt_selector_adam_step", "gt_plan_tune", "gt_selector_in_range"]:
        getattr(lib, f).restype = ctypes.c_int
    lib.gt_plan_enable_timing.argtypes = [P, ctypes.c_int]
    lib.gt_plan_timing.argtypes = [P, ctypes.POINTER(Timing)]
    lib.gt_plan_workspace_bytes.argtypes = [P]
    lib.gt_plan_workspace_bytes.restype = u64
    lib.gt_plan_destroy.argtypes = [P]
    lib.gt_plan_destroy.restype = None
    lib.gt_status_string.argtypes = [ctypes.c_int]
    lib.gt_status_string.restype = ctypes.c_char_p
    lib.gt_version.restype = u32
    lib.gt_last_cuda_error.restype = ctypes.c_char_p
    for f in ["gt_default_config", "gt_plan_create", "gt_plan_set_config", "gt_plan_get_config",
              "gt_transpose", "gt_transpose_host", "gt_plan_status", "gt_plan_stats",
              "gt_plan_enable_timing", "gt_plan_timing"]:
        getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(rc, what):
    if rc != GT_OK:
        if rc == 5 and _lib is not None:
            what = f"{what} ({_lib.gt_last_cuda_error().decode()})"
        raise GtError(rc, what)


def default_config(n: int, m: int) -> Config:
    c = Config()
    _check(load().gt_default_config(ctypes.byref(c), n, m), "gt_default_config")
    return c


def _ptr(t):
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return ctypes.c_void_p(t.data_ptr())
    return ctypes.c_void_p(t.ctypes.data)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """Owns a gt_plan: workspace for graphs with exactly n vertices and m
    edges, or, with n_cols, for n x n_cols sparse matrices with m entries."""

    def __init__(self, n: int, m: int, weighted: bool, config: Config | dict | None = None, stream=None,
                 n_cols: int | None = None):
        lib = load()
        self._lib = lib
        self.n, self.m, self.weighted = int(n), int(m), bool(weighted)
        self.n_cols = self.n if n_cols is None else int(n_cols)
        h = ctypes.c_void_p()
        if isinstance(config, dict):
            config = Config.from_dict(config)
        cfgp = ctypes.byref(config) if config is not None else None
        _check(lib.gt_plan_create_rect(ctypes.byref(h), self.n, self.n_cols, self.m, int(self.weighted), cfgp,
                                       _stream(stream) if stream is not None else None), "gt_plan_create_rect")
        self._h = h

    def shape(self):
        """(rows, columns, entries) the plan was made for."""
        r, c, e = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint64()
        _check(self._lib.gt_plan_shape(self._h, ctypes.byref(r), ctypes.byref(c), ctypes.byref(e)), "gt_plan_shape")
        return int(r.value), int(c.value), int(e.value)

    @property
    def handle(self):
        return self._h

    def config(self) -> Config:
        c = Config()
        _check(self._lib.gt_plan_get_config(self._h, ctypes.byref(c)), "gt_plan_get_config")
        return c

    def set_config(self, config: Config | dict):
        if isinstance(config, dict):
            config = Config.from_dict(config)
        _check(self._lib.gt_plan_set_config(self._h, ctypes.byref(config)), "gt_plan_set_config")

    def transpose(self, row_ptr, col_idx, vals, col_ptr, row_idx, vals_out, stream=None):
        """Enqueue CSR -> CSC on device tensors (u64/int64 row_ptr, u32/int32 col_idx)."""
        rc = self._lib.gt_transpose(self._h, _ptr(row_ptr), _ptr(col_idx), _ptr(vals), _ptr(col_ptr),
                                    _ptr(row_idx), _ptr(vals_out), _stream(stream))
        _check(rc, "gt_transpose")

    def transpose_sub(self, n, m, row_ptr, col_idx, vals, col_ptr, row_idx, vals_out, stream=None, n_cols=None):
        """Enqueue a graph (or, with n_cols, an n x n_cols matrix) no larger
        than the plan's on the plan's workspace."""
        nc = int(n) if n_cols is None else int(n_cols)
        rc = self._lib.gt_transpose_sub_rect(self._h, int(n), nc, int(m), _ptr(row_ptr), _ptr(col_idx), _ptr(vals),
                                             _ptr(col_ptr), _ptr(row_idx), _ptr(vals_out), _stream(stream))
        _check(rc, "gt_transpose_sub_rect")

    def transpose_host(self, row_ptr, col_idx, vals, col_ptr, row_idx, vals_out, stream=None):
        """CSR -> CSC on host arrays (pinned recommended); synchronous, returns status."""
        rc = self._lib.gt_transpose_host(self._h, _ptr(row_ptr), _ptr(col_idx), _ptr(vals), _ptr(col_ptr),
                                         _ptr(row_idx), _ptr(vals_out), _stream(stream))
        _check(rc, "gt_transpose_host")

    def transpose_host_async(self, row_ptr, col_idx, vals, col_ptr, row_idx, vals_out, stream=None):
        """Enqueue CSR -> CSC on pinned host arrays without waiting (see host_wait)."""
        rc = self._lib.gt_transpose_host_async(self._h, _ptr(row_ptr), _ptr(col_idx), _ptr(vals), _ptr(col_ptr),
                                               _ptr(row_idx), _ptr(vals_out), _stream(stream))
        _check(rc, "gt_transpose_host_async")

    def host_timing(self) -> dict:
        t = HostTiming()
        _check(self._lib.gt_plan_host_timing(self._h, ctypes.byref(t)), "gt_plan_host_timing")
        return t.as_dict()

    def host_wait(self):
        _check(self._lib.gt_plan_host_wait(self._h), "gt_plan_host_wait")

    def status(self) -> int:
        return self._lib.gt_plan_status(self._h)

    def check(self):
        _check(self.status(), "device status")

    def stats(self) -> dict:
        s = Stats()
        _check(self._lib.gt_plan_stats(self._h, ctypes.byref(s)), "gt_plan_stats")
        return s.as_dict()

    def enable_timing(self, on: bool = True):
        _check(self._lib.gt_plan_enable_timing(self._h, int(on)), "gt_plan_enable_timing")

    def timing(self) -> dict:
        t = Timing()
        _check(self._lib.gt_plan_timing(self._h, ctypes.byref(t)), "gt_plan_timing")
        return t.as_dict()

    def partition_times(self):
        """Step 3's per-partition busy times (ms) of the last call (GT_FLAG_PARTITION_TIMES)."""
        cnt = ctypes.c_uint32()
        _check(self._lib.gt_plan_partition_times(self._h, None, 0, ctypes.byref(cnt)), "gt_plan_partition_times")
        buf = (ctypes.c_float * max(1, cnt.value))()
        _check(self._lib.gt_plan_partition_times(self._h, buf, cnt.value, ctypes.byref(cnt)),
               "gt_plan_partition_times")
        return [float(x) for x in buf[:cnt.value]]

    def workspace_bytes(self) -> int:
        return int(self._lib.gt_plan_workspace_bytes(self._h))

    def tune(self, mode, row_ptr, col_idx, vals, col_ptr, row_idx, vals_out, selector=None, reps=3, stream=None):
        """gt_plan_tune: installs the chosen grid point; returns (index, table)."""
        table = (TuneEntry * TUNE_GRID)()
        chosen = ctypes.c_uint32()
        rc = self._lib.gt_plan_tune(self._h, int(mode), selector.handle if selector is not None else None,
                                    _ptr(row_ptr), _ptr(col_idx), _ptr(vals), _ptr(col_ptr), _ptr(row_idx),
                                    _ptr(vals_out), int(reps), table, ctypes.byref(chosen), _stream(stream))
        _check(rc, "gt_plan_tune")
        rows = [{"cfg": t.cfg.as_dict(), "ms": float(t.ms), "score": float(t.score), "status": int(t.status)}
                for t in table]
        return int(chosen.value), rows

    def close(self):
        if getattr(self, "_h", None):
            self._lib.gt_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchPlan:
    """Owns a gt_batch_plan and the device descriptor / status arrays of a
    graph list.

    graphs: sequence of dicts with n, m, row_ptr, col_idx, vals, col_ptr,
    row_idx, vals_out (torch tensors or raw device addresses) and, for an
    n x n_cols matrix, n_cols.  limits (dict of gt_batch_limits fields, or
    None = the limits of `graphs`) sizes the plan; transpose() runs the
    plan's own graph list, transpose_descs() any device descriptor array."""

    def __init__(self, graphs, weighted: bool, config: Config | dict | None = None, stream=None, limits=None):
        import torch
        lib = load()
        self._lib = lib
        self._h = None
        arr = (GraphDesc * max(1, len(graphs)))()

        def addr(x):
            if x is None:
                return None
            return x if isinstance(x, int) else x.data_ptr()
        for i, g in enumerate(graphs):
            arr[i] = GraphDesc(int(g["n"]), int(g.get("n_cols", 0)), int(g["m"]), addr(g["row_ptr"]), addr(g["col_idx"]),
                               addr(g.get("vals")), addr(g["col_ptr"]), addr(g["row_idx"]), addr(g.get("vals_out")))
        lim = BatchLimits()
        if limits is None:
            _check(lib.gt_batch_limits_from_descs(len(graphs), arr, ctypes.byref(lim)), "gt_batch_limits_from_descs")
        else:
            for k, v in limits.items():
                setattr(lim, k, int(v))
        if isinstance(config, dict):
            config = Config.from_dict(config)
        h = ctypes.c_void_p()
        cfgp = ctypes.byref(config) if config is not None else None
        _check(lib.gt_batch_plan_create(ctypes.byref(h), ctypes.byref(lim), int(weighted), cfgp, None),
               "gt_batch_plan_create")
        self._h = h
        self.n_graphs = len(graphs)
        raw = bytes(arr)[:ctypes.sizeof(GraphDesc) * len(graphs)] or bytes(16)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.d_descs = torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(dev)
        self.d_status = torch.zeros(max(1, len(graphs)), dtype=torch.int32, device=dev)

    def transpose(self, stream=None):
        self.transpose_descs(self.n_graphs, self.d_descs, self.d_status, stream)

    def transpose_descs(self, n_graphs, d_descs, d_status=None, stream=None):
        """gt_transpose_batched on a device descriptor array (tensor or
        address) and an optional device int32 status array."""
        dp = d_descs if isinstance(d_descs, int) else d_descs.data_ptr()
        sp = None if d_status is None else (d_status if isinstance(d_status, int) else d_status.data_ptr())
        _check(self._lib.gt_transpose_batched(self._h, int(n_graphs), dp, sp, _stream(stream)),
               "gt_transpose_batched")

    def graph_status(self):
        """Per-graph status codes of the last transpose() (synchronises)."""
        import torch
        torch.cuda.synchronize()
        return self.d_status[:self.n_graphs].cpu().tolist()

    def status(self) -> int:
        return self._lib.gt_batch_plan_status(self._h)

    def check(self):
        _check(self.status(), "batch device status")

    def info(self) -> dict:
        b = BatchInfo()
        _check(self._lib.gt_batch_plan_info(self._h, ctypes.byref(b)), "gt_batch_plan_info")
        return b.as_dict()

    def config(self) -> Config:
        c = Config()
        _check(self._lib.gt_batch_plan_get_config(self._h, ctypes.byref(c)), "gt_batch_plan_get_config")
        return c

    def set_config(self, config: Config | dict):
        if isinstance(config, dict):
            config = Config.from_dict(config)
        _check(self._lib.gt_batch_plan_set_config(self._h, ctypes.byref(config)), "gt_batch_plan_set_config")

    def tune(self, reps=3, stream=None):
        """gt_batch_plan_tune on the plan's graph list: (chosen index, ms per grid point)."""
        table = (ctypes.c_float * BATCH_TUNE_GRID)()
        chosen = ctypes.c_uint32()
        _check(self._lib.gt_batch_plan_tune(self._h, self.n_graphs, self.d_descs.data_ptr(), self.d_status.data_ptr(),
                                            int(reps), table, ctypes.byref(chosen), _stream(stream)),
               "gt_batch_plan_tune")
        return int(chosen.value), [float(x) for x in table]

    def close(self):
        if getattr(self, "_h", None):
            self._lib.gt_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_grid_config(index: int) -> Config:
    c = Config()
    _check(load().gt_batch_tune_grid_config(int(index), ctypes.byref(c)), "gt_batch_tune_grid_config")
    return c


def grid_config(index: int, n: int, m: int) -> Config:
    c = Config()
    _check(load().gt_tune_grid_config(int(index), int(n), int(m), ctypes.byref(c)), "gt_tune_grid_config")
    return c


def graph_features(row_ptr, col_idx, weighted: bool, seed: int = 0x5EED0001, out=None, stream=None, n_cols=None):
    """gt_graph_features_rect into a device f32 tensor of N_FEATURES
    (allocated if out is None); n_cols defaults to the row count."""
    import torch
    n = row_ptr.numel() - 1
    nc = n if n_cols is None else int(n_cols)
    m = col_idx.numel()
    if out is None:
        out = torch.empty(N_FEATURES, dtype=torch.float32, device=row_ptr.device)
    _check(load().gt_graph_features_rect(n, nc, m, int(weighted), _ptr(row_ptr), _ptr(col_idx), int(seed),
                                         _ptr(out), _stream(stream)), "gt_graph_features_rect")
    return out


def analytic_index(features_host, n: int, m: int) -> int:
    """gt_tune_analytic on a host float32 numpy array of N_FEATURES."""
    import numpy as np
    f = np.ascontiguousarray(features_host, dtype=np.float32)
    idx = ctypes.c_uint32()
    _check(load().gt_tune_analytic(ctypes.c_void_p(f.ctypes.data), int(n), int(m), ctypes.byref(idx)),
           "gt_tune_analytic")
    return int(idx.value)


class Selector:
    """Owns a gt_selector (MLP on the device; forward/backward/Adam in libgt)."""

    def __init__(self, params=None, seed: int = 1):
        import numpy as np
        lib = load()
        self._lib = lib
        self.n_params = int(lib.gt_selector_param_count())
        h = ctypes.c_void_p()
        arr = None
        if params is not None:
            arr = np.ascontiguousarray(params, dtype=np.float32)
            if arr.size != self.n_params:
                raise ValueError(f"expected {self.n_params} parameters, got {arr.size}")
        _check(lib.gt_selector_create(ctypes.byref(h), None if arr is None else ctypes.c_void_p(arr.ctypes.data),
                                      int(seed)), "gt_selector_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def params(self):
        import numpy as np
        out = np.empty(self.n_params, dtype=np.float32)
        _check(self._lib.gt_selector_get_params(self._h, ctypes.c_void_p(out.ctypes.data)), "gt_selector_get_params")
        return out

    def set_params(self, params):
        import numpy as np
        arr = np.ascontiguousarray(params, dtype=np.float32)
        if arr.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {arr.size}")
        _check(self._lib.gt_selector_set_params(self._h, ctypes.c_void_p(arr.ctypes.data)), "gt_selector_set_params")

    def forward(self, features, out=None, stream=None):
        import torch
        b = features.shape[0]
        if out is None:
            out = torch.empty(b, TUNE_GRID, dtype=torch.float32, device=features.device)
        _check(self._lib.gt_selector_forward(self._h, _ptr(features), b, _ptr(out), _stream(stream)),
               "gt_selector_forward")
        return out

    def backward(self, features, target, mask, loss=None, grads=None, stream=None):
        b = features.shape[0]
        _check(self._lib.gt_selector_backward(self._h, _ptr(features), _ptr(target), _ptr(mask), b, _ptr(loss),
                                              _ptr(grads), _stream(stream)), "gt_selector_backward")

    def in_range(self, features_host) -> bool:
        import numpy as np
        f = np.ascontiguousarray(features_host, dtype=np.float32)
        ok = ctypes.c_int()
        _check(self._lib.gt_selector_in_range(self._h, ctypes.c_void_p(f.ctypes.data), ctypes.byref(ok)),
               "gt_selector_in_range")
        return bool(ok.value)

    def adam_step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0, stream=None):
        _check(self._lib.gt_selector_adam_step(self._h, float(lr), float(beta1), float(beta2), float(eps),
                                               float(weight_decay), _stream(stream)), "gt_selector_adam_step")

    @classmethod
    def pretrained(cls):
        """The selector trained by selector_train.py on the library's own
        timings (parameters shipped beside this module)."""
        import numpy as np
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "selector_params.f32")
        return cls(np.fromfile(path, dtype="<f4"))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.gt_selector_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def transpose_u64(row_ptr, col_idx, vals=None, n_cols=None, stream=None):
    """gt_transpose_u64 on device tensors with 64-bit IDs (row_ptr int64[n_rows+1],
    col_idx int64[m], vals float32[m] or None); allocates the outputs and
    returns (col_ptr int64[n_cols+1], row_idx int64[m], vals_out or None).
    Synchronous; raises GtError on any non-OK status."""
    import torch
    n_rows = row_ptr.numel() - 1
    nc = n_rows if n_cols is None else int(n_cols)
    m = col_idx.numel()
    dev = row_ptr.device
    col_ptr = torch.empty(nc + 1, dtype=torch.int64, device=dev)
    row_idx = torch.empty(m, dtype=torch.int64, device=dev)
    vals_out = torch.empty(m, dtype=torch.float32, device=dev) if vals is not None else None
    rc = load().gt_transpose_u64(n_rows, nc, m, _ptr(row_ptr), _ptr(col_idx), _ptr(vals), _ptr(col_ptr),
                                 _ptr(row_idx), _ptr(vals_out), _stream(stream))
    _check(rc, "gt_transpose_u64")
    return col_ptr, row_idx, vals_out


def transpose_noalloc(row_ptr, col_idx, vals, col_ptr, row_idx, vals_out, stream=None):
    """gt_transpose_noalloc on caller-owned device tensors (no device allocation
    inside the call; synchronous).  Raises GtError on any non-OK status."""
    n = row_ptr.numel() - 1
    m = col_idx.numel()
    rc = load().gt_transpose_noalloc(n, m, _ptr(row_ptr), _ptr(col_idx), _ptr(vals), _ptr(col_ptr),
                                     _ptr(row_idx), _ptr(vals_out), _stream(stream))
    _check(rc, "gt_transpose_noalloc")


def transpose(row_ptr, col_idx, vals=None, config=None, stream=None, check=True, n_cols=None):
    """Convenience: allocate outputs (torch, same device) and transpose once
    (an n x n_cols matrix when n_cols is given, else a graph)."""
    import torch
    n = row_ptr.numel() - 1
    nc = n if n_cols is None else int(n_cols)
    m = col_idx.numel()
    dev = col_idx.device if m else row_ptr.device
    col_ptr = torch.empty(nc + 1, dtype=torch.int64, device=dev)
    row_idx = torch.empty(m, dtype=torch.int32, device=dev)
    vals_out = torch.empty(m, dtype=torch.float32, device=dev) if vals is not None else None
    plan = Plan(n, m, vals is not None, config, stream, n_cols=nc)
    try:
        plan.transpose(row_ptr, col_idx, vals, col_ptr, row_idx, vals_out, stream)
        if check:
            plan.check()
    finally:
        plan.close()
    return col_ptr, row_idx, vals_out
