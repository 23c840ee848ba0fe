"""B300-native dynamic volume lines for multi-field AMR data.

Thin ctypes binding over the C ABI of ``include/dvl.h`` (``lib/libdvl.so``,
built from ``csrc/`` by ``_build.py``).  This module only marshals arguments:
every step of the computation runs in the library's CUDA kernels.  It does not
fall back to anything if the library is missing -- importing it then raises.

Host arrays are numpy arrays (or CPU torch tensors); device arrays are CUDA
torch tensors on the context's device.  PyTorch provides device memory and the
stream; it computes nothing here.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from ._build import LIB as _LIB_PATH

__all__ = ["DVL", "DVLError", "lib", "SFC_MORTON", "SFC_HILBERT"]

OK, ERR_ARG, ERR_STATE, ERR_NOMEM, ERR_CUDA, ERR_RANGE, ERR_TIMEOUT, ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7
SFC_MORTON, SFC_HILBERT = 0, 1
MEM_HOST, MEM_DEVICE = 0, 1
MINIMP_BEFORE_SCALE, MINIMP_AFTER_POWER = 0, 1
VMAX_APPROX, VMAX_EXACT = 0, 1
WIDTH_EDGE, WIDTH_VOLUME = 0, 1
OPT_SPIN_LIMIT, OPT_FAULT_NO_PUBLISH, OPT_TIMING, OPT_ENTRIES = 1, 2, 3, 4
PLOT_MEAN, PLOT_Y = 0, 1
SCALE_LINEAR, SCALE_LOG10 = 0, 1

EXPORTS = ["dvl_create", "dvl_destroy", "dvl_load_amr", "dvl_build_order", "dvl_set_fields",
           "dvl_set_tf", "dvl_set_tfs", "dvl_update", "dvl_read_bins", "dvl_read_bins_all", "dvl_get_stats", "dvl_read_order",
           "dvl_read_widths", "dvl_sync", "dvl_set_option", "dvl_get_timings", "dvl_update_noalloc", "dvl_set_tf_ctrl", "dvl_read_alpha_means", "dvl_backward",
           "dvl_update_batch", "dvl_read_batch_bins", "dvl_read_batch_all", "dvl_batch_config",
           "dvl_read_batch_all_async", "dvl_stream", "dvl_rasterize", "dvl_brush", "dvl_select_keys",
           "dvl_set_field_scale", "dvl_read_values", "dvl_read_data_range",
           "dvl_status_string", "dvl_last_error",
           "dvl_server_create", "dvl_server_destroy", "dvl_server_add_dataset", "dvl_server_warmup",
           "dvl_server_submit", "dvl_server_wait", "dvl_server_get_stats", "dvl_server_reset_stats",
           "dvl_server_timeline", "dvl_server_last_error", "dvl_serve_bucket", "dvl_serve_admit"]


class dvl_params(ctypes.Structure):
    _fields_ = [("P", ctypes.c_float), ("min_importance", ctypes.c_float), ("width", ctypes.c_uint32),
                ("min_imp_mode", ctypes.c_uint32), ("vmax_mode", ctypes.c_uint32),
                ("width_mode", ctypes.c_uint32), ("want_alpha", ctypes.c_uint32)]


class dvl_bins(ctypes.Structure):
    _fields_ = [("mean", ctypes.c_void_p), ("min", ctypes.c_void_p), ("max", ctypes.c_void_p),
                ("y", ctypes.c_void_p), ("sum", ctypes.c_void_p), ("count", ctypes.c_void_p),
                ("mem_kind", ctypes.c_int)]


class dvl_roi(ctypes.Structure):
    _fields_ = [("first", ctypes.c_uint64), ("last", ctypes.c_uint64), ("n_cells", ctypes.c_uint64),
                ("key_first", ctypes.c_uint64), ("key_last", ctypes.c_uint64)]


class dvl_server_config(ctypes.Structure):
    _fields_ = [("mem_budget", ctypes.c_uint64), ("max_batch", ctypes.c_uint32), ("max_inflight", ctypes.c_uint32),
                ("n_entries", ctypes.c_uint32), ("max_width", ctypes.c_uint32), ("params", dvl_params)]


class dvl_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("mean_batch", ctypes.c_double), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("cells_per_s", ctypes.c_double), ("mem_used", ctypes.c_uint64), ("mem_budget", ctypes.c_uint64),
                ("slot_bytes", ctypes.c_uint64), ("n_datasets", ctypes.c_uint32), ("max_batch_seen", ctypes.c_uint32)]


class dvl_batch_span(ctypes.Structure):
    _fields_ = [("dataset", ctypes.c_uint32), ("requests", ctypes.c_uint32), ("start_ms", ctypes.c_double),
                ("end_ms", ctypes.c_double), ("run_start_ms", ctypes.c_double), ("run_end_ms", ctypes.c_double)]


class dvl_stats(ctypes.Structure):
    _fields_ = [("vmax", ctypes.c_float), ("inv_vmax", ctypes.c_float), ("f_upper", ctypes.c_float),
                ("Q", ctypes.c_int32), ("i", ctypes.c_int32), ("j", ctypes.c_int32),
                ("linear", ctypes.c_int32), ("pow_exact", ctypes.c_int32), ("F", ctypes.c_uint64),
                ("n_cells", ctypes.c_uint64), ("n_fields", ctypes.c_uint32), ("max_level", ctypes.c_uint32),
                ("entries", ctypes.c_uint32), ("pad", ctypes.c_uint32)]


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libdvl.so is not built ({_LIB_PATH}); run paper_2306_11612_b300/_build.py")
    L = ctypes.CDLL(_LIB_PATH)
    vp, u32, u64, i32, f32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_float
    sig = {
        "dvl_create": ([ctypes.POINTER(vp), i32, vp], i32),
        "dvl_destroy": ([vp], None),
        "dvl_load_amr": ([vp, u64, vp, vp, u32, vp, i32], i32),
        "dvl_build_order": ([vp, i32], i32),
        "dvl_set_fields": ([vp, u32, vp, i32], i32),
        "dvl_set_tf": ([vp, u32, vp, u32, f32, f32], i32),
        "dvl_update": ([vp, ctypes.POINTER(dvl_params)], i32),
        "dvl_read_bins": ([vp, u32, ctypes.POINTER(dvl_bins)], i32),
        "dvl_set_tfs": ([vp, u32, vp, u32, vp], i32),
        "dvl_read_bins_all": ([vp, ctypes.POINTER(dvl_bins)], i32),
        "dvl_get_stats": ([vp, ctypes.POINTER(dvl_stats)], i32),
        "dvl_read_order": ([vp, vp, vp, i32], i32),
        "dvl_read_widths": ([vp, vp, i32], i32),
        "dvl_sync": ([vp], i32),
        "dvl_set_option": ([vp, i32, ctypes.c_int64], i32),
        "dvl_get_timings": ([vp, ctypes.POINTER(ctypes.c_double), i32], i32),
        "dvl_update_noalloc": ([vp, u64, u32, vp, ctypes.c_size_t, vp, u32, vp, vp,
                                ctypes.POINTER(dvl_params), ctypes.POINTER(dvl_bins)], i32),
        "dvl_set_tf_ctrl": ([vp, vp, u32, u32, vp, i32], i32),
        "dvl_read_alpha_means": ([vp, vp, i32], i32),
        "dvl_backward": ([vp, vp, i32, vp, i32], i32),
        "dvl_update_batch": ([vp, vp, u32, u32, i32, vp, ctypes.POINTER(dvl_params), vp, vp, u32], i32),
        "dvl_read_batch_bins": ([vp, u32, u32, ctypes.POINTER(dvl_bins)], i32),
        "dvl_read_batch_all": ([vp, ctypes.POINTER(dvl_bins)], i32),
        "dvl_batch_config": ([vp, ctypes.POINTER(ctypes.c_int32)], i32),
        "dvl_read_batch_all_async": ([vp, ctypes.POINTER(dvl_bins)], i32),
        "dvl_stream": ([vp], vp),
        "dvl_rasterize": ([vp, u32, u32, u32, vp, vp, i32], i32),
        "dvl_brush": ([vp, u32, u32, ctypes.POINTER(dvl_roi), vp, i32], i32),
        "dvl_select_keys": ([vp, vp, u32, vp, i32], i32),
        "dvl_set_field_scale": ([vp, u32, i32], i32),
        "dvl_read_values": ([vp, u32, vp, i32], i32),
        "dvl_read_data_range": ([vp, vp, vp], i32),
        "dvl_server_create": ([ctypes.POINTER(vp), i32, ctypes.POINTER(dvl_server_config)], i32),
        "dvl_server_destroy": ([vp], None),
        "dvl_server_add_dataset": ([vp, u64, vp, vp, u32, vp, i32, ctypes.POINTER(u32)], i32),
        "dvl_server_warmup": ([vp], i32),
        "dvl_server_submit": ([vp, u32, vp, u32, ctypes.POINTER(u64)], i32),
        "dvl_server_wait": ([vp, u64, ctypes.c_double, ctypes.POINTER(dvl_bins)], i32),
        "dvl_server_get_stats": ([vp, ctypes.POINTER(dvl_server_stats)], i32),
        "dvl_server_reset_stats": ([vp], i32),
        "dvl_server_timeline": ([vp, vp, u32, vp], i32),
        "dvl_server_last_error": ([vp], ctypes.c_char_p),
        "dvl_serve_bucket": ([u32, u32], u32),
        "dvl_serve_admit": ([u32, u32, u32, u64, u64, u64], u32),
        "dvl_status_string": ([i32], ctypes.c_char_p),
        "dvl_last_error": ([vp], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    return L


lib = _load()


class DVLError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{lib.dvl_status_string(status).decode()} ({status}): {msg}")
        self.status = status


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr_kind(x):
    """(pointer, mem_kind, keepalive) of a numpy array or torch tensor."""
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), (MEM_DEVICE if x.is_cuda else MEM_HOST), x
    a = np.ascontiguousarray(x)
    return a.ctypes.data, MEM_HOST, a


class DVL:
    """One library context (``dvl_ctx``) on one GPU."""

    def __init__(self, device: int = 0, stream=None):
        h = ctypes.c_void_p()
        s = None
        if stream is not None:
            s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        rc = lib.dvl_create(ctypes.byref(h), device, s)
        if rc:
            raise DVLError(rc, "dvl_create")
        self._h = h
        self.device = device
        self.n = 0
        self.M = 0
        self.W = 0
        self._pairs = []

    def _check(self, rc):
        if rc:
            raise DVLError(rc, lib.dvl_last_error(self._h).decode())

    def torch_stream(self):
        """The library's CUDA stream as a torch stream (for ordering torch work)."""
        if getattr(self, "_tstream", None) is None:
            import torch
            self._tstream = torch.cuda.ExternalStream(lib.dvl_stream(self._h), device=self.device)
        return self._tstream

    def close(self):
        if getattr(self, "_h", None):
            lib.dvl_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- once per data set ----
    def dvl_load_amr(self, lower, level, fields):
        """lower (3, N) int32, level (N,) uint8, fields (M, N) float32 (all host or all device)."""
        lp, kind, k1 = _ptr_kind(lower)
        vp_, kind2, k2 = _ptr_kind(level)
        M = len(fields)
        fps = []
        keep = []
        for f in fields:
            p, k, kk = _ptr_kind(f)
            if k != kind:
                raise ValueError("all inputs must be in the same memory")
            fps.append(p)
            keep.append(kk)
        if kind2 != kind:
            raise ValueError("all inputs must be in the same memory")
        n = int(level.shape[0])
        arr = (ctypes.c_void_p * M)(*fps)
        self._check(lib.dvl_load_amr(self._h, n, lp, vp_, M, arr, kind))
        self.n, self.M = n, M

    load_amr = dvl_load_amr

    def dvl_build_order(self, sfc: int = SFC_HILBERT):
        self._check(lib.dvl_build_order(self._h, sfc))

    build_order = dvl_build_order

    def dvl_set_fields(self, fields):
        fps, keep, kind = [], [], None
        for f in fields:
            p, k, kk = _ptr_kind(f)
            kind = k if kind is None else kind
            fps.append(p)
            keep.append(kk)
        arr = (ctypes.c_void_p * len(fps))(*fps)
        self._check(lib.dvl_set_fields(self._h, len(fps), arr, kind))

    set_fields = dvl_set_fields

    def dvl_set_field_scale(self, field: int, scale: int):
        self._check(lib.dvl_set_field_scale(self._h, field, scale))

    set_field_scale = dvl_set_field_scale

    def dvl_read_values(self, field: int, out=None):
        """Field values in curve order as the update sees them (after the scale)."""
        if out is None:
            out = np.empty(self.n, np.float32)
        p, kind, _ = _ptr_kind(out)
        self._check(lib.dvl_read_values(self._h, field, p, kind))
        return out

    read_values = dvl_read_values

    def dvl_read_data_range(self):
        lo = np.empty(self.M, np.float32)
        hi = np.empty(self.M, np.float32)
        self._check(lib.dvl_read_data_range(self._h, lo.ctypes.data, hi.ctypes.data))
        return lo, hi

    read_data_range = dvl_read_data_range

    # ---- per edit ----
    def dvl_set_tf(self, field: int, alpha, lo: float = math.nan, hi: float = math.nan):
        a = np.ascontiguousarray(alpha, dtype=np.float32)
        self._check(lib.dvl_set_tf(self._h, field, a.ctypes.data, a.shape[0], lo, hi))

    set_tf = dvl_set_tf

    def dvl_set_tfs(self, alphas, lo=None, hi=None):
        """Alpha tables of all fields in one call: ``alphas`` (M, T) host
        floats; ``lo``/``hi`` per-field domains (None: data ranges)."""
        a = np.ascontiguousarray(alphas, dtype=np.float32)
        if a.ndim != 2:
            raise ValueError("alphas must be (n_fields, n_entries)")
        dom = None
        if lo is not None or hi is not None:
            M = a.shape[0]
            lo = [math.nan] * M if lo is None else lo
            hi = [math.nan] * M if hi is None else hi
            dom = (ctypes.c_float * (2 * M))(*[float(x) for x in list(lo) + list(hi)])
        self._check(lib.dvl_set_tfs(self._h, a.shape[0], a.ctypes.data, a.shape[1], dom))

    set_tfs = dvl_set_tfs

    def dvl_update(self, P=1.0, min_importance=0.025, width=1024, min_imp_mode=0, vmax_mode=0, width_mode=0,
                   want_alpha=0):
        p = dvl_params(P, min_importance, width, min_imp_mode, vmax_mode, width_mode, want_alpha)
        self._check(lib.dvl_update(self._h, ctypes.byref(p)))
        self.W = width

    update = dvl_update

    def dvl_set_tf_ctrl(self, ctrl, n_entries: int = 256, domain=None):
        """Alpha tables of all fields from (M, K) control points in [0, 1]
        (numpy / CPU tensor, or CUDA tensor: stays on the device)."""
        p, kind, keep = _ptr_kind(ctrl)
        dom = None
        if domain is not None:
            dom = (ctypes.c_float * (2 * self.M))(*[float(x) for x in domain])
        self._K = int(ctrl.shape[1])
        self._check(lib.dvl_set_tf_ctrl(self._h, p, self._K, n_entries, dom, kind))

    set_tf_ctrl = dvl_set_tf_ctrl

    def dvl_read_alpha_means(self, out=None):
        """(M, W) per-pixel mean of the cells' alpha (last update with want_alpha=1)."""
        if out is None:
            out = np.empty((self.M, self.W), np.float32)
        p, kind, keep = _ptr_kind(out)
        self._check(lib.dvl_read_alpha_means(self._h, p, kind))
        return out

    read_alpha_means = dvl_read_alpha_means

    def dvl_backward(self, grad_abar, out=None):
        """dL/dctrl (M, K) from dL/dabar (M, W), assignment frozen at the last update."""
        gp, gkind, gkeep = _ptr_kind(grad_abar)
        if out is None:
            out = np.empty((self.M, self._K), np.float32)
        op, okind, okeep = _ptr_kind(out)
        self._check(lib.dvl_backward(self._h, gp, gkind, op, okind))
        return out

    backward = dvl_backward

    def dvl_rasterize(self, height: int, value_kind: int = 1, bar_field: int = 0, lines=None, bars=None):
        """Line-plot image of the last update's bins: (lines, bars) uint8
        (height, W) arrays (numpy by default; CUDA tensors stay on the device)."""
        if lines is None and bars is None:
            lines = np.empty((height, self.W), np.uint8)
            bars = np.empty((height, self.W), np.uint8)
        pl, kl, keep_l = _ptr_kind(lines) if lines is not None else (None, None, None)
        pb, kb, keep_b = _ptr_kind(bars) if bars is not None else (None, None, None)
        kinds = {k for k in (kl, kb) if k is not None}
        if len(kinds) != 1:
            raise ValueError("outputs must be in the same memory")
        self._check(lib.dvl_rasterize(self._h, height, value_kind, bar_field, pl, pb, kinds.pop()))
        return lines, bars

    rasterize = dvl_rasterize

    def dvl_brush(self, p0: int, p1: int, mask=None):
        """Brushing a pixel ROI [p0, p1] of the last update's plot: the run of
        selected cells in curve order and its key range; ``mask=True`` also
        returns the per-cell selection (input order) as a numpy array, or pass
        an n-byte array / CUDA tensor to fill."""
        r = dvl_roi()
        if mask is True:
            mask = np.empty(self.n, np.uint8)
        pm, km, keep = _ptr_kind(mask) if mask is not None else (None, MEM_HOST, None)
        self._check(lib.dvl_brush(self._h, p0, p1, ctypes.byref(r), pm, km))
        out = {k: getattr(r, k) for k, _ in r._fields_}
        if mask is not None:
            out["mask"] = mask
        return out

    brush = dvl_brush

    def dvl_select_keys(self, ranges, mask=None):
        """Per-cell (input order) selection by inclusive curve-key ranges."""
        rr = np.ascontiguousarray(np.asarray(ranges, np.uint64).reshape(-1))
        if mask is None:
            mask = np.empty(self.n, np.uint8)
        pm, km, keep = _ptr_kind(mask)
        self._check(lib.dvl_select_keys(self._h, rr.ctypes.data, rr.size // 2, pm, km))
        return mask

    select_keys = dvl_select_keys

    @staticmethod
    def _bins_struct(W, out):
        if out is None:
            out = dict(mean=np.empty(W, np.float32), min=np.empty(W, np.float32), max=np.empty(W, np.float32),
                       y=np.empty(W, np.float32), sum=np.empty(W, np.float64), count=np.empty(W, np.uint32))
        b = dvl_bins()
        kind = None
        keep = []
        for name in ("mean", "min", "max", "y", "sum", "count"):
            if name in out and out[name] is not None:
                p, k, kk = _ptr_kind(out[name])
                if kind is not None and k != kind:
                    raise ValueError("all outputs must be in the same memory")
                kind = k
                keep.append(kk)
                setattr(b, name, p)
        b.mem_kind = kind if kind is not None else MEM_HOST
        return out, b, keep

    def dvl_read_bins(self, field: int, out: dict | None = None) -> dict:
        """Bins of one field.  ``out`` may map names (mean, min, max, y, sum,
        count) to preallocated arrays/tensors (all host or all device); by
        default fresh numpy arrays are returned."""
        out, b, keep = self._bins_struct(self.W, out)
        self._check(lib.dvl_read_bins(self._h, field, ctypes.byref(b)))
        return out

    def dvl_read_bins_all(self, out: dict | None = None) -> dict:
        """Bins of every field in one call: mean/min/max/y/sum of shape
        (M, W) (or M*W elements), count of W; one copy per array and one
        synchronisation.  ``out`` as for read_bins."""
        M, W = self.M, self.W
        if out is None:
            out = dict(mean=np.empty((M, W), np.float32), min=np.empty((M, W), np.float32),
                       max=np.empty((M, W), np.float32), y=np.empty((M, W), np.float32),
                       sum=np.empty((M, W), np.float64), count=np.empty(W, np.uint32))
        for name, x in out.items():
            if x is None:
                continue
            need = (W if name == "count" else M * W) * (8 if name == "sum" else 4)
            have = (x.numel() * x.element_size()) if hasattr(x, "numel") else x.nbytes
            if have < need:
                raise ValueError(f"out[{name!r}] holds {have} bytes, needs {need}")
        out, b, keep = self._bins_struct(0, out)
        self._check(lib.dvl_read_bins_all(self._h, ctypes.byref(b)))
        return out

    read_bins_all = dvl_read_bins_all

    def dvl_update_batch(self, alphas, pairs, domain=None, P=1.0, min_importance=0.025, min_imp_mode=0,
                         width_mode=0):
        """Batched update: ``alphas`` (K, M, T) alpha tables (numpy / CPU
        tensor, or a CUDA tensor that stays on the device), ``pairs`` a list
        of (tf_index, width); ``domain`` 2*M floats shared by all TFs (None =
        data ranges)."""
        p, kind, keep = _ptr_kind(alphas)
        K, M, T = (int(x) for x in alphas.shape)
        if self.M and M != self.M:
            raise ValueError(f"alphas has {M} fields, the data set {self.M}")
        tf = np.ascontiguousarray([q[0] for q in pairs], np.uint32)
        wd = np.ascontiguousarray([q[1] for q in pairs], np.uint32)
        dom = None
        if domain is not None:
            dom = (ctypes.c_float * (2 * self.M))(*[float(x) for x in domain])
        prm = dvl_params(P, min_importance, 1, min_imp_mode, 0, width_mode, 0)
        self._check(lib.dvl_update_batch(self._h, p, K, T, kind, dom, ctypes.byref(prm), tf.ctypes.data,
                                         wd.ctypes.data, len(pairs)))
        self._pairs = [(int(a), int(b)) for a, b in zip(tf, wd)]

    update_batch = dvl_update_batch

    def dvl_read_batch_bins(self, pair: int, field: int, out: dict | None = None) -> dict:
        """Bins of one field of pair ``pair`` of the last batched update."""
        W = self._pairs[pair][1] if 0 <= pair < len(self._pairs) else 1   # bad index: the library reports it
        out, b, keep = self._bins_struct(W, out)
        self._check(lib.dvl_read_batch_bins(self._h, pair, field, ctypes.byref(b)))
        return out

    read_batch_bins = dvl_read_batch_bins

    def batch_sizes(self):
        """(bins, counts) element totals of the last batch's layout."""
        nb = sum(self.M * w for _, w in self._pairs)
        return nb, sum(w for _, w in self._pairs)

    def dvl_read_batch_all(self, out: dict | None = None) -> dict:
        """All bins of the last batched update, pair-major (see dvl.h)."""
        nb, nc = self.batch_sizes()
        if out is None:
            out = dict(mean=np.empty(nb, np.float32), min=np.empty(nb, np.float32), max=np.empty(nb, np.float32),
                       y=np.empty(nb, np.float32), sum=np.empty(nb, np.float64), count=np.empty(nc, np.uint32))
        out, b, keep = self._bins_struct(0, out)
        self._check(lib.dvl_read_batch_all(self._h, ctypes.byref(b)))
        return out

    read_batch_all = dvl_read_batch_all

    def dvl_batch_config(self) -> dict:
        """Launch configuration chosen for the last batch shape."""
        c = (ctypes.c_int32 * 3)()
        self._check(lib.dvl_batch_config(self._h, c))
        return dict(group=c[0], ctas_per_sm=c[1], replayed=bool(c[2]))

    batch_config = dvl_batch_config

    read_bins = dvl_read_bins

    def dvl_get_stats(self) -> dict:
        s = dvl_stats()
        self._check(lib.dvl_get_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in s._fields_}

    get_stats = dvl_get_stats

    def dvl_read_order(self):
        keys = np.empty(self.n, np.uint64)
        perm = np.empty(self.n, np.uint32)
        self._check(lib.dvl_read_order(self._h, keys.ctypes.data, perm.ctypes.data, MEM_HOST))
        return keys, perm

    read_order = dvl_read_order

    def dvl_read_widths(self):
        q = np.empty(self.n, np.uint64)
        self._check(lib.dvl_read_widths(self._h, q.ctypes.data, MEM_HOST))
        return q

    read_widths = dvl_read_widths

    def dvl_sync(self):
        self._check(lib.dvl_sync(self._h))

    sync = dvl_sync

    def dvl_set_option(self, option: int, value: int):
        self._check(lib.dvl_set_option(self._h, option, value))

    set_option = dvl_set_option

    def dvl_get_timings(self):
        """Average device ms per stage over the updates timed since the last
        call (needs OPT_TIMING=1): prepare, width pass + scan, placement
        pass, finalize, and the number of updates."""
        ms = (ctypes.c_double * 5)()
        self._check(lib.dvl_get_timings(self._h, ms, 5))
        return dict(prepare=ms[0], pass_a=ms[1], pass_b=ms[2], finalize=ms[3], updates=int(ms[4]))

    get_timings = dvl_get_timings

    @property
    def handle(self):
        return self._h


def dvl_update_noalloc(stream, fields, pitch, level, alpha, domain, out, P=1.0, min_importance=0.025,
                       width=1024, min_imp_mode=0, vmax_mode=0, width_mode=0, n_cells=None):
    """Allocation-free update over caller-owned CUDA tensors (see dvl.h).

    ``fields``: float32 CUDA tensor holding M rows of ``pitch`` cells in curve
    order; ``level``: uint8 CUDA tensor; ``alpha``: (M, T) float32 CUDA tensor;
    ``domain``: 2M host floats; ``out``: dict of CUDA tensors mean/min/max/y
    (float32, M*W), sum (float64, M*W), count (int32/uint32, W).  Returns the
    status code (0 = ok) instead of raising, so callers can test rejections."""
    M, T = int(alpha.shape[0]), int(alpha.shape[1])
    n = int(level.shape[0]) if n_cells is None else int(n_cells)
    dom = (ctypes.c_float * (2 * M))(*[float(x) for x in domain])
    p = dvl_params(P, min_importance, width, min_imp_mode, vmax_mode, width_mode)
    b = dvl_bins()
    for k in ("mean", "min", "max", "y", "sum", "count"):
        setattr(b, k, out[k].data_ptr())
    b.mem_kind = MEM_DEVICE
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    return lib.dvl_update_noalloc(s, n, M, fields.data_ptr(), pitch, level.data_ptr(), T, alpha.data_ptr(),
                                  dom, ctypes.byref(p), ctypes.byref(b))
