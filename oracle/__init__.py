"""CPU oracle of the dynamic-volume-line computation -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``dvl_oracle.c`` (a plain,
sequential C restatement of the paper's Eq. 1-6 and Sec. 3.2) with ctypes and
numpy; ``brute.py`` holds an independent exact-rational brute force for tiny
inputs.  The CUDA library never imports, links or calls anything here.

Parity status per function (see the tests that pin each one):

* ``keys``       -- pinned: Morton against recursive Z-order traversal; Hilbert
                    against bijectivity, unit steps and octree contiguity.
* ``order``      -- pinned: against numpy's stable argsort.
* ``update``     -- pinned: exact-rational brute force (``brute.py``), the P = 0
                    closed form, constant-field closed forms, hand-worked golden
                    fixtures, and sum/count invariants.  Its threaded form
                    (``threads`` > 1, ``orc_update_mt``) is pinned to the
                    sequential one bit for bit; ``keys(threads=)`` likewise.
* ``alpha_grad`` -- pinned: float64 central differences (the loss is quadratic
                    in the control points once the assignment is fixed; with
                    given pixel weights ``g`` the functional is linear).
* ``rasterize``  -- pinned: a hand-worked golden image and the properties that
                    define the drawing (contiguous columns through the value's
                    row, 8-connected segments, bar heights).
* ``widths``     -- pinned: equal to ``update``'s per-cell widths for every
                    cell of a data set, given that data set's global quantities.
* ``log10f``, ``log_fields`` -- pinned: float64 log10 within 2 ulp over the
                    whole positive float range (subnormals included), exact
                    values at 1 and at powers of two with 16-bit logs, and the
                    clamp of values <= 0 to the smallest positive value.
* ``brush``, ``select_keys`` -- pinned: the exact-rational brute force's bins
                    give the same selections; hand-built key ranges.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dvl_oracle.c")
_HDR = os.path.join(_HERE, "dvl_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

SFC_MORTON, SFC_HILBERT = 0, 1
MINIMP_BEFORE_SCALE, MINIMP_AFTER_POWER = 0, 1
VMAX_APPROX, VMAX_EXACT = 0, 1
WIDTH_EDGE, WIDTH_VOLUME = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with strict IEEE semantics (no contraction)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"])
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [("P", ctypes.c_float), ("min_importance", ctypes.c_float),
                ("width", ctypes.c_uint32), ("min_imp_mode", ctypes.c_uint32),
                ("vmax_mode", ctypes.c_uint32), ("width_mode", ctypes.c_uint32)]


class Stats(ctypes.Structure):
    _fields_ = [("vmax", ctypes.c_float), ("inv_vmax", ctypes.c_float),
                ("f_upper", ctypes.c_float), ("Q", ctypes.c_int32), ("i", ctypes.c_int32),
                ("j", ctypes.c_int32), ("linear", ctypes.c_int32), ("pow_exact", ctypes.c_int32),
                ("F", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def _L():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        vp, u64, u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32
        _lib.orc_keys.argtypes = [u64, vp, vp, vp, vp, ctypes.c_int, vp]
        _lib.orc_order.argtypes = [u64, vp, vp]
        _lib.orc_update.argtypes = [u64, u32, vp, vp, u32, vp, vp, vp, ctypes.POINTER(Params)] + [vp] * 10 + [ctypes.POINTER(Stats)]
        _lib.orc_update_mt.argtypes = _lib.orc_update.argtypes + [ctypes.c_int]
        _lib.orc_keys_mt.argtypes = [u64, vp, vp, vp, vp, ctypes.c_int, vp, ctypes.c_int]
        _lib.orc_rasterize.argtypes = [u32, u32, u32, vp, u32, vp, vp]
        _lib.orc_brush.argtypes = [u64, vp, vp, u32, u32, vp, vp]
        _lib.orc_widths.argtypes = [u64, u32, vp, vp, u32, u32, vp, ctypes.POINTER(Params), u64, vp, vp, vp, vp, vp]
        _lib.orc_select_keys.argtypes = [u64, vp, u32, vp, vp]
        _lib.orc_select_keys.restype = None
        _lib.orc_alpha_grad.argtypes = [u64, u32, vp, vp, u32, u32, vp, vp, vp, ctypes.POINTER(Params), vp, vp, vp,
                                        vp, vp]
        _lib.orc_log10f.argtypes = [ctypes.c_float]
        _lib.orc_log10f.restype = ctypes.c_float
        _lib.orc_log_field.argtypes = [u64, vp]
        for f in (_lib.orc_keys, _lib.orc_keys_mt, _lib.orc_order, _lib.orc_update, _lib.orc_update_mt,
                  _lib.orc_alpha_grad, _lib.orc_log_field):
            f.restype = ctypes.c_int
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


class OracleError(RuntimeError):
    pass


def keys(lower: np.ndarray, level: np.ndarray, sfc: int, threads: int = 1) -> np.ndarray:
    """u64 space-filling-curve key per cell (Morton or Hilbert of the exact
    centroid 2*lower + 2^level, 21 bits per axis).  ``threads`` > 1 computes
    contiguous ranges of the cells at once (same keys)."""
    lower = np.ascontiguousarray(lower, np.int32)
    level = np.ascontiguousarray(level, np.uint8)
    n = level.shape[0]
    out = np.empty(n, np.uint64)
    if threads > 1:
        rc = _L().orc_keys_mt(n, _p(lower[0]), _p(lower[1]), _p(lower[2]), _p(level), sfc, _p(out), threads)
    else:
        rc = _L().orc_keys(n, _p(lower[0]), _p(lower[1]), _p(lower[2]), _p(level), sfc, _p(out))
    if rc:
        raise OracleError(f"orc_keys failed: {rc}")
    return out


def order(k: np.ndarray) -> np.ndarray:
    """Stable permutation sorting the keys (ties keep input order)."""
    k = np.ascontiguousarray(k, np.uint64)
    perm = np.empty(k.shape[0], np.uint32)
    rc = _L().orc_order(k.shape[0], _p(k), _p(perm))
    if rc:
        raise OracleError(f"orc_order failed: {rc}")
    return perm


def params(P=1.0, min_importance=0.025, width=1024, min_imp_mode=0, vmax_mode=0, width_mode=0):
    return Params(P, min_importance, width, min_imp_mode, vmax_mode, width_mode)


def update(fields: np.ndarray, level: np.ndarray, alpha: np.ndarray, dom_lo=None, dom_hi=None,
           per_cell: bool = False, threads: int = 1, **kw) -> dict:
    """One DVL update over cells already in curve order.

    ``fields`` (M, N) float32, ``level`` (N,) uint8, ``alpha`` (M, T) float32.
    ``dom_lo``/``dom_hi`` per field (NaN = data range).  Keyword arguments are
    :func:`params`.  Returns bins (sum/min/max/mean/mean64/y per field and the
    shared count), stats, and with ``per_cell`` the widths q and bins b1, b2.
    ``threads`` > 1 runs ``orc_update_mt``, which gives the same results bit
    for bit on that many host threads.
    """
    prm = params(**kw)
    fields = np.ascontiguousarray(fields, np.float32)
    level = np.ascontiguousarray(level, np.uint8)
    alpha = np.ascontiguousarray(alpha, np.float32)
    M, n = fields.shape
    T = alpha.shape[1]
    W = prm.width
    lo = np.full(M, np.nan, np.float32) if dom_lo is None else np.ascontiguousarray(dom_lo, np.float32)
    hi = np.full(M, np.nan, np.float32) if dom_hi is None else np.ascontiguousarray(dom_hi, np.float32)
    out = dict(sum=np.empty((M, W), np.float64), min=np.empty((M, W), np.float32),
               max=np.empty((M, W), np.float32), mean=np.empty((M, W), np.float32),
               mean64=np.empty((M, W), np.float64), y=np.empty((M, W), np.float32),
               count=np.empty(W, np.uint32))
    if per_cell:
        out.update(q=np.empty(n, np.uint64), b1=np.empty(n, np.uint32), b2=np.empty(n, np.uint32))
    st = Stats()
    args = (n, M, _p(fields), _p(level), T, _p(alpha), _p(lo), _p(hi), ctypes.byref(prm),
            _p(out["sum"]), _p(out["min"]), _p(out["max"]), _p(out["mean"]),
            _p(out["mean64"]), _p(out["y"]), _p(out["count"]), _p(out.get("q")),
            _p(out.get("b1")), _p(out.get("b2")), ctypes.byref(st))
    rc = _L().orc_update_mt(*args, int(threads)) if threads > 1 else _L().orc_update(*args)
    if rc:
        raise OracleError(f"orc_update failed: {rc}")
    out["stats"] = st.as_dict()
    return out


def alpha_grad(fields, level, ctrl, target, T=256, dom_lo=None, dom_hi=None, g=None, **kw) -> dict:
    """Loss, per-pixel mean alpha and its gradient w.r.t. the control points.

    With ``g`` (M, W), the gradient is that of sum(g * abar) instead (g takes
    the place of dL/dabar = 2 (abar - target))."""
    prm = params(**kw)
    fields = np.ascontiguousarray(fields, np.float32)
    level = np.ascontiguousarray(level, np.uint8)
    ctrl = np.ascontiguousarray(ctrl, np.float32)
    target = np.ascontiguousarray(target, np.float64)
    g = None if g is None else np.ascontiguousarray(g, np.float64)
    M, n = fields.shape
    K = ctrl.shape[1]
    W = prm.width
    lo = np.full(M, np.nan, np.float32) if dom_lo is None else np.ascontiguousarray(dom_lo, np.float32)
    hi = np.full(M, np.nan, np.float32) if dom_hi is None else np.ascontiguousarray(dom_hi, np.float32)
    abar = np.empty((M, W), np.float64)
    grad = np.empty((M, K), np.float64)
    loss = np.zeros(1, np.float64)
    rc = _L().orc_alpha_grad(n, M, _p(fields), _p(level), T, K, _p(ctrl), _p(lo), _p(hi),
                             ctypes.byref(prm), _p(target), _p(g), _p(abar), _p(grad), _p(loss))
    if rc:
        raise OracleError(f"orc_alpha_grad failed: {rc}")
    return dict(loss=float(loss[0]), abar=abar, grad=grad)


def sorted_inputs(lower, level, fields, sfc):
    """Sorted keys, permutation (perm[k] = input index of the k-th cell in
    curve order) and the cells' level/fields gathered into curve order."""
    k = keys(lower, level, sfc)
    perm = order(k)
    return k[perm], perm, np.ascontiguousarray(level[perm]), np.ascontiguousarray(fields[:, perm])


def rasterize(values: np.ndarray, height: int, bar_field: int = 0):
    """(lines, bars) uint8 images (height, W) of the (M, W) bin values in [0, 1]."""
    v = np.ascontiguousarray(values, np.float32)
    M, W = v.shape
    lines = np.zeros((height, W), np.uint8)
    bars = np.zeros((height, W), np.uint8)
    rc = _L().orc_rasterize(M, W, height, _p(v), bar_field, _p(lines), _p(bars))
    if rc:
        raise OracleError(f"orc_rasterize failed ({rc})")
    return lines, bars


def brush(b1: np.ndarray, b2: np.ndarray, p0: int, p1: int):
    """(first, last) cell of the pixel ROI [p0, p1] in curve order, or None."""
    b1 = np.ascontiguousarray(b1, np.uint32)
    b2 = np.ascontiguousarray(b2, np.uint32)
    f = np.zeros(1, np.uint64)
    l = np.zeros(1, np.uint64)
    rc = _L().orc_brush(b1.size, _p(b1), _p(b2), p0, p1, _p(f), _p(l))
    if rc == 1:
        return None
    if rc:
        raise OracleError(f"orc_brush failed ({rc})")
    return int(f[0]), int(l[0])


def select_keys(keys: np.ndarray, ranges) -> np.ndarray:
    """uint8 mask of the cells whose key lies in one of the inclusive ranges."""
    k = np.ascontiguousarray(keys, np.uint64)
    r = np.ascontiguousarray(np.asarray(ranges, np.uint64).reshape(-1))
    mask = np.zeros(k.size, np.uint8)
    _L().orc_select_keys(k.size, _p(k), r.size // 2, _p(r), _p(mask))
    return mask


def widths(n_total: int, dmin, dmax, max_level: int, alpha: np.ndarray, values: np.ndarray, level: np.ndarray,
           **kw):
    """Widths of sampled cells (values (M, k), level (k,)) of a data set of
    n_total cells with the given per-field data range and deepest level.
    Returns (q, Q, vmax)."""
    v = np.ascontiguousarray(values, np.float32)
    lv = np.ascontiguousarray(level, np.uint8)
    a = np.ascontiguousarray(alpha, np.float32)
    M, k = v.shape
    lo = np.ascontiguousarray(dmin, np.float32)
    hi = np.ascontiguousarray(dmax, np.float32)
    q = np.empty(k, np.uint64)
    Q = np.zeros(1, np.int32)
    vm = np.zeros(1, np.float32)
    p = params(**kw)
    rc = _L().orc_widths(n_total, M, _p(lo), _p(hi), max_level, a.shape[1], _p(a), ctypes.byref(p), k, _p(v),
                         _p(lv), _p(q), _p(Q), _p(vm))
    if rc:
        raise OracleError(f"orc_widths failed ({rc})")
    return q, int(Q[0]), float(vm[0])


def log10f(x) -> np.ndarray:
    """The log10 of the per-field log scale, element by element (float32,
    every value > 0)."""
    v = np.array(x, np.float32, copy=True).reshape(-1)
    if not np.all(v > 0):
        raise OracleError("log10f needs positive values")
    if v.size:
        _L().orc_log_field(v.size, _p(v))
    return v.reshape(np.shape(x))


def log_fields(fields: np.ndarray, log_mask: int) -> np.ndarray:
    """Copy of fields (M, n) with every field m whose bit is set in log_mask
    replaced by its log10 (values <= 0 take the smallest positive value)."""
    out = np.array(fields, np.float32, copy=True, order="C")
    for m in range(out.shape[0]):
        if log_mask >> m & 1:
            row = np.ascontiguousarray(out[m])
            rc = _L().orc_log_field(row.size, _p(row))
            if rc:
                raise OracleError(f"field {m}: no positive value for the log scale ({rc})")
            out[m] = row
    return out
