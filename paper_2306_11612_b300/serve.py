"""Python binding of the serving loop (include/dvl_serve.h).

Argument marshalling only: the scheduler, queues and admission run in the
library's native scheduler thread and every step of the computation in its
CUDA kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import DVLError, dvl_batch_span, dvl_bins, dvl_params, dvl_server_config, dvl_server_stats, lib, MEM_HOST

__all__ = ["DVLServer"]


class DVLServer:
    """A set of resident AMR data sets answering TF-edit requests."""

    def __init__(self, device: int = 0, *, mem_budget: int = 0, max_batch: int = 64, max_inflight: int = 8,
                 n_entries: int = 256, max_width: int = 4096, P: float = 1.0, min_importance: float = 0.025,
                 min_imp_mode: int = 0, width_mode: int = 0):
        cfg = dvl_server_config(mem_budget, max_batch, max_inflight, n_entries, max_width,
                                dvl_params(P, min_importance, 1, min_imp_mode, 0, width_mode, 0))
        h = ctypes.c_void_p()
        rc = lib.dvl_server_create(ctypes.byref(h), device, ctypes.byref(cfg))
        if rc:
            raise DVLError(rc, "dvl_server_create")
        self._h = h
        self.n_entries = n_entries
        self._M = {}
        self._W = {}

    def _check(self, rc):
        if rc:
            raise DVLError(rc, lib.dvl_server_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib.dvl_server_destroy(self._h)
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

    def add_dataset(self, lower, level, fields, sfc: int = 1) -> int:
        """Host arrays as DVL.load_amr; returns the data set's index."""
        lower = np.ascontiguousarray(lower, np.int32)
        level = np.ascontiguousarray(level, np.uint8)
        fields = [np.ascontiguousarray(f, np.float32) for f in fields]
        n = level.shape[0]
        ptrs = (ctypes.c_void_p * len(fields))(*[f.ctypes.data for f in fields])
        did = ctypes.c_uint32()
        self._check(lib.dvl_server_add_dataset(self._h, n, lower.ctypes.data, level.ctypes.data, len(fields), ptrs,
                                               sfc, ctypes.byref(did)))
        self._M[did.value] = len(fields)
        return did.value

    def warmup(self):
        self._check(lib.dvl_server_warmup(self._h))

    def submit(self, dataset: int, alpha, width: int) -> int:
        """Queues one request: ``alpha`` (M, n_entries) tables in [0, 1]."""
        a = np.ascontiguousarray(alpha, np.float32)
        rid = ctypes.c_uint64()
        self._check(lib.dvl_server_submit(self._h, dataset, a.ctypes.data, width, ctypes.byref(rid)))
        self._W[rid.value] = (dataset, width)
        return rid.value

    def wait(self, rid: int, timeout: float = -1.0) -> dict:
        """The request's bins: mean/min/max/y/sum as (M, W), count (W,)."""
        ds, W = self._W[rid]
        M = self._M[ds]
        out = dict(mean=np.empty((M, W), np.float32), min=np.empty((M, W), np.float32),
                   max=np.empty((M, W), np.float32), y=np.empty((M, W), np.float32),
                   sum=np.empty((M, W), np.float64), count=np.empty(W, np.uint32))
        b = dvl_bins(*[out[k].ctypes.data for k in ("mean", "min", "max", "y", "sum", "count")], MEM_HOST)
        rc = lib.dvl_server_wait(self._h, rid, timeout, ctypes.byref(b))
        if rc != -6:                                  # kept on a timeout (it may be waited for again)
            del self._W[rid]
        self._check(rc)
        return out

    def stats(self) -> dict:
        s = dvl_server_stats()
        self._check(lib.dvl_server_get_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in s._fields_}

    def reset_stats(self):
        self._check(lib.dvl_server_reset_stats(self._h))

    def timeline(self) -> np.ndarray:
        """The finished batches since the last reset as a structured array:
        dataset, requests, start_ms / end_ms (events on the data set's stream
        around its kernels) and run_start_ms / run_end_ms (the device clock
        when its first kernel started and its last kernel ended)."""
        n = ctypes.c_uint32()
        self._check(lib.dvl_server_timeline(self._h, None, 0, ctypes.byref(n)))
        out = (dvl_batch_span * max(n.value, 1))()
        self._check(lib.dvl_server_timeline(self._h, out, n.value, ctypes.byref(n)))
        arr = np.zeros(n.value, dtype=[("dataset", np.uint32), ("requests", np.uint32), ("start_ms", np.float64),
                                       ("end_ms", np.float64), ("run_start_ms", np.float64),
                                       ("run_end_ms", np.float64)])
        for i in range(n.value):
            o = out[i]
            arr[i] = (o.dataset, o.requests, o.start_ms, o.end_ms, o.run_start_ms, o.run_end_ms)
        return arr
