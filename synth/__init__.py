"""Seeded synthetic AMR inputs (cells, fields, transfer functions).

Input generation only: nothing here computes any step of the dynamic-volume-line
method.  The CPU oracle, the tests and the benchmark all draw their inputs from
this module, so both sides of every parity check see identical data.

Configurations (shapes follow the paper's evaluation data, Sec. 6: four
correlated fields dens/temp/pres/velmag on multi-level AMR):

* ``small``      -- 2 levels, 32^3 base cells (level 1) in 8^3-cell bricks, 16 of
                    the 64 bricks refined once: N = 90,112, logical grid 64^3.
* ``large``      -- 6 levels, 128^3 base cells (level 5), logical grid 4096^3,
                    refinement by a density-noise threshold chosen so that
                    N is about 4.0e8.
* ``paper``      -- 4 levels, about 35.8M cells (the size of the paper's data set).
* ``batched``    -- 5 levels, about 50M cells.
* ``diff``       -- 4 levels, about 20M cells.
* generic        -- :func:`threshold_amr` with any base, depth and threshold.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "amrgen.c")
_LIB = os.path.join(_HERE, "libamrgen.so")


def build(force: bool = False) -> str:
    """Compile ``libamrgen.so`` beside its source (gcc, pthreads)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               "-o", _LIB, _SRC, "-lm"])
    return _LIB


class _Cfg(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("base_n", ctypes.c_int32),
                ("n_levels", ctypes.c_int32), ("brick", ctypes.c_int32),
                ("n_refined", ctypes.c_int32), ("n_threads", ctypes.c_int32),
                ("tau", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("box_lo", ctypes.c_int32 * 3), ("box_n", ctypes.c_int32)]


_lib = None


def _L():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        _lib.amrgen_count_sample.argtypes = [P(_Cfg), ctypes.c_int64, ctypes.c_int64]
        _lib.amrgen_count_sample.restype = ctypes.c_int64
        _lib.amrgen_count.argtypes = [P(_Cfg), ctypes.c_void_p]
        _lib.amrgen_count.restype = ctypes.c_int64
        _lib.amrgen_fill.argtypes = [P(_Cfg), ctypes.c_void_p] + [ctypes.c_void_p] * 8
        _lib.amrgen_fill.restype = ctypes.c_int
        _lib.amrgen_bricks_count.argtypes = [P(_Cfg)]
        _lib.amrgen_bricks_count.restype = ctypes.c_int64
        _lib.amrgen_bricks_fill.argtypes = [P(_Cfg)] + [ctypes.c_void_p] * 8
        _lib.amrgen_bricks_fill.restype = ctypes.c_int
        _lib.amrgen_noise.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int64,
                                      ctypes.c_void_p, ctypes.c_void_p]
        _lib.amrgen_noise.restype = None
    return _lib


@dataclass
class AMR:
    """A set of AMR cells with M scalar fields.

    ``lower`` is (3, N) int32 (x, y, z lower corners on the logical grid),
    ``level`` is (N,) uint8 with 0 = finest (cell width 2**level), ``fields``
    is (M, N) float32 (dens, temp, pres, velmag), ``grid`` the logical-grid edge.
    """
    lower: np.ndarray
    level: np.ndarray
    fields: np.ndarray
    grid: int
    meta: dict

    @property
    def n(self) -> int:
        return int(self.level.shape[0])

    def subset(self, idx) -> "AMR":
        idx = np.asarray(idx)
        return AMR(np.ascontiguousarray(self.lower[:, idx]), np.ascontiguousarray(self.level[idx]),
                   np.ascontiguousarray(self.fields[:, idx]), self.grid, dict(self.meta, subset=True))


def _alloc(n: int, pinned: bool):
    if pinned:
        import torch
        mk = lambda shape, dt: torch.empty(shape, dtype=dt, pin_memory=True).numpy()
        return (mk((3, n), torch.int32), mk((n,), torch.uint8), mk((4, n), torch.float32))
    return (np.empty((3, n), np.int32), np.empty((n,), np.uint8), np.empty((4, n), np.float32))


def _ptrs(lower, level, fields):
    return [lower[0].ctypes.data, lower[1].ctypes.data, lower[2].ctypes.data, level.ctypes.data,
            fields[0].ctypes.data, fields[1].ctypes.data, fields[2].ctypes.data, fields[3].ctypes.data]


def bricks_amr(seed: int = 1, base_n: int = 32, brick: int = 8, n_refined: int = 16,
               pinned: bool = False) -> AMR:
    """Two-level brick AMR (the ``small`` configuration with the defaults)."""
    cfg = _Cfg(1, base_n, 2, brick, n_refined, 0, 0.0, seed)
    n = _L().amrgen_bricks_count(ctypes.byref(cfg))
    if n < 0:
        raise ValueError("invalid brick configuration")
    lower, level, fields = _alloc(n, pinned)
    if _L().amrgen_bricks_fill(ctypes.byref(cfg), *_ptrs(lower, level, fields)) != 0:
        raise RuntimeError("amrgen_bricks_fill failed")
    meta = dict(kind="bricks", seed=seed, base_n=base_n, brick=brick, n_refined=n_refined, levels=2)
    return AMR(lower, level, fields, base_n * 2, meta)


def threshold_amr(base_n: int, n_levels: int, tau: float, seed: int, pinned: bool = False,
                  n_threads: int = 0, box=None) -> AMR:
    """Threshold-refined AMR: a level-L cell splits while density noise > tau.

    ``box = ((x, y, z), n)`` restricts the output to the base cells of that
    sub-box (the same cells, fields and order as in the full data set)."""
    cfg = _Cfg(0, base_n, n_levels, 0, 0, n_threads, float(tau), seed)
    if box is not None:
        cfg.box_lo[:] = [int(v) for v in box[0]]
        cfg.box_n = int(box[1])
    nb = (cfg.box_n or base_n) ** 3
    counts = np.empty(nb, np.uint32)
    n = _L().amrgen_count(ctypes.byref(cfg), counts.ctypes.data)
    offsets = np.zeros(nb, np.int64)
    np.cumsum(counts[:-1], out=offsets[1:])
    lower, level, fields = _alloc(int(n), pinned)
    _L().amrgen_fill(ctypes.byref(cfg), offsets.ctypes.data, *_ptrs(lower, level, fields))
    meta = dict(kind="threshold", seed=seed, base_n=base_n, levels=n_levels, tau=float(tau),
                box=None if box is None else [list(box[0]), int(box[1])])
    if box is None:
        meta["_base_offsets"] = np.append(offsets, np.int64(n))      # first cell of every base cell, then n
    return AMR(lower, level, fields, base_n << (n_levels - 1), meta)


def sub_box(full: AMR, box, pinned: bool = False) -> AMR:
    """The cells of a sub-box of base cells, cut out of a whole threshold
    data set: the same cells, fields and order that ``threshold_amr(...,
    box=box)`` generates (base cells are written x fastest, each one's cells
    contiguous), without evaluating the noise again."""
    off = full.meta["_base_offsets"]
    base = int(full.meta["base_n"])
    (x0, y0, z0), e = [int(v) for v in box[0]], int(box[1])
    runs = []
    for z in range(z0, z0 + e):
        for y in range(y0, y0 + e):
            b = x0 + base * (y + base * z)
            runs.append((int(off[b]), int(off[b + e])))
    n = sum(b - a for a, b in runs)
    lower, level, fields = _alloc(n, pinned)
    pos = 0
    for a, b in runs:
        k = b - a
        lower[:, pos:pos + k] = full.lower[:, a:b]
        level[pos:pos + k] = full.level[a:b]
        fields[:, pos:pos + k] = full.fields[:, a:b]
        pos += k
    meta = {k: v for k, v in full.meta.items() if k != "_base_offsets"}
    meta["box"] = [[x0, y0, z0], e]
    return AMR(lower, level, fields, full.grid, meta)


def tau_for_target(base_n: int, n_levels: int, target: int, seed: int, sample_stride: int = 0,
                   iters: int = 24) -> float:
    """Bisects the refinement threshold so that the cell count is close to
    ``target``, estimating counts on every ``sample_stride``-th base cell."""
    nb = base_n ** 3
    if sample_stride <= 0:
        sample_stride = max(1, nb // 32768)
    cfg = _Cfg(0, base_n, n_levels, 0, 0, 0, 0.0, seed)

    def est(tau):
        cfg.tau = tau
        c = _L().amrgen_count_sample(ctypes.byref(cfg), sample_stride, sample_stride // 2)
        nsel = len(range(sample_stride // 2, nb, sample_stride))
        return c * nb / nsel

    lo, hi = -6.0, 6.0          # count decreases as tau grows
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if est(mid) > target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


# Named configurations.  The thresholds of the big ones were found with
# tau_for_target (sample stride as default) and are fixed here so that a
# configuration is one deterministic data set.
CONFIGS = {
    "small": dict(kind="bricks", seed=1),
    "large": dict(kind="threshold", base_n=128, n_levels=6, target=400_000_000, seed=2),
    "paper": dict(kind="threshold", base_n=64, n_levels=4, target=35_800_000, seed=6),
    "batched": dict(kind="threshold", base_n=96, n_levels=5, target=50_000_000, seed=3),
    "diff": dict(kind="threshold", base_n=64, n_levels=4, target=20_000_000, seed=4),
}
TAU = {"diff": 0.9971523284912109, "paper": 0.7737407684326172,
       "batched": 1.8879261016845703, "large": 2.1677913665771484}


def make(name: str, pinned: bool = False, box=None, **over) -> AMR:
    """Builds a named configuration (see the module docstring); ``box``
    selects a sub-box of base cells (see :func:`threshold_amr`)."""
    c = dict(CONFIGS[name], **over)
    if c["kind"] == "bricks":
        return bricks_amr(seed=c["seed"], pinned=pinned)
    tau = c.get("tau", TAU.get(name))
    if tau is None:
        tau = tau_for_target(c["base_n"], c["n_levels"], c["target"], c["seed"])
    a = threshold_amr(c["base_n"], c["n_levels"], tau, c["seed"], pinned=pinned, box=box)
    a.meta["name"] = name
    return a


def box_count(name: str, box) -> int:
    """Cells of a named threshold configuration inside a sub-box of base
    cells, counted without generating them."""
    c = CONFIGS[name]
    cfg = _Cfg(0, c["base_n"], c["n_levels"], 0, 0, 0, float(TAU[name]), c["seed"])
    cfg.box_lo[:] = [int(v) for v in box[0]]
    cfg.box_n = int(box[1])
    counts = np.empty(int(box[1]) ** 3, np.uint32)
    return int(_L().amrgen_count(ctypes.byref(cfg), counts.ctypes.data))


def serving_boxes(seed: int = 5, n: int = 8, lo: float = 1e6, hi: float = 2e8, name: str = "large"):
    """Sub-boxes of a named data set whose cell counts are log-uniform over
    [lo, hi]: the n targets are spaced evenly in log from lo to hi (a
    stratified log-uniform draw that always spans the range); each box has a
    random corner (seeded) and its edge bisected on the count.  Returns
    [(box, count)], one per serving data set."""
    rng = np.random.Generator(np.random.PCG64(seed))
    base = CONFIGS[name]["base_n"]
    out = []
    for i in range(n):
        target = float(np.exp(np.log(lo) + (np.log(hi) - np.log(lo)) * i / max(n - 1, 1)))
        corner = rng.uniform(0.0, 1.0, 3)
        best = None
        e_lo, e_hi = 1, base
        while e_lo <= e_hi:                      # smallest edge reaching the target
            e = (e_lo + e_hi) // 2
            x0 = [int(v * (base - e)) for v in corner]
            cnt = box_count(name, (x0, e))
            if best is None or abs(np.log(max(cnt, 1) / target)) < abs(np.log(max(best[1], 1) / target)):
                best = ((x0, e), cnt)
            if cnt < target:
                e_lo = e + 1
            else:
                e_hi = e - 1
        out.append(best)
    return out


# The serving data sets: serving_boxes() (seed 5, 8 sets, log-uniform sizes
# from 1e6 to 2e8 over the "large" configuration), fixed here with their counts
# so that generating them needs no search: 1.34M ... 200.0M cells, 382.5M in
# total.
SERVING = [(((71, 71, 45), 39), 1340564), (((29, 5, 39), 24), 2447689), (((40, 4, 4), 29), 4772020),
           (((87, 57, 20), 40), 10048121), (((34, 76, 70), 49), 20096538), (((92, 43, 54), 18), 46586674),
           (((45, 4, 37), 61), 97227745), (((6, 21, 1), 103), 200000058)]


def serving_datasets(pinned: bool = False, full: AMR = None):
    """The 8 serving data sets (sub-boxes of "large", see SERVING); cut out
    of ``full`` (the whole "large" data set) when it is given."""
    if full is not None:
        return [sub_box(full, box, pinned=pinned) for box, _ in SERVING]
    return [make("large", pinned=pinned, box=box) for box, _ in SERVING]


def random_tf(rng: np.random.Generator, n_entries: int = 256, n_points: int = 8) -> np.ndarray:
    """Random piecewise-linear alpha transfer function sampled into a table.

    ``n_points`` control points: x = 0 and x = 1 plus sorted uniform interior
    positions, alpha ~ U[0, 1]; the table entry e holds the polyline's value at
    e / (n_entries - 1), evaluated in float64 and stored as float32.
    """
    xs = np.concatenate([[0.0], np.sort(rng.uniform(0.0, 1.0, n_points - 2)), [1.0]])
    ys = rng.uniform(0.0, 1.0, n_points)
    s = np.arange(n_entries, dtype=np.float64) / (n_entries - 1)
    return np.interp(s, xs, ys).astype(np.float32)


def random_tfs(seed: int, n_fields: int = 4, n_entries: int = 256, n_points: int = 8) -> np.ndarray:
    """(n_fields, n_entries) float32 tables from one seed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.stack([random_tf(rng, n_entries, n_points) for _ in range(n_fields)])


def noise(seed: int, stream: int, xyz: np.ndarray) -> np.ndarray:
    """The generator's value noise at points (n, 3) in domain units."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    out = np.empty(xyz.shape[0], np.float64)
    _L().amrgen_noise(seed, stream, xyz.shape[0], xyz.ctypes.data, out.ctypes.data)
    return out
