"""Comparison helpers shared by the GPU parity tests.

Tolerances (floating point, from the arithmetic):
* per-pixel sums and means of t in [0, 1]: the GPU adds at most 32 float32
  values per lane and a 5-level warp tree before a float64 atomic, so its
  relative error is below (32 + 5) * 2^-24 ~ 2.2e-6; tests use 1e-5 relative.
  The range-query bins read t from fixed-point prefix tables that hold
  floor(t * 2^95), so every cell adds an absolute error below 2^-95 as well:
  the bound is 1e-5 |sum| + count * 2^-95 (it matters only where t is below
  ~1e-24, e.g. a linear field spanning tens of decades).
* y = alpha of the mean: exact, except when the float64 mean lies within
  1e-5 relative of a TF bucket boundary, where either neighbouring entry is
  accepted (the GPU sum order differs from the CPU's).
Everything integer (keys, order, widths, F, Q, counts) and min/max (exact
float32 values of t) must match bit for bit.
"""
import numpy as np

import oracle

REL = 1e-5


def assert_bins_match(g: dict, o: dict, m: int, T: int, alpha_row: np.ndarray):
    """g: GPU bins of field m (dvl_read_bins); o: oracle.update output."""
    cnt = o["count"]
    assert np.array_equal(g["count"], cnt), "counts differ"
    assert np.array_equal(g["min"].view(np.uint32), o["min"][m].view(np.uint32)), "min differs"
    assert np.array_equal(g["max"].view(np.uint32), o["max"][m].view(np.uint32)), "max differs"
    ref = o["sum"][m]
    err = np.abs(g["sum"] - ref)
    fix = cnt.astype(np.float64) * 2.0 ** -95 + 1e-38
    assert np.all(err <= REL * np.abs(ref) + fix), f"sum rel err {np.max(err / np.maximum(ref, 1e-30))}"
    mref = o["mean64"][m]
    err = np.abs(g["mean"].astype(np.float64) - mref)
    assert np.all(err <= REL * np.abs(mref) + 2.0 ** -95 + 1e-38), "mean differs"
    # y: exact away from bucket boundaries
    x = mref * T
    near = np.abs(x - np.round(x)) <= REL * np.maximum(x, 1.0)
    ok = g["y"] == o["y"][m]
    if not np.all(ok | near):
        bad = np.nonzero(~(ok | near))[0][:5]
        raise AssertionError(f"y differs at {bad}: {g['y'][bad]} vs {o['y'][m][bad]}")
    # at boundary pixels the value must be one of the neighbouring entries
    for p in np.nonzero(near & ~ok)[0]:
        k = int(np.round(x[p]))
        cands = {float(alpha_row[min(max(k + d, 0), T - 1)]) for d in (-1, 0)}
        assert float(g["y"][p]) in cands


def assert_grad_match(grad, fields, level, ctrl, g32, width, **kw):
    """Element-wise check of a GPU control-point gradient (float32, M x K)
    computed from the float32 pixel weights g32 (M x W) against the oracle's
    gradient for the same weights.

    Both sides add per (cell, pixel) terms g/count in float64 (in different
    orders), then the GPU rounds to float32.  So for every component k:
    |gpu - ref| <= 2^-24 |ref| + (n + W + 16) 2^-53 S_k, where S_k is the
    same gradient computed with |g| (the sum of the terms' magnitudes; the
    interpolation weights are non-negative) and n + W bounds the number of
    (cell, pixel) terms.
    """
    g = np.asarray(g32, np.float32).astype(np.float64)
    target = np.zeros_like(g)
    ref = oracle.alpha_grad(fields, level, ctrl, target, width=width, g=g, **kw)["grad"]
    mag = oracle.alpha_grad(fields, level, ctrl, target, width=width, g=np.abs(g), **kw)["grad"]
    n = fields.shape[1]
    bound = 2.0 ** -24 * np.abs(ref) + (n + width + 16) * 2.0 ** -53 * mag + 1e-300
    err = np.abs(np.asarray(grad, np.float64) - ref)
    bad = err > bound
    assert not np.any(bad), f"{int(bad.sum())} components off, worst ratio {np.max(err / bound):.3g}"
