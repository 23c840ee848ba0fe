"""Pins of the oracle's line-plot rasterisation (CPU only).

A hand-worked image (tests/golden/raster_4x5.json) fixes the row mapping and
the split of each segment between its two columns; seeded random plots are
checked against the properties that define a drawn polyline and bar plot,
with the value rows recomputed here from the float32 mapping: every column of
a line is one run of rows through its own value's row, neighbouring columns
touch (8-connected), a segment's rows are all drawn by its two columns and
none beyond its end rows, and bars fill from the value's row to the baseline.
"""
import json
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "raster_4x5.json")


def test_golden_image():
    g = json.load(open(GOLDEN))
    lines, bars = oracle.rasterize(np.array(g["values"], np.float32), g["H"], g["bar_field"])
    assert np.array_equal(lines, np.array(g["lines"], np.uint8))
    assert np.array_equal(bars, np.array(g["bars"], np.uint8))


def _rows(v, H):
    x = (np.float32(1.0) - v.astype(np.float32)) * np.float32(H - 1)
    return np.clip(np.floor(x + np.float32(0.5)).astype(np.int64), 0, H - 1)


@pytest.mark.parametrize("M,W,H,seed", [(1, 1, 1, 0), (1, 7, 1, 1), (4, 64, 33, 2), (8, 300, 128, 3),
                                        (3, 1000, 2, 4), (2, 50, 500, 5)])
def test_polyline_and_bar_properties(M, W, H, seed):
    rng = np.random.default_rng(seed)
    v = rng.uniform(0, 1, (M, W)).astype(np.float32)
    v[:, rng.integers(0, W, max(1, W // 10))] = rng.choice([0.0, 1.0])   # extremes
    bar_field = M - 1
    lines, bars = oracle.rasterize(v, H, bar_field)
    r = _rows(v, H)
    for m in range(M):
        cov = (lines >> m) & 1
        lo = np.full(W, -1)
        hi = np.full(W, -1)
        for p in range(W):
            rows = np.nonzero(cov[:, p])[0]
            assert rows.size, "every column of a line is drawn"
            lo[p], hi[p] = rows[0], rows[-1]
            assert rows.size == hi[p] - lo[p] + 1, "one contiguous run"
            assert lo[p] <= r[m, p] <= hi[p], "through the value's own row"
            nb = [r[m, q] for q in (p - 1, p, p + 1) if 0 <= q < W]
            assert min(nb) <= lo[p] and hi[p] <= max(nb), "not beyond the segments' end rows"
        for p in range(W - 1):
            assert max(lo[p], lo[p + 1]) <= min(hi[p], hi[p + 1]) + 1, "8-connected"
            a, b = sorted((r[m, p], r[m, p + 1]))
            for row in range(a, b + 1):
                assert cov[row, p] or cov[row, p + 1], "the segment has no gap"
    for p in range(W):
        col = bars[:, p]
        assert col.sum() == H - r[bar_field, p] and np.all(col[r[bar_field, p]:] == 1)


def test_constant_plot_is_one_row():
    v = np.full((2, 20), 0.3, np.float32)
    lines, bars = oracle.rasterize(v, 11, 1)
    row = int(np.floor(np.float32(0.7) * np.float32(10) + np.float32(0.5)))
    assert np.all(lines[row] == 3) and lines.sum() == 3 * 20
    assert bars[row:].all() and not bars[:row].any()


def test_rasterize_rejects_bad_arguments():
    with pytest.raises(oracle.OracleError):
        oracle.rasterize(np.zeros((9, 4), np.float32), 4)
    with pytest.raises(oracle.OracleError):
        oracle.rasterize(np.zeros((2, 4), np.float32), 4, bar_field=2)
