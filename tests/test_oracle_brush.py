"""Pins of the oracle's brushing and linking (Sec. 3.5) (CPU only).

The selection of a pixel ROI is checked against a direct enumeration over the
exact-rational brute force's bins (oracle/brute.py), which never uses the
oracle's fixed-point widths; the key-range selection against hand-built
ranges and numpy's searchsorted (a library routine) over the sorted keys.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle.brute import brute_update


@pytest.mark.parametrize("seed", range(12))
def test_brush_matches_brute_force_bins(seed):
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(1, 150))
    M = int(rng.integers(1, 4))
    T = 8
    W = int(rng.choice([1, 3, 16, 64]))
    fields = (rng.integers(0, 64, (M, n)) / 16.0).astype(np.float32)
    alpha = (rng.integers(0, 9, (M, T)) / 8.0).astype(np.float32)
    if M >= 2:
        alpha[0, 0], alpha[1, 0] = 0.0, 1.0
    level = rng.integers(0, 4, n).astype(np.uint8)
    r = oracle.update(fields, level, alpha, per_cell=True, P=1, min_importance=0.25, width=W)
    b = brute_update(fields.tolist(), level.tolist(), alpha.tolist(), W, P=1, min_importance=Fraction(1, 4))
    for _ in range(10):
        p0 = int(rng.integers(0, W))
        p1 = int(rng.integers(p0, W))
        sel = [c for c in range(n) if b["b1"][c] <= p1 and b["b2"][c] >= p0]
        got = oracle.brush(r["b1"], r["b2"], p0, p1)
        if not sel:
            assert got is None
        else:
            assert got == (sel[0], sel[-1]) and len(sel) == sel[-1] - sel[0] + 1


def test_brush_arguments():
    b1 = np.array([0, 0, 1, 2], np.uint32)
    b2 = np.array([0, 1, 2, 2], np.uint32)
    assert oracle.brush(b1, b2, 1, 1) == (1, 2)
    assert oracle.brush(b1, b2, 0, 2) == (0, 3)
    assert oracle.brush(b1, b2, 3, 5) is None
    with pytest.raises(oracle.OracleError):
        oracle.brush(b1, b2, 2, 1)


def test_select_keys_against_searchsorted():
    rng = np.random.default_rng(7)
    keys = np.sort(rng.choice(1 << 40, 5000, replace=False)).astype(np.uint64)
    ranges = [(int(keys[10]), int(keys[99])), (int(keys[4000]) - 1, int(keys[4000]) + 1), (5, 4)]
    mask = oracle.select_keys(keys, ranges)
    ref = np.zeros(keys.size, np.uint8)
    for lo, hi in ranges:
        a, b = np.searchsorted(keys, np.uint64(lo), "left"), np.searchsorted(keys, np.uint64(hi), "right")
        ref[a:b] = 1
    assert np.array_equal(mask, ref) and mask.sum() == 91
