"""Pins of the oracle's space-filling-curve keys and stable order (CPU only).

The oracle's key functions are checked against properties that define the
curves, never against a retyped copy of their bit formulas:

* Morton: the order of a cube of finest cells equals a recursive depth-first
  traversal of octants (x fastest), i.e. the textbook Z-order.
* Hilbert (Skilling 2004): on cubes of 2^k finest cells the order is a
  bijection that starts at the origin cell, takes unit face-adjacent steps
  and visits every aligned sub-cube contiguously.
* Both: a coarse cell's key lies within the key range of the finest cells it
  covers (the centroid of Sec. 2.2 keeps AMR cells in curve order).
* Order: equal to numpy's stable argsort (a library routine).
"""
import itertools

import numpy as np
import pytest

import oracle


def cube_cells(k, level=0, origin=(0, 0, 0)):
    w = 1 << level
    side = 1 << k
    idx = np.array(list(itertools.product(range(side), repeat=3)), np.int64)[:, ::-1]  # x fastest
    lower = (idx * w + np.array(origin)).T.astype(np.int32)
    return np.ascontiguousarray(lower), np.full(idx.shape[0], level, np.uint8)


def zorder(origin, size):
    if size == 1:
        yield tuple(origin)
        return
    h = size // 2
    for o in range(8):
        dx, dy, dz = o & 1, (o >> 1) & 1, (o >> 2) & 1
        yield from zorder((origin[0] + dx * h, origin[1] + dy * h, origin[2] + dz * h), h)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_morton_is_recursive_zorder(k):
    seq = np.array(list(zorder((0, 0, 0), 1 << k)), np.int32).T
    keys = oracle.keys(np.ascontiguousarray(seq), np.zeros(seq.shape[1], np.uint8), oracle.SFC_MORTON)
    assert np.all(np.diff(keys.astype(np.float64)) > 0)


def test_morton_single_bits():
    # a single set bit of one axis lands on the interleaved position
    for d in range(3):
        for b in range(0, 20, 3):
            lower = np.zeros((3, 1), np.int32)
            lower[d, 0] = 1 << b            # centroid coordinate 2*2^b + 1
            k = oracle.keys(lower, np.zeros(1, np.uint8), oracle.SFC_MORTON)[0]
            others = sum(1 << (3 * 0 + e) for e in range(3) if e != d)   # the "+1" bits
            assert int(k) == (1 << (3 * (b + 1) + d)) | (1 << d) | others


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_hilbert_bijective_adjacent_contiguous(k):
    lower, level = cube_cells(k)
    keys = oracle.keys(lower, level, oracle.SFC_HILBERT)
    assert len(np.unique(keys)) == keys.size
    order = np.argsort(keys, kind="stable")
    pts = lower[:, order].T.astype(np.int64)
    assert tuple(pts[0]) == (0, 0, 0)
    steps = np.abs(np.diff(pts, axis=0)).sum(1)
    assert np.all(steps == 1), "consecutive Hilbert cells must share a face"
    # every aligned sub-cube of edge 2^j is one contiguous run of the order
    for j in range(1, k):
        block = tuple((pts >> j).T)
        ids = np.ravel_multi_index(block, (1 << (k - j),) * 3)
        changes = np.count_nonzero(np.diff(ids))
        assert changes == (1 << (3 * (k - j))) - 1


@pytest.mark.parametrize("sfc", [oracle.SFC_MORTON, oracle.SFC_HILBERT])
def test_coarse_cell_key_within_children(sfc):
    rng = np.random.default_rng(5)
    for _ in range(40):
        L = int(rng.integers(1, 6))
        lo = (rng.integers(0, 1 << (12 - L), 3) << L).astype(np.int32)
        coarse = oracle.keys(lo.reshape(3, 1), np.array([L], np.uint8), sfc)[0]
        fl, flev = cube_cells(L, 0, tuple(int(x) for x in lo))
        fine = oracle.keys(fl, flev, sfc)
        assert fine.min() < coarse < fine.max()


@pytest.mark.parametrize("sfc", [oracle.SFC_MORTON, oracle.SFC_HILBERT])
def test_hilbert_morton_keys_fit_extent(sfc):
    # cells inside a 2^g logical grid have centroids < 2^(g+1): keys < 8^(g+1)
    rng = np.random.default_rng(1)
    g = 7
    lev = rng.integers(0, 3, 500).astype(np.uint8)
    lo = (rng.integers(0, 1 << g, (3, 500)) >> lev << lev).astype(np.int32)
    lo = np.minimum(lo, (1 << g) - (1 << lev.astype(np.int32))).astype(np.int32)
    k = oracle.keys(lo, lev, sfc)
    assert int(k.max()) < 8 ** (g + 1)


def test_keys_reject_out_of_range():
    with pytest.raises(oracle.OracleError):
        oracle.keys(np.array([[-1], [0], [0]], np.int32), np.zeros(1, np.uint8), 0)
    with pytest.raises(oracle.OracleError):
        oracle.keys(np.array([[(1 << 20) - 1], [0], [0]], np.int32), np.ones(1, np.uint8), 0)
    with pytest.raises(oracle.OracleError):
        oracle.keys(np.zeros((3, 1), np.int32), np.array([21], np.uint8), 0)


def test_order_matches_stable_argsort():
    rng = np.random.default_rng(3)
    for n in [0, 1, 2, 17, 1000, 4099]:
        k = rng.integers(0, 64, n).astype(np.uint64) << np.uint64(40)   # many ties
        assert np.array_equal(oracle.order(k), np.argsort(k, kind="stable").astype(np.uint32))


def test_small_config_order_is_permutation():
    import synth
    a = synth.make("small")
    k = oracle.keys(a.lower, a.level, oracle.SFC_MORTON)
    perm = oracle.order(k)
    assert np.array_equal(np.sort(perm), np.arange(a.n, dtype=np.uint32))
    ks = k[perm]
    assert np.all(ks[1:] > ks[:-1])          # non-overlapping cells: no ties
