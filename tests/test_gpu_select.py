"""Brushing and linking on the GPU vs the CPU oracle (GPU).

A pixel ROI must select exactly the oracle's run of cells (from its per-cell
bins), with the same curve keys and the same per-cell mask in input order;
key-range selection must equal the oracle's test of every cell's key.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
dvl = pytest.importorskip("paper_2306_11612_b300")
torch = pytest.importorskip("torch")


def _case(n, seed, M=4):
    rng = np.random.default_rng(seed)
    lev = rng.integers(0, 5, n).astype(np.uint8)
    g = 1 << 10
    lo = rng.integers(0, g, (3, n)) >> lev << lev
    lo = np.ascontiguousarray(np.minimum(lo, g - (1 << lev.astype(np.int64))).astype(np.int32))
    return lo, lev, rng.lognormal(0, 1.5, (M, n)).astype(np.float32), synth.random_tfs(seed, n_fields=M)


@pytest.mark.parametrize("n,W", [(70001, 1024), (5000, 4096), (1, 16), (20000, 1)])
def test_brush_matches_oracle(n, W):
    lo, lev, f, alpha = _case(n, n)
    keys, perm, lev_s, fl_s = oracle.sorted_inputs(lo, lev, f, oracle.SFC_HILBERT)
    o = oracle.update(fl_s, lev_s, alpha, None, None, per_cell=True, width=W)
    ctx = dvl.DVL(0)
    try:
        ctx.load_amr(lo, lev, f)
        ctx.build_order(dvl.SFC_HILBERT)
        ctx.set_tfs(alpha)
        ctx.update(width=W)
        rng = np.random.default_rng(1)
        rois = [(0, W - 1), (0, 0), (W - 1, W - 1)] + [tuple(sorted(rng.integers(0, W, 2))) for _ in range(6)]
        for p0, p1 in rois:
            p0, p1 = int(p0), int(p1)
            ref = oracle.brush(o["b1"], o["b2"], p0, p1)
            got = ctx.brush(p0, p1, mask=True)
            if ref is None:
                assert got["n_cells"] == 0 and not got["mask"].any()
                continue
            assert (got["first"], got["last"]) == ref and got["n_cells"] == ref[1] - ref[0] + 1
            assert (got["key_first"], got["key_last"]) == (int(keys[ref[0]]), int(keys[ref[1]]))
            m = np.zeros(n, np.uint8)
            m[perm[ref[0]:ref[1] + 1]] = 1
            assert np.array_equal(got["mask"], m)
        # key ranges of two ROIs select the same cells (the linked 3D view)
        a, b = ctx.brush(0, W // 3), ctx.brush(W // 2, W - 1)
        ranges = [(a["key_first"], a["key_last"]), (b["key_first"], b["key_last"]), (5, 3)]
        mask = ctx.select_keys(ranges)
        in_order = oracle.select_keys(keys, ranges)          # curve order
        ref = np.zeros(n, np.uint8)
        ref[perm] = in_order
        assert np.array_equal(mask, ref)
        dm = torch.empty(n, dtype=torch.uint8, device="cuda:0")
        ctx.select_keys(ranges, mask=dm)
        ctx.sync()
        assert np.array_equal(dm.cpu().numpy(), ref)
    finally:
        ctx.close()


def test_brush_states_and_errors():
    lo, lev, f, alpha = _case(3000, 3)
    ctx = dvl.DVL(0)
    try:
        ctx.load_amr(lo, lev, f)
        ctx.build_order(1)
        with pytest.raises(dvl.DVLError):
            ctx.brush(0, 1)                                   # no update yet
        ctx.set_tfs(alpha)
        ctx.update(width=64)
        with pytest.raises(dvl.DVLError):
            ctx.brush(5, 4)
        with pytest.raises(dvl.DVLError):
            ctx.brush(0, 64)
        assert ctx.brush(0, 63)["n_cells"] == 3000
        assert not ctx.select_keys([]).any()
        with pytest.raises(dvl.DVLError):
            ctx.select_keys([(0, 1)] * 1025)
    finally:
        ctx.close()
