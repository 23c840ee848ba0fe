"""Line-plot rasterisation on the GPU vs the CPU oracle (GPU).

The kernel draws the bins of the last update; the oracle draws the same bin
values (read back from the GPU), so the images must match bit for bit.  Sizes
cover one column and one row, ragged row blocks, tall images, 1-8 fields, both
value kinds, every bar field, and device outputs.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
dvl = pytest.importorskip("paper_2306_11612_b300")
torch = pytest.importorskip("torch")


def _ctx(M=4, n=20000, seed=1):
    rng = np.random.default_rng(seed)
    lev = rng.integers(0, 4, n).astype(np.uint8)
    g = 1 << 9
    lo = rng.integers(0, g, (3, n)) >> lev << lev
    lo = np.ascontiguousarray(np.minimum(lo, g - (1 << lev.astype(np.int64))).astype(np.int32))
    fields = rng.lognormal(0, 1.0, (M, n)).astype(np.float32)
    ctx = dvl.DVL(0)
    ctx.load_amr(lo, lev, fields)
    ctx.build_order(dvl.SFC_HILBERT)
    ctx.set_tfs(synth.random_tfs(seed, n_fields=M))
    return ctx


def _values(ctx, M, kind):
    return np.stack([ctx.read_bins(m)["mean" if kind == dvl.PLOT_MEAN else "y"] for m in range(M)])


@pytest.mark.parametrize("M,W,H", [(4, 1024, 512), (4, 1, 1), (1, 7, 1), (2, 333, 33), (8, 4096, 100),
                                   (3, 20000, 2), (4, 257, 1000)])
def test_raster_matches_oracle(M, W, H):
    ctx = _ctx(M)
    try:
        ctx.update(width=W)
        for kind in (dvl.PLOT_MEAN, dvl.PLOT_Y):
            vals = _values(ctx, M, kind)
            for bar in sorted({0, M - 1}):
                lines, bars = ctx.rasterize(H, kind, bar)
                ol, ob = oracle.rasterize(vals, H, bar)
                assert np.array_equal(lines, ol), (kind, bar)
                assert np.array_equal(bars, ob), (kind, bar)
    finally:
        ctx.close()


def test_raster_device_outputs_and_errors():
    ctx = _ctx()
    try:
        with pytest.raises(dvl.DVLError):
            ctx.rasterize(64)                                # no update yet
        ctx.update(width=640)
        dl = torch.empty((300, 640), dtype=torch.uint8, device="cuda:0")
        db = torch.empty((300, 640), dtype=torch.uint8, device="cuda:0")
        ctx.rasterize(300, dvl.PLOT_Y, 2, lines=dl, bars=db)
        ctx.sync()
        ol, ob = oracle.rasterize(_values(ctx, 4, dvl.PLOT_Y), 300, 2)
        assert np.array_equal(dl.cpu().numpy(), ol) and np.array_equal(db.cpu().numpy(), ob)
        only = np.empty((300, 640), np.uint8)
        ctx.rasterize(300, dvl.PLOT_Y, 2, lines=only)        # one output only
        assert np.array_equal(only, ol)
        for bad in [dict(height=0), dict(height=65537), dict(height=8, value_kind=2), dict(height=8, bar_field=4)]:
            with pytest.raises(dvl.DVLError):
                ctx.rasterize(**bad)
    finally:
        ctx.close()
