"""Differentiable pattern on the GPU vs the CPU oracle (GPU).

The per-pixel mean alpha (forward) and its gradient with respect to the
alpha control points (adjoint kernel, assignment held fixed) are compared
with oracle.alpha_grad, whose gradient is pinned by float64 central
differences (tests/test_oracle_grad.py).  Tolerances: alpha means 1e-5
relative (float32 tables vs float64 in the oracle, sums as in the bins);
gradients component by component against the oracle's gradient for the very
float32 pixel weights the GPU was given (tests/_cmp.assert_grad_match: float64
accumulation on both sides, float32 output).
"""
import numpy as np
import pytest

import oracle
import synth
from tests._cmp import assert_grad_match

pytestmark = pytest.mark.gpu
dvl = pytest.importorskip("paper_2306_11612_b300")
torch = pytest.importorskip("torch")


def _case(seed, amr, K=64, W=257):
    rng = np.random.default_rng(seed)
    ctrl = (rng.integers(0, 1025, (4, K)) / 1024.0).astype(np.float32)
    target = rng.uniform(0, 1, (4, W))
    return ctrl, target


def _ctx(amr, sfc=dvl.SFC_HILBERT):
    ctx = dvl.DVL(0)
    ctx.load_amr(amr.lower, amr.level, amr.fields)
    ctx.build_order(sfc)
    return ctx


@pytest.mark.parametrize("kw", [dict(P=1.0), dict(P=2.0, min_importance=0.1), dict(P=0.0)])
def test_alpha_means_and_gradient_match_oracle(kw):
    amr = synth.make("small")
    W = 257
    ctrl, target = _case(1, amr, W=W)
    _, _, lev, fl = oracle.sorted_inputs(amr.lower, amr.level, amr.fields, oracle.SFC_HILBERT)
    ref = oracle.alpha_grad(fl, lev, ctrl, target, width=W, **kw)
    ctx = _ctx(amr)
    try:
        ctx.set_tf_ctrl(ctrl, 256)
        ctx.update(width=W, want_alpha=1, **kw)
        abar = ctx.read_alpha_means()
        assert np.allclose(abar, ref["abar"], rtol=1e-5, atol=1e-7)
        g = (2.0 * (ref["abar"] - target)).astype(np.float32)
        grad = ctx.backward(g)
        assert_grad_match(grad, fl, lev, ctrl, g, W, **kw)
        # the bins of the alpha-means update equal those of a plain update
        b = ctx.read_bins(2)
        ctx.update(width=W, **kw)
        b0 = ctx.read_bins(2)
        assert np.array_equal(b["count"], b0["count"]) and np.array_equal(b["min"], b0["min"])
    finally:
        ctx.close()


@pytest.mark.parametrize("W,M,n", [(2048, 4, 0), (16384, 4, 0), (65536, 4, 0), (5000, 3, 70001), (777, 1, 4097),
                                   (3000, 8, 33333)])
def test_gradient_wide_plots_and_field_counts(W, M, n):
    """Steps that cross pixel boundaries in every form: a few pixels per step
    (entry counts per pixel), many narrow pixels per step (per-cell adds) and
    cells wider than a pixel; 1, 3, 4 and 8 fields, ragged sizes."""
    if n == 0:
        amr = synth.make("small")
        lower, level, fields = amr.lower, amr.level, amr.fields
    else:
        rng = np.random.default_rng(n)
        level = rng.integers(0, 6, n).astype(np.uint8)
        g = 1 << 10
        lo = rng.integers(0, g, (3, n)) >> level << level
        lower = np.ascontiguousarray(np.minimum(lo, g - (1 << level.astype(np.int64))).astype(np.int32))
        fields = rng.lognormal(0, 1.5, (M, n)).astype(np.float32)
    rng = np.random.default_rng(W + M)
    K = 16
    ctrl = (rng.integers(0, 1025, (M, K)) / 1024.0).astype(np.float32)
    target = rng.uniform(0, 1, (M, W))
    _, _, lev, fl = oracle.sorted_inputs(lower, level, fields, oracle.SFC_HILBERT)
    ref = oracle.alpha_grad(fl, lev, ctrl, target, width=W, P=1.0)
    ctx = dvl.DVL(0)
    try:
        ctx.load_amr(lower, level, fields)
        ctx.build_order(dvl.SFC_HILBERT)
        ctx.set_tf_ctrl(ctrl, 256)
        ctx.update(width=W, want_alpha=1, P=1.0)
        assert np.allclose(ctx.read_alpha_means(), ref["abar"], rtol=1e-5, atol=1e-7)
        g = (2.0 * (ref["abar"] - target)).astype(np.float32)
        grad = ctx.backward(g)
        assert_grad_match(grad, fl, lev, ctrl, g, W, P=1.0)
    finally:
        ctx.close()


def test_autograd_function_matches_oracle():
    from paper_2306_11612_b300.diff import alpha_means
    amr = synth.make("small")
    W = 300
    ctrl, target = _case(2, amr, W=W)
    _, _, lev, fl = oracle.sorted_inputs(amr.lower, amr.level, amr.fields, oracle.SFC_HILBERT)
    ref = oracle.alpha_grad(fl, lev, ctrl, target, width=W, P=1.0)
    ctx = _ctx(amr)
    try:
        dev = torch.device("cuda:0")
        c = torch.tensor(ctrl, device=dev, requires_grad=True)
        t = torch.tensor(target, device=dev, dtype=torch.float32)
        abar = alpha_means(ctx, c, width=W, P=1.0)
        loss = ((abar.double() - t.double()) ** 2).sum()
        loss.backward()
        assert abs(loss.item() - ref["loss"]) <= 1e-5 * ref["loss"]
        # the weights autograd handed to the adjoint: dL/dabar in float64, cast
        # to abar's float32
        a64 = abar.detach().cpu().numpy().astype(np.float64)
        g = (2.0 * (a64 - t.cpu().numpy().astype(np.float64))).astype(np.float32)
        assert_grad_match(c.grad.cpu().numpy(), fl, lev, ctrl, g, W, P=1.0)
    finally:
        ctx.close()


def test_gradient_at_diff_config_scale():
    """20M-cell 4-level data set, 64 control points per field, W = 2048."""
    amr = synth.make("diff")
    W = 2048
    ctrl, target = _case(4, amr, W=W)
    _, _, lev, fl = oracle.sorted_inputs(amr.lower, amr.level, amr.fields, oracle.SFC_HILBERT)
    ref = oracle.alpha_grad(fl, lev, ctrl, target, width=W, P=1.0)
    ctx = _ctx(amr)
    try:
        ctx.set_tf_ctrl(ctrl, 256)
        ctx.update(width=W, want_alpha=1, P=1.0)
        assert np.allclose(ctx.read_alpha_means(), ref["abar"], rtol=1e-5, atol=1e-7)
        g = (2.0 * (ref["abar"] - target)).astype(np.float32)
        grad = ctx.backward(g)
        assert_grad_match(grad, fl, lev, ctrl, g, W, P=1.0)
    finally:
        ctx.close()


def test_gradient_after_a_batch_with_other_domains():
    """The adjoint reads the cells' kept TF entries only while they are the
    ones the last update read: a batched update with other TF domains in
    between rebuilds them, and the adjoint then normalises the field values
    itself; the gradient is the same as before the batch (float64 sums whose
    order may differ: 1e-6 relative)."""
    amr = synth.make("small")
    W = 300
    ctrl, target = _case(5, amr, W=W)
    ctx = _ctx(amr)
    try:
        ctx.set_tf_ctrl(ctrl, 256)
        ctx.update(width=W, want_alpha=1)
        g = (2.0 * (ctx.read_alpha_means() - target)).astype(np.float32)
        g1 = ctx.backward(g).copy()
        lo = np.min(amr.fields, axis=1)
        hi = np.max(amr.fields, axis=1)
        dom = list(lo + 0.3 * (hi - lo)) + list(lo + 0.8 * (hi - lo))
        ctx.update_batch(np.stack([synth.random_tfs(9)] * 2), [(0, 128), (1, 64)], domain=dom)
        g2 = ctx.backward(g)
        assert np.allclose(g2, g1, rtol=1e-6, atol=1e-9 * np.max(np.abs(g1)))
    finally:
        ctx.close()


def test_state_errors():
    amr = synth.make("small")
    ctx = _ctx(amr)
    try:
        ctx.set_tfs(synth.random_tfs(3))
        ctx.update(width=64)
        with pytest.raises(dvl.DVLError) as e:
            ctx.read_alpha_means()
        assert e.value.status == dvl.ERR_STATE
        ctx.update(width=64, want_alpha=1)
        with pytest.raises(dvl.DVLError) as e:
            ctx._K = 8
            ctx.backward(np.zeros((4, 64), np.float32))   # tables were not set from control points
        assert e.value.status == dvl.ERR_STATE
        with pytest.raises(dvl.DVLError) as e:
            ctx.set_tf_ctrl(np.full((4, 8), 1.5, np.float32))
        assert e.value.status == dvl.ERR_ARG
    finally:
        ctx.close()
