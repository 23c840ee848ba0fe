"""Pin of the oracle's gradient of per-pixel mean alpha (CPU only).

With the cell-to-pixel assignment held fixed, the per-pixel mean alpha is
linear in the transfer-function control points, so the L2 loss is quadratic
and float64 central differences equal the derivative up to rounding.  The
tests pick parameters under which the assignment provably does not move when
the control points do: P = 0 (all widths 1), and P = 1 with minimum
importance 1 and the exact max V (every V/maxV <= 1, so f = 2^L).
"""
import numpy as np
import pytest

import oracle
import synth


def _setup(seed, n=3000, K=64, W=257):
    a = synth.bricks_amr(seed=seed, base_n=16, brick=4, n_refined=8)
    _, perm, lev, fl = oracle.sorted_inputs(a.lower, a.level, a.fields, oracle.SFC_HILBERT)
    rng = np.random.default_rng(seed)
    lev, fl = lev[:n], fl[:, :n]
    ctrl = (rng.integers(64, 1024 - 64, (4, K)) / 1024.0).astype(np.float32)   # multiples of 2^-10
    target = rng.uniform(0, 1, (4, W))
    return fl, lev, ctrl, target


@pytest.mark.parametrize("kw", [dict(P=0.0), dict(P=1.0, min_importance=1.0, vmax_mode=1)])
def test_gradient_matches_central_differences(kw):
    fl, lev, ctrl, target = _setup(3)
    W = target.shape[1]
    base = oracle.alpha_grad(fl, lev, ctrl, target, width=W, **kw)
    rng = np.random.default_rng(0)
    h = 2.0 ** -6                               # exact in float32 at these control points
    picks = rng.choice(ctrl.size, 32, replace=False)
    for flat in picks:
        m, k = divmod(int(flat), ctrl.shape[1])
        cp, cm = ctrl.copy(), ctrl.copy()
        cp[m, k] += h
        cm[m, k] -= h
        lp = oracle.alpha_grad(fl, lev, cp, target, width=W, **kw)["loss"]
        lm = oracle.alpha_grad(fl, lev, cm, target, width=W, **kw)["loss"]
        fd = (lp - lm) / (2 * h)
        g = base["grad"][m, k]
        assert abs(fd - g) <= 1e-9 * max(1.0, abs(g)), (m, k, fd, g)


def test_abar_is_mean_of_table_alpha():
    # with P = 0 and K = T the table equals the control points (x = e exactly)
    fl, lev, _, target = _setup(5, n=500, K=256, W=50)
    rng = np.random.default_rng(1)
    ctrl = rng.uniform(0, 1, (4, 256)).astype(np.float32)
    r = oracle.alpha_grad(fl, lev, ctrl, target, width=50, P=0.0)
    u = oracle.update(fl, lev, ctrl, per_cell=True, P=0.0, width=50)
    # direct restatement of the mean over covering cells, entries from t
    n = lev.shape[0]
    lo, hi = fl.min(1), fl.max(1)
    s = (np.float32(1) / (hi - lo)).astype(np.float32)
    t = np.clip(((fl - lo[:, None]).astype(np.float32) * s[:, None]).astype(np.float32), 0, 1)
    e = np.minimum(np.floor(t * np.float32(256)).astype(np.int64), 255)
    a = np.take_along_axis(ctrl.astype(np.float64), e, 1)
    expect = np.zeros((4, 50))
    for c in range(n):
        for p in range(u["b1"][c], u["b2"][c] + 1):
            expect[:, p] += a[:, c]
    expect /= u["count"][None, :]
    assert np.allclose(r["abar"], expect, rtol=1e-12, atol=0)


@pytest.mark.parametrize("kw", [dict(P=0.0), dict(P=1.0, min_importance=1.0, vmax_mode=1)])
def test_gradient_of_given_pixel_weights_matches_central_differences(kw):
    """With pixel weights g in place of dL/dabar, the gradient is that of the
    linear functional sum(g * abar); central differences of that functional
    (linear in the control points) equal it up to rounding."""
    fl, lev, ctrl, target = _setup(4)
    W = target.shape[1]
    rng = np.random.default_rng(2)
    g = rng.normal(size=(4, W)).astype(np.float32).astype(np.float64)
    base = oracle.alpha_grad(fl, lev, ctrl, target, width=W, g=g, **kw)
    h = 2.0 ** -6
    for flat in rng.choice(ctrl.size, 32, replace=False):
        m, k = divmod(int(flat), ctrl.shape[1])
        cp, cm = ctrl.copy(), ctrl.copy()
        cp[m, k] += h
        cm[m, k] -= h
        fp = float(np.sum(g * oracle.alpha_grad(fl, lev, cp, target, width=W, **kw)["abar"]))
        fm = float(np.sum(g * oracle.alpha_grad(fl, lev, cm, target, width=W, **kw)["abar"]))
        fd = (fp - fm) / (2 * h)
        assert abs(fd - base["grad"][m, k]) <= 1e-9 * max(1.0, abs(fd)), (m, k, fd, base["grad"][m, k])
    # g = 2 (abar - target) gives the loss gradient
    lg = oracle.alpha_grad(fl, lev, ctrl, target, width=W, **kw)
    gg = oracle.alpha_grad(fl, lev, ctrl, target, width=W, g=2.0 * (lg["abar"] - target), **kw)
    assert np.array_equal(lg["grad"], gg["grad"])
