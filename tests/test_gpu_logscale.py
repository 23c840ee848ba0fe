"""Per-field log10 value scale: CUDA path vs the oracle (GPU).

The scaled values are compared bit for bit (both sides run the same sequence
of correctly rounded float32 operations), the data ranges exactly, and the
bins of an update on log-scaled fields with tests/_cmp.py's tolerances
against the oracle's update of the oracle-scaled fields.  Edge cases: values
<= 0 (they take the smallest positive value), subnormal minima, switching the
scale on and off after the order is built, new values through set_fields, a
field without a positive value, and the batched path on scaled fields.
"""
import numpy as np
import pytest

import oracle
import synth
from tests._cmp import assert_bins_match

pytestmark = pytest.mark.gpu

dvl = pytest.importorskip("paper_2306_11612_b300")


def _decade_fields(seed, n, M=4):
    """Positive fields spanning many decades (lognormal in log10 space), with
    zeros, negatives and a subnormal in some of them."""
    rng = np.random.default_rng(seed)
    e = rng.normal(0.0, 6.0, (M, n))                   # ~ +-18 decades
    f = np.power(10.0, np.clip(e, -37.0, 37.0)).astype(np.float32)
    if n > 10:
        f[0, rng.integers(0, n, n // 50 + 1)] = 0.0
        f[2, rng.integers(0, n, n // 50 + 1)] = -rng.uniform(0, 5, n // 50 + 1).astype(np.float32)
        f[3, rng.integers(0, n)] = np.float32(3e-42)   # subnormal minimum
    return f


def _amr(seed, n, M=4):
    rng = np.random.default_rng(seed)
    lev = rng.integers(0, 6, n).astype(np.uint8)
    g = 1 << 10
    lo = rng.integers(0, g, (3, n)) >> lev << lev
    lo = np.minimum(lo, g - (1 << lev.astype(np.int64))).astype(np.int32)
    return np.ascontiguousarray(lo), lev, _decade_fields(seed + 1, n, M)


def _ctx(lower, level, fields, sfc, mask, scale_before_order=True):
    ctx = dvl.DVL(0)
    ctx.load_amr(lower, level, fields)
    if scale_before_order:
        for m in range(fields.shape[0]):
            if mask >> m & 1:
                ctx.set_field_scale(m, dvl.SCALE_LOG10)
    ctx.build_order(sfc)
    if not scale_before_order:
        for m in range(fields.shape[0]):
            if mask >> m & 1:
                ctx.set_field_scale(m, dvl.SCALE_LOG10)
    return ctx


def _check_values(ctx, fl_s, mask):
    ref = oracle.log_fields(fl_s, mask)
    lo, hi = ctx.read_data_range()
    for m in range(fl_s.shape[0]):
        g = ctx.read_values(m)
        assert np.array_equal(g.view(np.uint32), ref[m].view(np.uint32)), f"field {m} values differ"
        assert lo[m] == ref[m].min() and hi[m] == ref[m].max(), f"field {m} range"
    return ref


@pytest.mark.parametrize("n,mask,sfc,before", [(1, 1, oracle.SFC_MORTON, True),
                                               (5000, 0b1101, oracle.SFC_HILBERT, True),
                                               (16385, 0b1111, oracle.SFC_MORTON, False),
                                               (70001, 0b0101, oracle.SFC_HILBERT, False)])
def test_scaled_values_bit_exact(n, mask, sfc, before):
    lower, level, fields = _amr(n, n)
    _, _, _, fl_s = oracle.sorted_inputs(lower, level, fields, sfc)
    ctx = _ctx(lower, level, fields, sfc, mask, before)
    try:
        _check_values(ctx, fl_s, mask)
    finally:
        ctx.close()


@pytest.mark.parametrize("n,mask,P,W", [(20000, 0b1111, 1.0, 1024), (33000, 0b0011, 2.0, 333),
                                        (4097, 0b1000, 0.0, 4096)])
def test_update_on_scaled_fields(n, mask, P, W):
    lower, level, fields = _amr(100 + n, n)
    sfc = oracle.SFC_HILBERT
    _, _, lev_s, fl_s = oracle.sorted_inputs(lower, level, fields, sfc)
    alpha = synth.random_tfs(n % 31)
    ref = oracle.log_fields(fl_s, mask)
    o = oracle.update(ref, lev_s, alpha, P=P, width=W, per_cell=True)
    ctx = _ctx(lower, level, fields, sfc, mask)
    try:
        for m in range(4):
            ctx.set_tf(m, alpha[m])
        ctx.update(P=P, width=W)
        st = ctx.get_stats()
        for k in ("Q", "F", "i", "j"):
            assert st[k] == o["stats"][k], k
        assert np.array_equal(ctx.read_widths(), o["q"])
        for m in range(4):
            assert_bins_match(ctx.read_bins(m), o, m, alpha.shape[1], alpha[m])
    finally:
        ctx.close()


def test_scale_toggle_and_user_domain():
    n = 12000
    lower, level, fields = _amr(9, n)
    sfc = oracle.SFC_MORTON
    _, _, lev_s, fl_s = oracle.sorted_inputs(lower, level, fields, sfc)
    ctx = _ctx(lower, level, fields, sfc, 0)
    try:
        _check_values(ctx, fl_s, 0)
        ctx.set_field_scale(1, dvl.SCALE_LOG10)
        ctx.set_field_scale(3, dvl.SCALE_LOG10)
        _check_values(ctx, fl_s, 0b1010)
        ctx.set_field_scale(1, dvl.SCALE_LINEAR)
        ref = _check_values(ctx, fl_s, 0b1000)
        # a user domain in log units
        alpha = synth.random_tfs(4)
        dom_lo = [float(ref[m].min()) for m in range(4)]
        dom_hi = [float(ref[m].max()) for m in range(4)]
        dom_lo[3], dom_hi[3] = -20.0, 10.0
        for m in range(4):
            ctx.set_tf(m, alpha[m], dom_lo[m], dom_hi[m])
        ctx.update(P=1.0, width=1500)
        o = oracle.update(ref, lev_s, alpha, dom_lo, dom_hi, P=1.0, width=1500)
        for m in range(4):
            assert_bins_match(ctx.read_bins(m), o, m, alpha.shape[1], alpha[m])
        # all back to linear: the raw values and ranges return
        ctx.set_field_scale(3, dvl.SCALE_LINEAR)
        _check_values(ctx, fl_s, 0)
    finally:
        ctx.close()


def test_set_fields_keeps_scale_and_refuses_nonpositive():
    n = 9000
    lower, level, fields = _amr(21, n)
    sfc = oracle.SFC_HILBERT
    _, perm, _, fl_s = oracle.sorted_inputs(lower, level, fields, sfc)
    ctx = _ctx(lower, level, fields, sfc, 0b0110)
    try:
        new = _decade_fields(77, n)
        ctx.set_fields(list(new))
        _check_values(ctx, np.ascontiguousarray(new[:, perm]), 0b0110)
        bad = new.copy()
        bad[2] = -np.abs(bad[2])               # field 2 loses every positive value
        with pytest.raises(dvl.DVLError) as ei:
            ctx.set_fields(list(bad))
        assert ei.value.status == dvl.ERR_RANGE
        _check_values(ctx, np.ascontiguousarray(bad[:, perm]), 0b0010)   # field 2 back to linear
        with pytest.raises(dvl.DVLError) as ei:
            ctx.set_field_scale(2, dvl.SCALE_LOG10)
        assert ei.value.status == dvl.ERR_RANGE
        with pytest.raises(dvl.DVLError) as ei:
            ctx.set_field_scale(4, dvl.SCALE_LOG10)
        assert ei.value.status == dvl.ERR_ARG
        with pytest.raises(dvl.DVLError) as ei:
            ctx.set_field_scale(0, 7)
        assert ei.value.status == dvl.ERR_ARG
    finally:
        ctx.close()


def test_batch_on_scaled_fields():
    n = 40000
    lower, level, fields = _amr(31, n)
    sfc = oracle.SFC_HILBERT
    ctx = _ctx(lower, level, fields, sfc, 0b1011)
    try:
        K = 5
        alphas = np.stack([synth.random_tfs(200 + k) for k in range(K)])
        pairs = [(k, w) for k in range(K) for w in (512, 2048)]
        ctx.update_batch(alphas, pairs, P=1.0)
        got = [[ctx.read_batch_bins(i, m) for m in range(4)] for i in range(len(pairs))]
        for i, (k, w) in enumerate(pairs):
            for m in range(4):
                ctx.set_tf(m, alphas[k][m])
            ctx.update(P=1.0, width=w)
            for m in range(4):
                ref = ctx.read_bins(m)
                g = got[i][m]
                for key in ("count", "min", "max", "y"):
                    assert np.array_equal(g[key], ref[key]), (i, m, key)
                assert np.array_equal(g["sum"], ref["sum"]), (i, m)
    finally:
        ctx.close()
