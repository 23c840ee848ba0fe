"""CUDA path vs the CPU oracle, element by element (GPU).

Keys, permutation, fixed-point widths, Q, F, counts and min/max are compared
bit for bit; sums and means to 1e-5 relative; y exactly away from TF bucket
boundaries (see tests/_cmp.py).  Sizes span several scan tiles (16384 cells)
and ragged tails; the edge cases are N = 0/1, N around tile and chunk sizes,
W = 1, W > N, one field, eight fields, zero widths and the all-zero fallback.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from tests._cmp import assert_bins_match

pytestmark = pytest.mark.gpu

dvl = pytest.importorskip("paper_2306_11612_b300")


@pytest.fixture(scope="module")
def small():
    return synth.make("small")


def run_gpu(amr_or_parts, alpha, sfc, dom=None, **kw):
    lower, level, fields = amr_or_parts
    ctx = dvl.DVL(0)
    ctx.load_amr(lower, level, fields)
    ctx.build_order(sfc)
    for m in range(fields.shape[0]):
        lo, hi = (math.nan, math.nan) if dom is None else (dom[0][m], dom[1][m])
        ctx.set_tf(m, alpha[m], lo, hi)
    ctx.update(**kw)
    out = [ctx.read_bins(m) for m in range(fields.shape[0])]
    return ctx, out


def check_update(lower, level, fields, alpha, sfc=oracle.SFC_MORTON, dom=None, check_order=True, **kw):
    keys, perm, lev_s, fl_s = oracle.sorted_inputs(lower, level, fields, sfc)
    o = oracle.update(fl_s, lev_s, alpha, None if dom is None else dom[0], None if dom is None else dom[1],
                      per_cell=True, **kw)
    ctx, g = run_gpu((lower, level, fields), alpha, sfc, dom, **kw)
    try:
        st = ctx.get_stats()
        for k in ("Q", "F", "i", "j", "linear", "pow_exact"):
            assert st[k] == o["stats"][k], (k, st[k], o["stats"][k])
        for k in ("vmax", "inv_vmax", "f_upper"):
            assert np.float32(st[k]) == np.float32(o["stats"][k]), k
        if check_order:
            gk, gp = ctx.read_order()
            assert np.array_equal(gk, keys) and np.array_equal(gp, perm)
        q = ctx.read_widths()
        assert np.array_equal(q, o["q"]), "fixed-point widths differ"
        T = alpha.shape[1]
        for m in range(fields.shape[0]):
            assert_bins_match(g[m], o, m, T, alpha[m])
    finally:
        ctx.close()
    return o


@pytest.mark.parametrize("P,mi,W", [(1.0, 0.025, 1024), (0.0, 0.025, 1024), (2.0, 0.025, 4096),
                                    (0.5, 0.0, 333), (5.0, 0.25, 1024), (1.5, 0.1, 1), (1.0, 0.025, 65536)])
def test_small_config_morton(small, P, mi, W):
    alpha = synth.random_tfs(11)
    check_update(small.lower, small.level, small.fields, alpha, oracle.SFC_MORTON, P=P, min_importance=mi, width=W)


def test_small_config_hilbert_and_modes(small):
    alpha = synth.random_tfs(12)
    check_update(small.lower, small.level, small.fields, alpha, oracle.SFC_HILBERT, P=1.0, width=2048,
                 min_imp_mode=1)
    check_update(small.lower, small.level, small.fields, alpha, oracle.SFC_HILBERT, P=2.0, width=1024,
                 vmax_mode=1, width_mode=1)


def _random_amr(seed, n, M):
    rng = np.random.default_rng(seed)
    lev = rng.integers(0, 6, n).astype(np.uint8)
    g = 1 << 10
    lo = rng.integers(0, g, (3, n)) >> lev << lev
    lo = np.minimum(lo, g - (1 << lev.astype(np.int64))).astype(np.int32)
    fields = rng.lognormal(0, 1.5, (M, n)).astype(np.float32)
    return np.ascontiguousarray(lo), lev, fields


@pytest.mark.parametrize("n", [1, 3, 127, 128, 129, 1023, 1024, 1025, 2047, 2048, 2049, 4095, 4096, 4097, 8193, 12288, 20479,
                               16383, 16384, 16385, 20000, 70001])
def test_ragged_sizes(n):
    lo, lev, fields = _random_amr(n, n, 4)
    alpha = synth.random_tfs(n % 97)
    # overlapping random cells may share centroids: ties keep input order
    check_update(lo, lev, fields, alpha, oracle.SFC_HILBERT, P=1.0, width=512)


def test_entry_stream_equals_field_stream(small):
    """With tables of at most 256 entries the width pass streams each cell's
    kept TF entries instead of its field values; the entries follow the TF
    domain, the table size and the data.  Over a sequence of edits on one
    context (alpha only, a new domain, a smaller table, a table of more than
    256 entries, new field values, back to 256 entries) every result equals
    that of a context that streams the field values, bit for bit, widths and
    alpha means included."""
    rng = np.random.default_rng(31)
    lower, level, fields = small.lower, small.level, small.fields
    ctxs = []
    for use in (1, 0):
        c = dvl.DVL(0)
        c.set_option(dvl.OPT_ENTRIES, use)
        c.load_amr(lower, level, fields)
        c.build_order(oracle.SFC_HILBERT)
        ctxs.append(c)
    lo_d = np.min(fields, axis=1)
    hi_d = np.max(fields, axis=1)
    f2 = (fields * rng.uniform(0.5, 1.5, fields.shape)).astype(np.float32)
    steps = [("alpha", synth.random_tfs(40), None), ("alpha", synth.random_tfs(41), None),
             ("domain", synth.random_tfs(41), (lo_d + 0.1 * (hi_d - lo_d), lo_d + 0.7 * (hi_d - lo_d))),
             ("T64", synth.random_tfs(42, n_entries=64), None), ("T512", synth.random_tfs(43, n_entries=512), None),
             ("fields", synth.random_tfs(44), None), ("T256", synth.random_tfs(45), None)]
    try:
        for name, alpha, dom in steps:
            outs = []
            for c in ctxs:
                if name == "fields":
                    c.set_fields(f2)
                for m in range(fields.shape[0]):
                    lo, hi = (math.nan, math.nan) if dom is None else (float(dom[0][m]), float(dom[1][m]))
                    c.set_tf(m, alpha[m], lo, hi)
                c.update(width=1536, want_alpha=1)
                outs.append((c.read_widths(), [c.read_bins(m) for m in range(fields.shape[0])], c.read_alpha_means()))
            (qa, ba, aa), (qb, bb, ab) = outs
            assert np.array_equal(qa, qb), name
            for x, y in zip(ba, bb):
                for k in x:
                    assert np.array_equal(np.asarray(x[k]).view(np.uint8), np.asarray(y[k]).view(np.uint8)), (name, k)
            assert np.array_equal(np.asarray(aa).view(np.uint8), np.asarray(ab).view(np.uint8)), name
    finally:
        for c in ctxs:
            c.close()


def test_fixed_point_sums_across_magnitudes():
    """The value tables keep the exact sums of floor(t 2^95) in five 23-bit
    limbs and skip the lower ones for stretches of cells whose t is 0 or at
    least 2^-23 (two limbs) or 2^-46 (three).  With the TF domain [0, 1], t
    equals the field value, so spatially smooth fields put whole runs of
    pixels in each regime: t from 1 down to 2^-130 (subnormals, and values
    whose bits lie only in the lowest limbs), t in [2^-46, 2^-23), exact
    zeros next to 2^-70, and a random mix.  Sums must match the oracle to
    1e-5 relative in every pixel, the tiniest included."""
    n = 300_000
    lower, level, _ = _random_amr(77, n, 1)
    rng = np.random.default_rng(78)
    x, y, z = (lower.astype(np.float64) + 0.5) / 1024.0
    f = np.empty((4, n), np.float32)
    f[0] = np.exp2(-130.0 * x).astype(np.float32)
    f[1] = np.where(x < 0.5, 0.75, np.exp2(-40.0) * (1.0 + y)).astype(np.float32)
    f[2] = np.where(z < 0.5, 0.0, np.exp2(-70.0) * (1.0 + x)).astype(np.float32)
    f[3] = (rng.random(n) * np.exp2(-60.0 * rng.random(n))).astype(np.float32)
    dom = (np.zeros(4, np.float32), np.ones(4, np.float32))
    alpha = synth.random_tfs(79)
    for W in (1024, 8192):
        check_update(lower, level, f, alpha, oracle.SFC_HILBERT, dom=dom, P=1.0, width=W)


@pytest.mark.parametrize("M", [1, 2, 3, 5, 8])
def test_field_counts(M):
    lo, lev, fields = _random_amr(100 + M, 30000, M)
    alpha = synth.random_tfs(M, n_fields=M)
    check_update(lo, lev, fields, alpha, oracle.SFC_MORTON, P=1.0, width=777)


def test_wide_plot_and_zero_widths():
    n = 3000
    lo, lev, f1 = _random_amr(7, n, 1)
    fields = np.repeat(f1, 4, axis=0)
    fields[1, ::7] *= 3.0
    alpha = np.repeat(synth.random_tfs(5, n_fields=1), 4, axis=0)
    alpha[1, 255] = 1.0 - alpha[0, 255]
    dom = ([0.0] * 4, [float(fields.max())] * 4)
    o = check_update(lo, lev, fields, alpha, oracle.SFC_MORTON, dom=dom, P=8.0, min_importance=1e-4, width=20000)
    assert np.any(o["q"] == 0)


def test_all_zero_widths_linear_fallback():
    n = 9000
    lo, lev, _ = _random_amr(8, n, 2)
    fields = np.ones((2, n), np.float32)
    alpha = np.zeros((2, 16), np.float32)
    o = check_update(lo, lev, fields, alpha, oracle.SFC_MORTON, P=1.0, min_importance=0.0, width=100)
    assert o["stats"]["linear"] == 1


def test_tf_sizes_and_user_domain(small):
    rng = np.random.default_rng(3)
    for T in (2, 16, 1000, 4096):
        alpha = rng.uniform(0, 1, (4, T)).astype(np.float32)
        lo = [float(np.quantile(small.fields[m], 0.1)) for m in range(4)]
        hi = [float(np.quantile(small.fields[m], 0.9)) for m in range(4)]
        check_update(small.lower, small.level, small.fields, alpha, oracle.SFC_MORTON, dom=(lo, hi),
                     check_order=False, P=1.0, width=1024)


def test_powf_mode_tolerance(small):
    """P with 2P not an integer: powf on both sides, widths agree to float32
    rounding, so the assignment may move by at most one pixel at a boundary."""
    alpha = synth.random_tfs(13)
    keys, perm, lev_s, fl_s = oracle.sorted_inputs(small.lower, small.level, small.fields, oracle.SFC_MORTON)
    o = oracle.update(fl_s, lev_s, alpha, per_cell=True, P=0.7, width=1024)
    ctx, g = run_gpu((small.lower, small.level, small.fields), alpha, oracle.SFC_MORTON, P=0.7, width=1024)
    try:
        st = ctx.get_stats()
        assert st["Q"] == o["stats"]["Q"] and st["pow_exact"] == 0
        q = ctx.read_widths().astype(np.float64)
        rel = np.abs(q - o["q"]) / np.maximum(o["q"], 1)
        assert np.max(rel) <= 4 * 2.0 ** -23
        assert np.abs(int(st["F"]) - int(o["stats"]["F"])) <= 4 * 2.0 ** -23 * o["stats"]["F"]
        c = g[0]["count"].astype(np.int64)
        assert np.abs(c - o["count"].astype(np.int64)).sum() <= 8
    finally:
        ctx.close()


def test_set_fields_keeps_order(small):
    alpha = synth.random_tfs(21)
    ctx = dvl.DVL(0)
    try:
        ctx.load_amr(small.lower, small.level, small.fields)
        ctx.build_order(oracle.SFC_HILBERT)
        ctx.set_tfs(alpha)
        newf = np.ascontiguousarray(small.fields[::-1] * np.float32(1.5))
        ctx.set_fields(newf)
        ctx.update(P=1.0, width=1024)
        _, perm, lev_s, fl_s = oracle.sorted_inputs(small.lower, small.level, newf, oracle.SFC_HILBERT)
        o = oracle.update(fl_s, lev_s, alpha, per_cell=True, P=1.0, width=1024)
        assert ctx.get_stats()["F"] == o["stats"]["F"]
        for m in range(4):
            assert_bins_match(ctx.read_bins(m), o, m, 256, alpha[m])
    finally:
        ctx.close()


def test_device_inputs_and_outputs(small):
    torch = pytest.importorskip("torch")
    alpha = synth.random_tfs(31)
    dev = torch.device("cuda:0")
    lower = torch.from_numpy(small.lower).to(dev)
    level = torch.from_numpy(small.level).to(dev)
    fields = torch.from_numpy(small.fields).to(dev)
    stream = torch.cuda.current_stream()
    ctx = dvl.DVL(0, stream)
    try:
        ctx.load_amr(lower, level, fields)
        ctx.build_order(oracle.SFC_MORTON)
        ctx.set_tfs(alpha)
        ctx.update(P=1.0, width=1024)
        out = {k: torch.empty(1024, dtype=dt, device=dev) for k, dt in
               [("mean", torch.float32), ("min", torch.float32), ("max", torch.float32),
                ("y", torch.float32), ("sum", torch.float64), ("count", torch.int32)]}
        ctx.read_bins(2, out)
        h = ctx.read_bins(2)
        for k in out:
            assert np.array_equal(out[k].cpu().numpy().view(h[k].dtype), h[k])
    finally:
        ctx.close()


def test_set_tfs_equals_per_field_tables(small):
    """dvl_set_tfs: the same update as one dvl_set_tf per field (bit for bit),
    with and without user domains; a refused call leaves the tables as they
    were."""
    alpha = synth.random_tfs(41)
    M = small.fields.shape[0]
    lo = [float(np.percentile(small.fields[m], 10)) for m in range(M)]
    hi = [float(np.percentile(small.fields[m], 90)) for m in range(M)]
    lo[1], hi[1] = math.nan, math.nan                  # field 1 keeps its data range
    ctx = dvl.DVL(0)
    try:
        ctx.load_amr(small.lower, small.level, small.fields)
        ctx.build_order(oracle.SFC_HILBERT)
        for dom in (None, (lo, hi)):
            for m in range(M):
                ctx.set_tf(m, alpha[m], math.nan if dom is None else lo[m], math.nan if dom is None else hi[m])
            ctx.update(P=1.0, width=777)
            one = ctx.read_bins_all()
            if dom is None:
                ctx.set_tfs(alpha)
            else:
                ctx.set_tfs(alpha, lo, hi)
            ctx.update(P=1.0, width=777)
            allb = ctx.read_bins_all()
            for k in one:
                assert np.array_equal(one[k], allb[k]), (dom is None, k)
        bad = alpha.copy()
        bad[3, 7] = 1.5
        with pytest.raises(dvl.DVLError) as e:
            ctx.set_tfs(bad)
        assert e.value.status == dvl.ERR_ARG
        with pytest.raises(dvl.DVLError) as e:
            ctx.set_tfs(alpha[:2])
        assert e.value.status == dvl.ERR_ARG
        ctx.update(P=1.0, width=777)                   # the last accepted tables
        again = ctx.read_bins_all()
        for k in again:
            assert np.array_equal(again[k], allb[k]), k
    finally:
        ctx.close()


def test_read_bins_all_equals_per_field_reads(small):
    """dvl_read_bins_all: every field's row, bit for bit what dvl_read_bins
    gives, into host and device buffers; the oracle agrees; refused before
    the first update and for short buffers."""
    torch = pytest.importorskip("torch")
    alpha = synth.random_tfs(37)
    W, M = 1000, small.fields.shape[0]
    keys, perm, lev_s, fl_s = oracle.sorted_inputs(small.lower, small.level, small.fields, oracle.SFC_HILBERT)
    o = oracle.update(fl_s, lev_s, alpha, per_cell=True, P=1.0, min_importance=0.025, width=W)
    ctx = dvl.DVL(0)
    try:
        ctx.load_amr(small.lower, small.level, small.fields)
        ctx.build_order(oracle.SFC_HILBERT)
        with pytest.raises(dvl.DVLError) as e:
            ctx.read_bins_all()
        assert e.value.status == dvl.ERR_STATE
        ctx.set_tfs(alpha)
        ctx.update(P=1.0, min_importance=0.025, width=W)
        allb = ctx.read_bins_all()
        dev = torch.device("cuda:0")
        outd = {k: torch.empty(W if k == "count" else M * W, dtype=dt, device=dev) for k, dt in
                [("mean", torch.float32), ("min", torch.float32), ("max", torch.float32),
                 ("y", torch.float32), ("sum", torch.float64), ("count", torch.int32)]}
        ctx.read_bins_all(outd)
        for m in range(M):
            one = ctx.read_bins(m)
            row = {k: (allb[k] if k == "count" else allb[k][m]) for k in one}
            for k in one:
                assert np.array_equal(row[k], one[k]), (m, k)
                d = outd[k].cpu().numpy()
                d = d if k == "count" else d.reshape(M, W)[m]
                assert np.array_equal(d.view(one[k].dtype), one[k]), (m, k, "device")
            assert_bins_match(row, o, m, alpha.shape[1], alpha[m])
        with pytest.raises(ValueError):
            ctx.read_bins_all({"mean": np.empty(M * W - 1, np.float32)})
    finally:
        ctx.close()


def test_timeout_is_reported_and_context_survives(small):
    """The first scan tile withholds its sum: the waits of its successors run
    out (bounded), the update reports DVL_ERR_TIMEOUT, and the next update on
    the same context is correct."""
    lo, lev, fields = _random_amr(5, 40000, 4)
    alpha = synth.random_tfs(41)
    ctx = dvl.DVL(0)
    try:
        ctx.load_amr(lo, lev, fields)
        ctx.build_order(oracle.SFC_MORTON)
        ctx.set_tfs(alpha)
        ctx.set_option(dvl.OPT_SPIN_LIMIT, 2000)
        ctx.set_option(dvl.OPT_FAULT_NO_PUBLISH, 1)
        ctx.update(P=1.0, width=256)
        with pytest.raises(dvl.DVLError) as e:
            ctx.read_bins(0)
        assert e.value.status == dvl.ERR_TIMEOUT
        ctx.set_option(dvl.OPT_SPIN_LIMIT, 1 << 22)
        ctx.update(P=1.0, width=256)
        _, _, lev_s, fl_s = oracle.sorted_inputs(lo, lev, fields, oracle.SFC_MORTON)
        o = oracle.update(fl_s, lev_s, alpha, P=1.0, width=256)
        assert_bins_match(ctx.read_bins(0), o, 0, 256, alpha[0])
    finally:
        ctx.close()


def test_errors_and_state_machine(small):
    ctx = dvl.DVL(0)
    try:
        with pytest.raises(dvl.DVLError) as e:
            ctx.update()
        assert e.value.status == dvl.ERR_STATE
        with pytest.raises(dvl.DVLError) as e:
            ctx.build_order(0)
        assert e.value.status == dvl.ERR_STATE
        bad = small.lower.copy()
        bad[0, 5] = -1
        with pytest.raises(dvl.DVLError) as e:
            ctx.load_amr(bad, small.level, small.fields)
        assert e.value.status == dvl.ERR_RANGE
        badf = small.fields.copy()
        badf[1, 7] = np.nan
        with pytest.raises(dvl.DVLError) as e:
            ctx.load_amr(small.lower, small.level, badf)
        assert e.value.status == dvl.ERR_RANGE
        ctx.load_amr(small.lower, small.level, small.fields)
        with pytest.raises(dvl.DVLError) as e:
            ctx.set_tf(0, np.full(256, 1.5, np.float32))
        assert e.value.status == dvl.ERR_ARG
        with pytest.raises(dvl.DVLError) as e:
            ctx.set_tf(9, np.zeros(256, np.float32))
        assert e.value.status == dvl.ERR_ARG
        ctx.build_order(0)
        ctx.set_tf(0, np.zeros(256, np.float32))
        with pytest.raises(dvl.DVLError) as e:
            ctx.update()                         # fields 1..3 have no TF
        assert e.value.status == dvl.ERR_STATE
        ctx.set_tfs(synth.random_tfs(1))
        with pytest.raises(dvl.DVLError) as e:
            ctx.update(width=0)
        assert e.value.status == dvl.ERR_ARG
        with pytest.raises(dvl.DVLError) as e:
            ctx.update(P=-1.0)
        assert e.value.status == dvl.ERR_ARG
        ctx.update(width=100)
        ctx.sync()
    finally:
        ctx.close()


def test_empty_dataset():
    ctx = dvl.DVL(0)
    try:
        ctx.load_amr(np.zeros((3, 0), np.int32), np.zeros(0, np.uint8), np.zeros((2, 0), np.float32))
        ctx.build_order(1)
        ctx.set_tfs(synth.random_tfs(1, n_fields=2))
        ctx.update(width=64)
        b = ctx.read_bins(1)
        assert np.all(b["count"] == 0) and np.all(b["sum"] == 0) and np.all(b["y"] == 0)
        assert ctx.get_stats()["F"] == 0
    finally:
        ctx.close()
