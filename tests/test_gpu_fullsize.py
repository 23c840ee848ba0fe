"""Parity at the full benchmark size (GPU).

The 413,554,163-cell "large" data set in the configuration bench.py times
(Hilbert order, W = 4096, P = 1, minimum importance 0.025, the benchmark's
first TF).  The oracle cannot run the whole update in seconds, so:

* order: the permutation is one (every cell appears once), keys strictly
  increase, and 1M sampled keys equal the oracle's keys of their input cells;
* widths: 1M sampled cells' fixed-point widths equal the oracle's, computed one
  by one from the data set's global quantities (data range and deepest level,
  taken from the input arrays); Q and max V equal the oracle's; F equals the
  sum of all widths;
* bins: properties that hold at any size (no empty pixel when F > 0, counts
  cover every cell, min <= mean <= max within [0, 1], y is the TF at the mean's
  entry); an update that also computes alpha means gives the same bins bit
  for bit, and alpha means in [0, 1];
* and the whole update against the oracle: the oracle's key of every cell
  (threaded orc_keys), which the library's permutation must put in strictly
  increasing order -- with distinct keys that is the one stable order -- then
  the oracle's update of all 413.6M cells in that order (threaded
  orc_update_mt, bit-identical to the sequential oracle): Q, F, max V, and
  every pixel of every field (tests/_cmp.py).
"""
import os

import numpy as np
import pytest

import oracle
import synth
from tests._cmp import assert_bins_match

pytestmark = pytest.mark.gpu
dvl = pytest.importorskip("paper_2306_11612_b300")

W, P, MI, T = 4096, 1.0, 0.025, 256


@pytest.fixture(scope="module")
def full():
    amr = synth.make("large")
    tf = synth.random_tfs(1000)                  # bench.py's first TF set
    ctx = dvl.DVL(0)
    ctx.load_amr(amr.lower, amr.level, amr.fields)
    ctx.build_order(dvl.SFC_HILBERT)
    ctx.set_tfs(tf)
    ctx.update(P=P, min_importance=MI, width=W)
    keys, perm = ctx.read_order()
    yield amr, ctx, tf, keys, perm
    ctx.close()


def test_order_at_full_size(full):
    amr, ctx, tf, keys, perm = full
    n = amr.n
    assert keys.size == n == perm.size
    seen = np.zeros(n, bool)
    seen[perm] = True
    assert seen.all(), "perm is a permutation"
    assert np.all(keys[1:] > keys[:-1]), "keys strictly increase (non-overlapping cells)"
    rng = np.random.default_rng(11)
    k = np.sort(rng.choice(n, 1_000_000, replace=False))
    c = perm[k]
    ok = oracle.keys(np.ascontiguousarray(amr.lower[:, c]), np.ascontiguousarray(amr.level[c]), oracle.SFC_HILBERT)
    assert np.array_equal(ok, keys[k])


def test_widths_at_full_size(full):
    amr, ctx, tf, keys, perm = full
    q = ctx.read_widths()
    st = ctx.get_stats()
    assert st["F"] == int(q.sum(dtype=np.uint64)) and not st["linear"]
    rng = np.random.default_rng(12)
    k = rng.choice(amr.n, 1_000_000, replace=False)
    c = perm[k]
    qo, Q, vmax = oracle.widths(amr.n, amr.fields.min(1), amr.fields.max(1), int(amr.level.max()), tf,
                                np.ascontiguousarray(amr.fields[:, c]), np.ascontiguousarray(amr.level[c]),
                                P=P, min_importance=MI)
    assert Q == st["Q"] and np.float32(vmax) == np.float32(st["vmax"])
    assert np.array_equal(qo, q[k])


def test_bins_at_full_size(full):
    amr, ctx, tf, keys, perm = full
    ctx.update(P=P, min_importance=MI, width=W)
    rq = [ctx.read_bins(m) for m in range(4)]
    cnt = rq[0]["count"].astype(np.int64)
    assert np.all(cnt >= 1) and cnt.sum() >= amr.n
    for m in range(4):
        b = rq[m]
        assert np.all((b["min"] >= 0) & (b["max"] <= 1) & (b["min"] <= b["max"]))
        mean64 = b["sum"] / cnt
        assert np.all(mean64 >= b["min"] * (1 - 1e-6)) and np.all(mean64 <= b["max"] * (1 + 1e-6) + 1e-30)
        e = np.minimum(np.floor(b["mean"].astype(np.float32) * np.float32(T)).astype(np.int64), T - 1)
        assert np.array_equal(b["y"], tf[m][e])
    # with alpha means (pass A also sums the cells' alphas): the same bins
    ctx.update(P=P, min_importance=MI, width=W, want_alpha=1)
    pl = [ctx.read_bins(m) for m in range(4)]
    for m in range(4):
        for k in ("count", "sum", "min", "max", "mean", "y"):
            assert np.array_equal(pl[m][k].view(np.uint8), rq[m][k].view(np.uint8)), (m, k)
    am = ctx.read_alpha_means()
    assert am.shape == (4, W) and np.all((am >= 0) & (am <= 1))


def test_log_scale_at_full_size(full):
    """dens, pres and velmag on the log10 scale: 1M sampled scaled values bit
    for bit against the oracle's log10 of their input cells, the data range
    equal to the min/max of all scaled values, 1M sampled widths against the
    oracle given that range, and the bins' properties; then back to linear."""
    import torch
    amr, ctx, tf, keys, perm = full
    n = amr.n
    logm = (0, 2, 3)
    for m in logm:
        ctx.set_field_scale(m, dvl.SCALE_LOG10)
    try:
        rng = np.random.default_rng(14)
        k = np.sort(rng.choice(n, 1_000_000, replace=False))
        c = perm[k]
        kd = torch.from_numpy(k.astype(np.int64)).cuda()
        lo, hi = ctx.read_data_range()
        sample = np.empty((4, k.size), np.float32)
        buf = torch.empty(n, dtype=torch.float32, device="cuda")
        for m in range(4):
            ctx.read_values(m, out=buf)
            ctx.sync()
            assert lo[m] == buf.min().item() and hi[m] == buf.max().item(), m
            sample[m] = buf[kd].cpu().numpy()
            raw = np.ascontiguousarray(amr.fields[m, c])
            if m in logm:
                pos = amr.fields[m][amr.fields[m] > 0].min()
                ref = oracle.log10f(np.where(raw > 0, raw, pos).astype(np.float32))
            else:
                ref = raw
            assert np.array_equal(sample[m].view(np.uint32), ref.view(np.uint32)), m
        del buf
        ctx.update(P=P, min_importance=MI, width=W)
        q = ctx.read_widths()
        st = ctx.get_stats()
        qo, Q, vmax = oracle.widths(n, lo, hi, int(amr.level.max()), tf, sample,
                                    np.ascontiguousarray(amr.level[c]), P=P, min_importance=MI)
        assert Q == st["Q"] and np.float32(vmax) == np.float32(st["vmax"])
        assert np.array_equal(qo, q[k])
        cnt = ctx.read_bins(0)["count"].astype(np.int64)
        assert np.all(cnt >= 1) and cnt.sum() >= n
        for m in range(4):
            b = ctx.read_bins(m)
            assert np.all((b["min"] >= 0) & (b["max"] <= 1) & (b["min"] <= b["max"]))
            e = np.minimum(np.floor(b["mean"].astype(np.float32) * np.float32(T)).astype(np.int64), T - 1)
            assert np.array_equal(b["y"], tf[m][e])
    finally:
        for m in logm:
            ctx.set_field_scale(m, dvl.SCALE_LINEAR)


def test_update_matches_oracle_at_full_size(full):
    amr, ctx, tf, keys, perm = full
    threads = max(1, min(os.cpu_count() or 1, 64))
    ko = oracle.keys(amr.lower, amr.level, oracle.SFC_HILBERT, threads=threads)
    ko = ko[perm]
    assert np.array_equal(ko, keys), "library keys differ from the oracle's"
    assert np.all(ko[1:] > ko[:-1]), "the permutation does not sort the oracle's keys"
    del ko
    lev = np.ascontiguousarray(amr.level[perm])
    fl = np.empty((4, amr.n), np.float32)
    for m in range(4):
        np.take(amr.fields[m], perm, out=fl[m])
    o = oracle.update(fl, lev, tf, P=P, min_importance=MI, width=W, threads=threads)
    del fl, lev
    ctx.set_tfs(tf)
    ctx.update(P=P, min_importance=MI, width=W)
    st = ctx.get_stats()
    for k in ("Q", "F", "i", "j", "linear"):
        assert st[k] == o["stats"][k], (k, st[k], o["stats"][k])
    assert np.float32(st["vmax"]) == np.float32(o["stats"]["vmax"])
    for m in range(4):
        assert_bins_match(ctx.read_bins(m), o, m, T, tf[m])
