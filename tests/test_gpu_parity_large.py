"""Range-query bins against the oracle at benchmark-like sizes (GPU).

dvl_update's and dvl_update_batch's bins are compared with oracle.update,
every pixel of every field (tests/_cmp.py: counts, min and max bit for bit,
sums within 1e-5 relative plus count * 2^-95, y exact away from TF bucket
boundaries), on data sets large enough to take the query paths that small
inputs never reach.  The oracle sorts its own keys and runs its threaded form
(orc_update_mt, bit-identical to the sequential oracle; see
test_oracle_threads.py) so that each update takes seconds.

* The 20.0M-cell 4-level data set (the differentiable configuration):
  9,766 chunks, so the pixel-boundary search takes two 32-way rounds before
  its last probe; 156,250 steps, so the min/max sparse table has 18 levels;
  the chunk-prefix scan runs 5 blocks chained by look-back.  W = 2048 and
  65,536 (several pixels per step), P = 1 and P = 2.
* One batch on it: 8 TFs x the widths 512 ... 65,536 (widths that divide a
  wider one of the same TF read that one's pixel bounds), every pair against
  the oracle.
* A 74.2M-cell sub-box of the 413.6M-cell data set (Hilbert, W = 4096, the
  benchmark's settings): 36,213 chunks (three search rounds), 579,400 steps
  (20 sparse-table levels), 18 scan blocks.
"""
import os

import numpy as np
import pytest

import oracle
import synth
from tests._cmp import assert_bins_match

pytestmark = pytest.mark.gpu
dvl = pytest.importorskip("paper_2306_11612_b300")

THREADS = max(1, min(os.cpu_count() or 1, 64))


def _sorted(amr):
    """The oracle's own curve order: its keys, numpy's stable argsort (the
    library routine orc_order is pinned against), cells gathered."""
    k = oracle.keys(amr.lower, amr.level, oracle.SFC_HILBERT, threads=THREADS)
    perm = np.argsort(k, kind="stable").astype(np.uint32)
    return k[perm], perm, np.ascontiguousarray(amr.level[perm]), np.ascontiguousarray(amr.fields[:, perm])


def _loaded(amr):
    ctx = dvl.DVL(0)
    ctx.load_amr(amr.lower, amr.level, amr.fields)
    ctx.build_order(dvl.SFC_HILBERT)
    return ctx


def _check(ctx, o, alpha, expect_stats=True):
    st = ctx.get_stats()
    if expect_stats:
        for k in ("Q", "F", "i", "j", "linear"):
            assert st[k] == o["stats"][k], (k, st[k], o["stats"][k])
        assert np.float32(st["vmax"]) == np.float32(o["stats"]["vmax"])
    for m in range(alpha.shape[0]):
        assert_bins_match(ctx.read_bins(m), o, m, alpha.shape[1], alpha[m])


@pytest.fixture(scope="module")
def diff_set():
    amr = synth.make("diff")
    keys, perm, lev, fl = _sorted(amr)
    ctx = _loaded(amr)
    gk, gp = ctx.read_order()
    assert np.array_equal(gk, keys) and np.array_equal(gp, perm), "order differs from the oracle's"
    yield amr, lev, fl, ctx
    ctx.close()


@pytest.mark.parametrize("W,P,mi", [(2048, 1.0, 0.025), (65536, 1.0, 0.025), (2048, 2.0, 0.1), (65536, 0.5, 0.0)])
def test_bins_20M(diff_set, W, P, mi):
    amr, lev, fl, ctx = diff_set
    assert amr.n > 19_000_000
    alpha = synth.random_tfs(W + int(10 * P))
    ctx.set_tfs(alpha)
    ctx.update(P=P, min_importance=mi, width=W)
    o = oracle.update(fl, lev, alpha, P=P, min_importance=mi, width=W, threads=THREADS)
    _check(ctx, o, alpha)


def test_batch_20M(diff_set):
    amr, lev, fl, ctx = diff_set
    K = 8
    alphas = np.stack([synth.random_tfs(7000 + k) for k in range(K)])
    widths = [2048, 65536, 512, 4096, 1024, 16384, 2048, 777]
    pairs = [(k, widths[k]) for k in range(K)] + [(1, 2048), (3, 1024)]
    ctx.update_batch(alphas, pairs, P=1.0, min_importance=0.025)
    got = [[ctx.read_batch_bins(q, m) for m in range(4)] for q in range(len(pairs))]
    for q, (k, W) in enumerate(pairs):
        o = oracle.update(fl, lev, alphas[k], P=1.0, min_importance=0.025, width=W, threads=THREADS)
        for m in range(4):
            assert_bins_match(got[q][m], o, m, alphas.shape[2], alphas[k, m])


def test_bins_74M_sub_box_of_large():
    box = ((68, 43, 24), 43)                     # 43^3 base cells of the 128^3
    amr = synth.make("large", box=box)
    assert amr.n == 74_163_139
    keys, perm, lev, fl = _sorted(amr)
    ctx = _loaded(amr)
    try:
        gk, gp = ctx.read_order()
        assert np.array_equal(gk, keys) and np.array_equal(gp, perm), "order differs from the oracle's"
        del gk, gp, keys, perm
        alpha = synth.random_tfs(1000)
        ctx.set_tfs(alpha)
        ctx.update(P=1.0, min_importance=0.025, width=4096)
        o = oracle.update(fl, lev, alpha, P=1.0, min_importance=0.025, width=4096, threads=THREADS)
        _check(ctx, o, alpha)
    finally:
        ctx.close()
