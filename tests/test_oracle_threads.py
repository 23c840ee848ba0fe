"""The threaded oracle equals the sequential one bit for bit (CPU only).

orc_update_mt splits the per-cell work over host threads (contiguous ranges
of cells; each pixel filled by one thread with its cells in curve order) and
is used for the all-cores CPU baseline and for oracle runs at benchmark
sizes.  Every output -- widths, pixel ranges, F, Q, max V, counts, sums (as
float64 bits), min/max, means, y -- must equal orc_update's exactly, for any
thread count, including more threads than cells or pixels, zero widths, the
all-zero fallback, empty input and every mode.  orc_keys_mt must equal
orc_keys.
"""
import numpy as np
import pytest

import oracle
import synth

KEYS = ("sum", "min", "max", "mean", "mean64", "y", "count", "q", "b1", "b2")


def _same(a, b):
    for k in KEYS:
        assert a[k].dtype == b[k].dtype and np.array_equal(a[k].view(np.uint8), b[k].view(np.uint8)), k
    assert a["stats"] == b["stats"]


def _random(seed, n, M):
    rng = np.random.default_rng(seed)
    fields = rng.lognormal(0, 1.5, (M, n)).astype(np.float32)
    level = rng.integers(0, 6, n).astype(np.uint8)
    alpha = rng.uniform(0, 1, (M, 256)).astype(np.float32)
    return fields, level, alpha


@pytest.mark.parametrize("threads", [2, 3, 8, 61])
@pytest.mark.parametrize("kw", [dict(P=1.0, min_importance=0.025, width=1024),
                                dict(P=2.0, min_importance=0.1, width=4096, min_imp_mode=1),
                                dict(P=0.7, min_importance=0.0, width=333, vmax_mode=1),
                                dict(P=0.0, width=7), dict(P=1.0, width=1), dict(P=1.5, width=65536, width_mode=1)])
def test_mt_equals_sequential_small_config(threads, kw):
    a = synth.make("small")
    _, _, lev, fl = oracle.sorted_inputs(a.lower, a.level, a.fields, oracle.SFC_HILBERT)
    alpha = synth.random_tfs(21)
    _same(oracle.update(fl, lev, alpha, per_cell=True, **kw),
          oracle.update(fl, lev, alpha, per_cell=True, threads=threads, **kw))


@pytest.mark.parametrize("n,M,W", [(0, 2, 16), (1, 4, 5), (5, 3, 1000), (1000, 1, 64), (4097, 8, 100)])
def test_mt_edge_sizes(n, M, W):
    fields, level, alpha = _random(n + M, n, M)
    for threads in (2, 16):
        _same(oracle.update(fields, level, alpha, per_cell=True, width=W),
              oracle.update(fields, level, alpha, per_cell=True, width=W, threads=threads))


def test_mt_zero_widths_fallback_and_user_domain():
    fields, level, alpha = _random(3, 5000, 4)
    fields[1] = fields[0]
    alpha[1] = alpha[0]
    dom = ([0.0, 0.0, 1.0, 0.5], [2.0, 2.0, 3.0, 4.0])
    kw = dict(P=8.0, min_importance=1e-4, width=20000)
    _same(oracle.update(fields, level, alpha, dom[0], dom[1], per_cell=True, **kw),
          oracle.update(fields, level, alpha, dom[0], dom[1], per_cell=True, threads=5, **kw))
    same = np.repeat(fields[:1], 2, axis=0)
    a2 = np.repeat(alpha[:1], 2, axis=0)
    r = oracle.update(same, level, a2, per_cell=True, P=1.0, min_importance=0.0, width=300)
    assert r["stats"]["linear"] == 1
    _same(r, oracle.update(same, level, a2, per_cell=True, P=1.0, min_importance=0.0, width=300, threads=7))


def test_mt_signed_zero_extremes():
    # -0 and +0 compare equal: the first one met is the data minimum in both
    fields = np.array([[0.0, -0.0, 1.0, 2.0, -0.0, 0.5] * 50, [-0.0, 0.0, 3.0, 1.0, 0.0, 2.0] * 50], np.float32)
    level = np.zeros(fields.shape[1], np.uint8)
    alpha = synth.random_tfs(3, n_fields=2)
    for threads in (2, 3, 4, 50):
        _same(oracle.update(fields, level, alpha, per_cell=True, width=40),
              oracle.update(fields, level, alpha, per_cell=True, width=40, threads=threads))


@pytest.mark.parametrize("sfc", [oracle.SFC_MORTON, oracle.SFC_HILBERT])
def test_keys_mt_equals_keys(sfc):
    a = synth.make("small")
    k1 = oracle.keys(a.lower, a.level, sfc)
    for threads in (2, 7, 64):
        assert np.array_equal(oracle.keys(a.lower, a.level, sfc, threads=threads), k1)
