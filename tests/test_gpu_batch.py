"""Batched updates (many TFs x viewports in one call) on the GPU.

Each (TF, width) pair of a batch must give the same bins as a plain update
with that TF and width: bit for bit against the GPU's single-TF path (both
compute the same exact integer widths and fixed-point value sums), and
against the CPU oracle with the tolerances of tests/_cmp.py.  The batches
span several shared-memory groups of TFs, ragged group tails, several scan
tiles, repeated and mixed widths, W = 1, the empty data set, and the replay
of the captured graph.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from tests._cmp import assert_bins_match

pytestmark = pytest.mark.gpu

dvl = pytest.importorskip("paper_2306_11612_b300")
torch = pytest.importorskip("torch")


def _tfs(seed, K, M=4, T=256):
    return np.stack([synth.random_tfs(seed * 1000 + k, n_fields=M, n_entries=T) for k in range(K)])


def _ctx(lower, level, fields, sfc=oracle.SFC_HILBERT):
    ctx = dvl.DVL(0)
    ctx.load_amr(lower, level, fields)
    ctx.build_order(sfc)
    return ctx


def _same(a, b):
    for k in ("count", "sum", "min", "max", "mean", "y"):
        assert np.array_equal(a[k].view(np.uint8), b[k].view(np.uint8)), k


def _check_vs_single(ctx, alphas, pairs, dom=None, **kw):
    M = alphas.shape[1]
    ctx.update_batch(alphas, pairs, domain=dom, **kw)
    got = [[ctx.read_batch_bins(q, m) for m in range(M)] for q in range(len(pairs))]
    for q, (k, W) in enumerate(pairs):
        for m in range(M):
            lo, hi = (math.nan, math.nan) if dom is None else (dom[m], dom[M + m])
            ctx.set_tf(m, alphas[k, m], lo, hi)
        ctx.update(width=W, **kw)
        for m in range(M):
            _same(got[q][m], ctx.read_bins(m))
    return got


def test_batch_matches_oracle(small_amr=None):
    amr = synth.make("small")
    alphas = _tfs(3, 3)
    pairs = [(0, 1024), (1, 333), (2, 4096), (0, 1)]
    _, _, lev, fl = oracle.sorted_inputs(amr.lower, amr.level, amr.fields, oracle.SFC_HILBERT)
    ctx = _ctx(amr.lower, amr.level, amr.fields)
    try:
        for P, mi in [(1.0, 0.025), (2.0, 0.1)]:
            ctx.update_batch(alphas, pairs, P=P, min_importance=mi)
            for q, (k, W) in enumerate(pairs):
                o = oracle.update(fl, lev, alphas[k], None, None, P=P, min_importance=mi, width=W)
                for m in range(4):
                    assert_bins_match(ctx.read_batch_bins(q, m), o, m, alphas.shape[2], alphas[k, m])
    finally:
        ctx.close()


@pytest.mark.parametrize("K", [1, 5, 8, 19, 70])
def test_batch_equals_single_updates(K):
    amr = synth.make("small")
    alphas = _tfs(K, K)
    rng = np.random.default_rng(K)
    pairs = [(k, int(rng.choice([64, 512, 1000, 2048]))) for k in range(K)]
    pairs += [(int(rng.integers(0, K)), 777), (0, 1)]
    ctx = _ctx(amr.lower, amr.level, amr.fields)
    try:
        _check_vs_single(ctx, alphas, pairs, P=1.0)
        _check_vs_single(ctx, alphas, pairs[: max(1, len(pairs) // 2)], P=1.5, min_importance=0.05,
                         min_imp_mode=1, width_mode=1)
    finally:
        ctx.close()


@pytest.mark.parametrize("n", [1, 129, 2049, 16385, 70001])
def test_batch_ragged_sizes(n):
    rng = np.random.default_rng(n)
    lev = rng.integers(0, 6, n).astype(np.uint8)
    g = 1 << 10
    lo = rng.integers(0, g, (3, n)) >> lev << lev
    lo = np.ascontiguousarray(np.minimum(lo, g - (1 << lev.astype(np.int64))).astype(np.int32))
    fields = rng.lognormal(0, 1.5, (3, n)).astype(np.float32)
    alphas = _tfs(n % 31, 11, M=3, T=200)
    pairs = [(k, 300 + 17 * k) for k in range(11)]
    dom = [0.1, 0.0, 0.5, 4.0, 2.0, 6.0]
    ctx = _ctx(lo, lev, fields)
    try:
        _check_vs_single(ctx, alphas, pairs, dom=dom, P=1.0)
        _check_vs_single(ctx, alphas, pairs, P=0.5)
    finally:
        ctx.close()


def test_batch_entries_equal_field_values():
    """The batched width pass reads the cells' kept TF entries (tables of at
    most 256 entries) or, with DVL_OPT_ENTRIES = 0, their field values; over
    a table size change (entries rebuilt alone), a domain change (rebuilt
    with the value tables) and a table of more than 256 entries, both give
    the same bins bit for bit."""
    amr = synth.make("small")
    ctxs = [_ctx(amr.lower, amr.level, amr.fields) for _ in range(2)]
    ctxs[1].set_option(dvl.OPT_ENTRIES, 0)
    lo = np.min(amr.fields, axis=1)
    hi = np.max(amr.fields, axis=1)
    dom = list(lo + 0.2 * (hi - lo)) + list(lo + 0.6 * (hi - lo))
    runs = [(_tfs(5, 9), None), (_tfs(6, 9, T=100), None), (_tfs(7, 9, T=100), dom), (_tfs(8, 5, T=400), dom),
            (_tfs(9, 9), None)]
    try:
        for alphas, d in runs:
            pairs = [(k, 257 + 31 * k) for k in range(alphas.shape[0])]
            out = []
            for c in ctxs:
                c.update_batch(alphas, pairs, domain=d)
                out.append([[c.read_batch_bins(q, m) for m in range(4)] for q in range(len(pairs))])
            for qa, qb in zip(*out):
                for x, y in zip(qa, qb):
                    _same(x, y)
    finally:
        for c in ctxs:
            c.close()


def test_batch_graph_replay_and_device_tfs():
    amr = synth.make("small")
    K = 24
    alphas = _tfs(7, K)
    pairs = [(k, 1024) for k in range(K)]
    ctx = _ctx(amr.lower, amr.level, amr.fields)
    try:
        ctx.update_batch(alphas, pairs)
        first = [ctx.read_batch_bins(q, 1) for q in range(K)]
        assert ctx.batch_config()["replayed"] is False
        # same shape, new TFs from device memory: the captured graph is replayed
        alphas2 = _tfs(8, K)
        t = torch.tensor(alphas2, device="cuda:0")
        ctx.update_batch(t, pairs)
        cfg = ctx.batch_config()
        assert cfg["replayed"] is True and cfg["group"] >= 1 and cfg["ctas_per_sm"] >= 1
        second = [ctx.read_batch_bins(q, 1) for q in range(K)]
        ref = _check_vs_single(ctx, alphas2, pairs)
        for q in range(K):
            _same(second[q], ref[q][1])
        # back to the first TFs: results equal the first call's
        ctx.update_batch(alphas, pairs)
        for q in range(K):
            _same(ctx.read_batch_bins(q, 1), first[q])
        # the bulk read holds every pair's bins in the documented layout
        allb = ctx.read_batch_all()
        M = alphas.shape[1]
        for q in (0, 7, K - 1):
            off = q * M * 1024 + 1 * 1024
            for k in ("mean", "min", "max", "y", "sum"):
                assert np.array_equal(allb[k][off:off + 1024].view(np.uint8), first[q][k].view(np.uint8)), k
            assert np.array_equal(allb["count"][q * 1024:(q + 1) * 1024], first[q]["count"])
    finally:
        ctx.close()


def test_batch_errors():
    amr = synth.make("small")
    ctx = dvl.DVL(0)
    try:
        alphas = _tfs(1, 2)
        with pytest.raises(dvl.DVLError):
            ctx.update_batch(alphas, [(0, 64)])            # no data set
        ctx.load_amr(amr.lower, amr.level, amr.fields)
        ctx.build_order(1)
        with pytest.raises(dvl.DVLError):
            ctx.update_batch(alphas, [(2, 64)])            # TF index out of range
        with pytest.raises(dvl.DVLError):
            ctx.update_batch(alphas, [(0, 0)])             # width 0
        bad = alphas.copy()
        bad[1, 2, 5] = 1.5
        with pytest.raises(dvl.DVLError):
            ctx.update_batch(bad, [(0, 64)])               # alpha outside [0, 1]
        with pytest.raises(dvl.DVLError):
            ctx.read_batch_bins(0, 0)                      # no batch has run
        ctx.update_batch(alphas, [(1, 64)])
        with pytest.raises(dvl.DVLError):
            ctx.read_batch_bins(1, 0)                      # pair out of range
        # a device table outside [0, 1] is flagged on the device
        t = torch.tensor(bad, device="cuda:0")
        ctx.update_batch(t, [(0, 64)])
        with pytest.raises(dvl.DVLError) as e:
            ctx.read_batch_bins(0, 0)
        assert e.value.status == dvl.ERR_RANGE
        ctx.update_batch(alphas, [(0, 64)])                # context still usable
        ctx.read_batch_bins(0, 0)
    finally:
        ctx.close()


def test_batch_empty_dataset():
    ctx = dvl.DVL(0)
    try:
        ctx.load_amr(np.zeros((3, 0), np.int32), np.zeros(0, np.uint8), np.zeros((2, 0), np.float32))
        ctx.build_order(1)
        ctx.update_batch(_tfs(2, 3, M=2), [(0, 64), (2, 5)])
        b = ctx.read_batch_bins(1, 1)
        assert np.all(b["count"] == 0) and np.all(b["sum"] == 0) and np.all(b["y"] == 0)
    finally:
        ctx.close()


def test_batch_at_benchmark_size():
    # the batched workload bench.py times: 50.6M cells, 64 TFs x W in {512,
    # 1024, 2048, 4096}; sampled pairs equal plain updates bit for bit (the
    # plain path is checked against the oracle at full size)
    amr = synth.make("batched")
    K = 64
    alphas = np.stack([synth.random_tfs(k * 100_003, n_entries=256) for k in range(K)])
    widths = (512, 1024, 2048, 4096)
    pairs = [(k, w) for k in range(K) for w in widths]
    ctx = _ctx(amr.lower, amr.level, amr.fields)
    try:
        ctx.update_batch(alphas, pairs)
        allb = ctx.read_batch_all()
        offs, o = [], 0
        for _, w in pairs:
            offs.append(o)
            o += 4 * w
        rng = np.random.default_rng(3)
        for q in sorted(rng.choice(len(pairs), 6, replace=False)):
            k, w = pairs[q]
            ctx.set_tfs(alphas[k])
            ctx.update(width=w)
            for m in range(4):
                b = ctx.read_bins(m)
                sl = slice(offs[q] + m * w, offs[q] + (m + 1) * w)
                for key in ("mean", "min", "max", "y", "sum"):
                    assert np.array_equal(allb[key][sl].view(np.uint8), b[key].view(np.uint8)), (q, m, key)
    finally:
        ctx.close()


def test_batch_shared_bounds_across_widths():
    # widths of one TF that divide a wider one read its pixel bounds (every
    # r-th boundary); chains, equal widths and non-divisible widths together
    amr = synth.make("small")
    alphas = _tfs(9, 2)
    widths = [7, 14, 28, 28, 3, 21, 1000, 2000, 1, 4096, 999]
    pairs = [(0, w) for w in widths] + [(1, w) for w in (512, 2048, 333)]
    ctx = _ctx(amr.lower, amr.level, amr.fields)
    try:
        _check_vs_single(ctx, alphas, pairs, P=1.0)
        _check_vs_single(ctx, alphas, pairs, P=2.0, min_importance=0.1)
    finally:
        ctx.close()
