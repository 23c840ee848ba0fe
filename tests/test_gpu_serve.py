"""Serving loop (resident data sets, continuous batching) on the GPU.

Every served result must equal, bit for bit, the same request served alone
and a plain dvl_update with the same tables and width on the same data set;
one request is also checked against the CPU oracle.  Memory admission limits
batch sizes to the budget and fails requests that can never fit, without
stopping the server.
"""
import threading

import numpy as np
import pytest

import oracle
import synth
from tests._cmp import assert_bins_match

pytestmark = pytest.mark.gpu

dvl = pytest.importorskip("paper_2306_11612_b300")
from paper_2306_11612_b300.serve import DVLServer  # noqa: E402


def _random_amr(seed, n, M=4):
    rng = np.random.default_rng(seed)
    lev = rng.integers(0, 5, n).astype(np.uint8)
    g = 1 << 9
    lo = rng.integers(0, g, (3, n)) >> lev << lev
    lo = np.ascontiguousarray(np.minimum(lo, g - (1 << lev.astype(np.int64))).astype(np.int32))
    return lo, lev, rng.lognormal(0, 1.2, (M, n)).astype(np.float32)


def _datasets():
    a = synth.make("small")
    return [(a.lower, a.level, a.fields), _random_amr(1, 70001), _random_amr(2, 20000)]


def _same(a, b):
    for k in ("count", "sum", "min", "max", "mean", "y"):
        assert np.array_equal(np.asarray(a[k]).view(np.uint8), np.asarray(b[k]).view(np.uint8)), k


def _requests(n, seed=0):
    rng = np.random.default_rng(seed)
    return [(int(rng.integers(0, 3)), synth.random_tfs(seed * 1000 + i), int(rng.choice([512, 1024, 2048])))
            for i in range(n)]


def test_result_alone_equals_in_mix_and_plain():
    data = _datasets()
    reqs = _requests(48)
    R = 17
    with DVLServer(0, max_batch=16, max_inflight=4, max_width=2048) as srv:
        for lo, lev, f in data:
            srv.add_dataset(lo, lev, f)
        alone = srv.wait(srv.submit(*reqs[R]), timeout=120)
        srv.reset_stats()
        ids = [None] * len(reqs)

        def client(part):
            for i in part:
                ids[i] = srv.submit(*reqs[i])

        th = [threading.Thread(target=client, args=(range(t, len(reqs), 3),)) for t in range(3)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        res = [srv.wait(i, timeout=120) for i in ids]
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["failed"] == 0
        assert st["batches"] < len(reqs), "requests that queued together were batched"
        assert st["p50_ms"] > 0 and st["p99_ms"] >= st["p50_ms"]
    _same(res[R], alone)
    # equal to plain single-request updates on separate contexts
    for i in (0, 5, R, 30, 47):
        ds, alpha, W = reqs[i]
        ctx = dvl.DVL(0)
        try:
            ctx.load_amr(*data[ds])
            ctx.build_order(dvl.SFC_HILBERT)
            ctx.set_tfs(alpha)
            ctx.update(width=W)
            for m in range(4):
                b = ctx.read_bins(m)
                _same({k: res[i][k][m] if k != "count" else res[i][k] for k in b}, b)
        finally:
            ctx.close()


def test_served_request_matches_oracle():
    a = synth.make("small")
    alpha = synth.random_tfs(77)
    with DVLServer(0, max_batch=4, max_width=1024) as srv:
        srv.add_dataset(a.lower, a.level, a.fields)
        r = srv.wait(srv.submit(0, alpha, 1000), timeout=120)
    _, _, lev, fl = oracle.sorted_inputs(a.lower, a.level, a.fields, oracle.SFC_HILBERT)
    o = oracle.update(fl, lev, alpha, None, None, width=1000)
    for m in range(4):
        assert_bins_match({k: (r[k][m] if k != "count" else r[k]) for k in r}, o, m, 256, alpha[m])


def test_memory_admission_limits_batches():
    lo, lev, f = _random_amr(3, 50000)
    with DVLServer(0, max_batch=16, max_width=1024) as srv:
        srv.add_dataset(lo, lev, f)
        st = srv.stats()
    resident, slot = st["mem_used"], st["slot_bytes"]
    assert resident > 0 and slot > 0
    # room for the data set and two TF slots: batches of at most 2
    with DVLServer(0, mem_budget=resident + int(2.5 * slot), max_batch=16, max_width=1024) as srv:
        srv.add_dataset(lo, lev, f)
        tfs = [synth.random_tfs(i) for i in range(10)]
        ids = [srv.submit(0, t, 1024) for t in tfs]
        res = [srv.wait(i, timeout=120) for i in ids]
        st = srv.stats()
        assert st["completed"] == 10 and st["max_batch_seen"] <= 2
        assert st["mem_used"] <= st["mem_budget"]
        alone = srv.wait(srv.submit(0, tfs[3], 1024), timeout=120)
        _same(res[3], alone)
    # room for the data set only: requests fail, the server keeps running
    with DVLServer(0, mem_budget=resident + 1, max_batch=16, max_width=1024) as srv:
        srv.add_dataset(lo, lev, f)
        with pytest.raises(dvl.DVLError) as e:
            srv.wait(srv.submit(0, tfs[0], 1024), timeout=120)
        assert e.value.status == dvl.ERR_NOMEM
        with pytest.raises(dvl.DVLError):
            srv.wait(srv.submit(0, tfs[1], 1024), timeout=120)
    # not even the data set fits
    with DVLServer(0, mem_budget=resident // 2, max_batch=4, max_width=1024) as srv:
        with pytest.raises(dvl.DVLError) as e:
            srv.add_dataset(lo, lev, f)
        assert e.value.status == dvl.ERR_NOMEM


def test_server_errors_and_warmup():
    lo, lev, f = _random_amr(4, 3000)
    with DVLServer(0, max_batch=8, max_width=512) as srv:
        did = srv.add_dataset(lo, lev, f)
        srv.warmup()
        assert srv.stats()["completed"] == 0                # warm-up is not counted
        t = synth.random_tfs(1)
        with pytest.raises(dvl.DVLError):
            srv.submit(did + 1, t, 256)                     # no such data set
        with pytest.raises(dvl.DVLError):
            srv.submit(did, t, 513)                         # wider than max_width
        bad = t.copy()
        bad[0, 3] = -0.5
        with pytest.raises(dvl.DVLError):
            srv.submit(did, bad, 256)                       # alpha outside [0, 1]
        r = srv.wait(srv.submit(did, t, 256), timeout=120)
        assert r["count"].sum() >= 3000


def _overlap_ms(tl, a="run_start_ms", b="run_end_ms"):
    """Device time during which batches of at least two different data sets
    were running (the union of their pairwise intersections), and the time at
    least one batch was running."""
    ev = []
    for r in tl:
        ev.append((float(r[a]), 1, int(r["dataset"])))
        ev.append((float(r[b]), -1, int(r["dataset"])))
    ev.sort(key=lambda e: (e[0], e[1]))
    active, last, both, busy = {}, None, 0.0, 0.0
    for t, d, ds in ev:
        if last is not None:
            live = [k for k, c in active.items() if c > 0]
            if len(live) >= 1:
                busy += t - last
            if len(live) >= 2:
                both += t - last
        active[ds] = active.get(ds, 0) + d
        last = t
    return both, busy


def test_datasets_overlap_on_device():
    """Batches of different data sets run on their own streams at the same
    time.  With a stream of requests for two data sets, the timeline shows
    batches of both data sets in flight on the device together: the CUDA
    events recorded around their kernels on the two streams give intersecting
    spans.  Each batch's device-clock run interval (its first kernel's start
    to its last kernel's end) lies inside its event span.  Whether kernels of
    the two execute at the same instant depends on how fast requests arrive
    relative to a batch's run time (here a Python loop submits them); the
    benchmark's serving record reports that share of busy time at the
    offered and the saturated load.  Every result still equals a plain
    update."""
    # data sets large enough that a batch's device time (~0.4 ms) exceeds the
    # host time of launching the next one
    a = synth.make("paper", box=((0, 0, 0), 48))
    b = synth.make("paper", box=((16, 16, 16), 48))
    assert a.n > 12_000_000 and b.n > 12_000_000
    reqs = [(i % 2, synth.random_tfs(4000 + i), 1024) for i in range(64)]
    with DVLServer(0, max_batch=8, max_inflight=2, max_width=1024) as srv:
        for d in (a, b):
            srv.add_dataset(d.lower, d.level, d.fields)
        srv.warmup()
        srv.reset_stats()
        ids = [srv.submit(*r) for r in reqs]
        got = [srv.wait(i, timeout=120) for i in ids]
        tl = srv.timeline()
        st = srv.stats()
    assert len(tl) == st["batches"] and set(tl["dataset"].tolist()) == {0, 1}
    assert int(tl["requests"].sum()) == len(reqs)
    assert np.all(tl["end_ms"] > tl["start_ms"]) and tl["start_ms"].min() == 0.0
    assert np.all(tl["run_end_ms"] > tl["run_start_ms"]) and tl["run_start_ms"].min() == 0.0
    # a batch runs inside its events' span (different clocks: compare durations)
    assert np.all(tl["run_end_ms"] - tl["run_start_ms"] <= tl["end_ms"] - tl["start_ms"] + 0.05)
    rows = "\n".join(f"ds {r['dataset']} k {r['requests']} ev [{r['start_ms']:.3f}, {r['end_ms']:.3f}] "
                      f"run [{r['run_start_ms']:.3f}, {r['run_end_ms']:.3f}]" for r in tl)
    both_ev, _ = _overlap_ms(tl, "start_ms", "end_ms")
    assert both_ev > 0.0, "no two data sets' batches in flight together:\n" + rows
    both_run, busy = _overlap_ms(tl)
    assert 0.0 <= both_run <= busy
    ctxs = []
    try:
        for d in (a, b):
            c = dvl.DVL(0)
            c.load_amr(d.lower, d.level, d.fields)
            c.build_order(dvl.SFC_HILBERT)
            ctxs.append(c)
        for (ds, tf, W), g in zip(reqs, got):
            ctxs[ds].set_tfs(tf)
            ctxs[ds].update(width=W)
            for m in range(4):
                ref = ctxs[ds].read_bins(m)
                _same({k: (g[k][m] if k != "count" else g[k]) for k in g}, ref)
    finally:
        for c in ctxs:
            c.close()
