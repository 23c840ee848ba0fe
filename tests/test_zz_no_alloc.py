"""The allocation-free entry point (dvl_update_noalloc) gives the same bins as
dvl_update (GPU).

dvl_update_noalloc serves callers that may not allocate device memory where
they run an update (a render callback inside someone else's memory budget, a
fixed-pool process, code that must not trigger cudaFree's device-wide sync):
it works on the caller's buffers plus one fixed scratch array inside the
library.  This file is collected last on purpose.  Two calls in a row (with
different transfer functions, widths and exponents) must each match the
context-based dvl_update on the same cells, within the tolerances of the other
parity tests: counts and min/max bit for bit, sums and means to 1e-5
relative, y exactly away from TF bucket boundaries.  And the calls must leave
device memory as they found it: the free memory the driver reports and the
bytes torch holds are the same before and after a repeat of the same calls
(the first round of calls may load the library's kernels and its fixed
scratch array, which the driver does on first use).
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

dvl = pytest.importorskip("paper_2306_11612_b300")
torch = pytest.importorskip("torch")


def _reference(ctx, alpha, **kw):
    ctx.set_tfs(alpha)
    ctx.update(**kw)
    return [ctx.read_bins(m) for m in range(alpha.shape[0])]


def _compare(ref, got, m, W, T):
    sl = slice(m * W, (m + 1) * W)
    assert np.array_equal(got["count"][:W].view(np.uint32), ref["count"])
    assert np.array_equal(got["min"][sl].view(np.uint32), ref["min"].view(np.uint32))
    assert np.array_equal(got["max"][sl].view(np.uint32), ref["max"].view(np.uint32))
    assert np.allclose(got["sum"][sl], ref["sum"], rtol=1e-5, atol=0)
    assert np.allclose(got["mean"][sl], ref["mean"], rtol=1e-5, atol=0)
    x = ref["mean"].astype(np.float64) * T
    away = np.abs(x - np.round(x)) > 1e-5 * np.maximum(x, 1.0)
    assert np.array_equal(got["y"][sl][away], ref["y"][away])


def test_noalloc_matches_update_on_two_calls():
    amr = synth.make("small")
    n, M = amr.n, 4
    dev = torch.device("cuda:0")
    ctx = dvl.DVL(0)
    try:
        ctx.load_amr(amr.lower, amr.level, amr.fields)
        ctx.build_order(dvl.SFC_HILBERT)
        _, perm = ctx.read_order()
        pitch = (n + 3) // 4 * 4 + 4            # any multiple of 4 >= n rounded up
        fields = np.zeros((M, pitch), np.float32)
        fields[:, :n] = amr.fields[:, perm]
        level = np.zeros(pitch, np.uint8)
        level[:n] = amr.level[perm]
        d_fields = torch.from_numpy(fields).to(dev)
        d_level = torch.from_numpy(level).to(dev)
        stream = torch.cuda.current_stream()
        nan = float("nan")
        calls = []
        for seed, kw in [(3, dict(P=1.0, min_importance=0.025, width=1024)),
                         (4, dict(P=2.0, min_importance=0.1, width=333))]:
            alpha = synth.random_tfs(seed)
            W = kw["width"]
            out = {k: torch.full((M * W,), 7, dtype=dt, device=dev) for k, dt in
                   [("mean", torch.float32), ("min", torch.float32), ("max", torch.float32),
                    ("y", torch.float32), ("sum", torch.float64)]}
            out["count"] = torch.full((W,), 7, dtype=torch.int32, device=dev)
            calls.append((alpha, torch.from_numpy(alpha).to(dev), kw, out, _reference(ctx, alpha, **kw)))
        torch.cuda.synchronize()
        for rnd in range(2):
            if rnd == 1:
                free0, held0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
            for call, (alpha, d_alpha, kw, out, ref) in enumerate(calls):
                for v in out.values():
                    v.fill_(7)
                rc = dvl.dvl_update_noalloc(stream, d_fields, pitch, d_level, d_alpha, [nan] * (2 * M), out,
                                            n_cells=n, **kw)
                assert rc == dvl.OK, (rnd, call, rc)
                got = {k: v.cpu().numpy() for k, v in out.items()}
                for m in range(M):
                    _compare(ref[m], got, m, kw["width"], alpha.shape[1])
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, "device memory changed across allocation-free calls"
        assert torch.cuda.memory_allocated() == held0
        # levels only 4-byte aligned: pass A reads the cells directly instead
        # of through bulk copies (which need 16-byte aligned rows)
        lev_store = torch.zeros(pitch + 16, dtype=torch.uint8, device=dev)
        d_level4 = lev_store[4:4 + pitch]
        d_level4.copy_(d_level)
        kw = dict(P=1.0, min_importance=0.025, width=700)
        alpha = synth.random_tfs(5)
        ref = _reference(ctx, alpha, **kw)
        out = {k: torch.full((M * 700,), 7, dtype=dt, device=dev) for k, dt in
               [("mean", torch.float32), ("min", torch.float32), ("max", torch.float32),
                ("y", torch.float32), ("sum", torch.float64)]}
        out["count"] = torch.full((700,), 7, dtype=torch.int32, device=dev)
        assert d_level4.data_ptr() % 16 == 4
        rc = dvl.dvl_update_noalloc(stream, d_fields, pitch, d_level4, torch.from_numpy(alpha).to(dev),
                                    [nan] * (2 * M), out, n_cells=n, **kw)
        assert rc == dvl.OK
        got = {k: v.cpu().numpy() for k, v in out.items()}
        for m in range(M):
            _compare(ref[m], got, m, 700, alpha.shape[1])
        # sizes beyond the fixed scratch are refused before any GPU work
        rc = dvl.dvl_update_noalloc(stream, d_fields, pitch, d_level, torch.from_numpy(alpha).to(dev),
                                    [nan] * (2 * M), out, n_cells=476_749_825, width=333)
        assert rc == dvl.ERR_RANGE
    finally:
        ctx.close()
