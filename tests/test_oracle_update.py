"""Pins of the oracle's DVL update (CPU only).

Each check ties the C oracle to something other than itself:
* a hand-worked example (tests/golden/worked_4cells.json);
* the exact-rational brute force of oracle/brute.py, on dyadic inputs where
  every float32 step is exact (so the results must agree exactly), and on
  random inputs with the oracle's integer widths (placement and binning);
* closed forms: P = 0 is the linear mapping b = floor(c W / N) (the row-major
  baseline of Sec. 2.2); a constant field gives V = 0 and widths (m 2^L)^P;
* invariants: the spans tile [0, F), every pixel is covered, the counter
  equals the number of (cell, pixel) incidences.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle.brute import brute_update

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "worked_4cells.json")))
    fields = np.array(g["fields"], np.float32)
    level = np.array(g["level"], np.uint8)
    alpha = np.array(g["alpha"], np.float32)
    for case in g["cases"]:
        r = oracle.update(fields, level, alpha, per_cell=True, P=case["P"],
                          min_importance=g["min_importance"], width=g["W"])
        st = r["stats"]
        assert st["vmax"] == g["vmax"] and (st["i"], st["j"]) == (g["i"], g["j"])
        unit = 2.0 ** st["Q"]
        assert np.array_equal(r["q"], (np.array(case["f"]) * unit).astype(np.uint64))
        assert st["F"] == int(case["F_over_unit"] * unit)
        assert r["b1"].tolist() == g["b1"] and r["b2"].tolist() == g["b2"]
        assert r["count"].tolist() == g["count"]
        assert np.array_equal(r["sum"], np.array(g["sum"]))
        assert np.array_equal(r["min"], np.array(g["min"], np.float32))
        assert np.array_equal(r["max"], np.array(g["max"], np.float32))
        assert np.allclose(r["mean64"], np.array(g["mean"]), rtol=1e-15, atol=0)
        assert np.array_equal(r["y"], np.array(g["y"], np.float32))


def _dyadic_case(rng, n, M, T, allow_zero_vmax=False):
    """Inputs on which every float32 operation of the update is exact."""
    k = int(rng.integers(1, 5))
    hi = 1 << k
    fields = rng.integers(0, hi + 1, (M, n)).astype(np.float32)
    fields[:, 0] = 0
    fields[:, -1] = hi                     # data range [0, 2^k] for every field
    alpha = (rng.integers(0, 9, (M, T)) / 8.0).astype(np.float32)
    if M >= 2 and not allow_zero_vmax:
        a = int(rng.integers(0, T))        # force max V = 1 (exact reciprocal)
        alpha[0, a], alpha[1, a] = 0.0, 1.0
    level = rng.integers(0, 4, n).astype(np.uint8)
    return fields, level, alpha


@pytest.mark.parametrize("seed", range(40))
def test_brute_force_exact_on_dyadic_inputs(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 200))
    M = int(rng.integers(1, 5))
    T = int(rng.choice([4, 8, 16]))
    W = int(rng.choice([1, 2, 3, 7, 16, 64, 300]))
    P = int(rng.choice([0, 1, 2, 3]))
    mi = Fraction(int(rng.choice([0, 1, 8])), 32)
    mode = int(rng.integers(0, 2))
    wmode = int(rng.integers(0, 2)) if P <= 2 else 0
    fields, level, alpha = _dyadic_case(rng, n, M, T)
    r = oracle.update(fields, level, alpha, per_cell=True, P=P, min_importance=float(mi), width=W,
                      min_imp_mode=mode, width_mode=wmode)
    b = brute_update(fields.tolist(), level.tolist(), alpha.tolist(), W, P=P, min_importance=mi,
                     min_imp_mode=mode, width_mode=wmode)
    st = r["stats"]
    assert Fraction(float(st["vmax"])) == b["vmax"] and (st["i"], st["j"]) == (b["i"], b["j"])
    unit = Fraction(2) ** st["Q"]
    if not st["linear"]:
        assert [Fraction(int(x)) for x in r["q"]] == [f * unit for f in b["f"]]
    assert r["b1"].tolist() == b["b1"] and r["b2"].tolist() == b["b2"]
    assert r["count"].tolist() == b["count"]
    for m in range(M):
        for p in range(W):
            if b["count"][p]:
                assert Fraction(float(r["sum"][m, p])) == b["sum"][m][p]   # dyadic sums are exact
                assert Fraction(float(r["min"][m, p])) == b["min"][m][p]
                assert Fraction(float(r["max"][m, p])) == b["max"][m][p]


@pytest.mark.parametrize("seed", range(12))
def test_brute_force_placement_random_inputs(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 400))
    M = int(rng.integers(1, 5))
    T = 256
    W = int(rng.choice([1, 5, 64, 1000]))
    fields = rng.lognormal(0, 2, (M, n)).astype(np.float32)
    alpha = rng.uniform(0, 1, (M, T)).astype(np.float32)
    level = rng.integers(0, 6, n).astype(np.uint8)
    P = float(rng.choice([0.5, 1.0, 1.5, 2.0, 5.0]))
    r = oracle.update(fields, level, alpha, per_cell=True, P=P, min_importance=0.025, width=W)
    b = brute_update(fields.tolist(), level.tolist(), alpha.tolist(), W, widths=r["q"].tolist())
    assert r["b1"].tolist() == b["b1"] and r["b2"].tolist() == b["b2"]
    assert r["count"].tolist() == b["count"]
    for m in range(M):
        for p in range(W):
            if b["count"][p]:
                assert abs(r["sum"][m, p] - float(b["sum"][m][p])) <= 1e-6 * float(b["sum"][m][p]) + 1e-12
    # the fixed-point widths follow the real-valued Eq. 3 to float32 accuracy
    if P in (1.0, 2.0):
        bf = brute_update(fields.tolist(), level.tolist(), alpha.tolist(), W, P=int(P),
                          min_importance=Fraction(0.025))
        unit = 2.0 ** r["stats"]["Q"]
        exact = np.array([float(f) * unit for f in bf["f"]])
        assert np.all(np.abs(r["q"] - exact) <= 1e-5 * exact + 1.0)


@pytest.mark.parametrize("n,W", [(1, 1), (7, 3), (100, 1024), (1000, 64), (4097, 4096)])
def test_p0_is_linear_mapping(n, W):
    rng = np.random.default_rng(n)
    fields = rng.normal(size=(2, n)).astype(np.float32)
    alpha = rng.uniform(size=(2, 256)).astype(np.float32)
    level = rng.integers(0, 5, n).astype(np.uint8)
    r = oracle.update(fields, level, alpha, per_cell=True, P=0.0, width=W)
    c = np.arange(n, dtype=object)
    b1 = [min(x * W // n, W - 1) for x in c]
    b2 = [min(-((-(x + 1) * W) // n) - 1, W - 1) for x in c]
    assert r["b1"].tolist() == b1 and r["b2"].tolist() == b2


def test_constant_field_widths():
    rng = np.random.default_rng(7)
    n = 500
    fields = np.full((3, n), 2.5, np.float32)
    alpha = np.repeat(rng.uniform(size=(1, 256)).astype(np.float32), 3, axis=0)  # identical TFs
    level = rng.integers(0, 4, n).astype(np.uint8)
    for P in (1.0, 2.0, 3.0):
        r = oracle.update(fields, level, alpha, per_cell=True, P=P, min_importance=0.125, width=97)
        assert r["stats"]["vmax"] == 0.0
        unit = 2.0 ** r["stats"]["Q"]
        expect = np.array([(0.125 * 2.0 ** int(L)) ** P * unit for L in level])
        assert np.array_equal(r["q"].astype(np.float64), expect)


def test_single_level_uniform_when_variation_zero():
    n, W = 999, 128
    fields = np.ones((2, n), np.float32)
    alpha = np.zeros((2, 256), np.float32)
    r1 = oracle.update(fields, np.full(n, 2, np.uint8), alpha, per_cell=True, P=1, width=W)
    r0 = oracle.update(fields, np.full(n, 2, np.uint8), alpha, per_cell=True, P=0, width=W)
    assert np.array_equal(r1["b1"], r0["b1"]) and np.array_equal(r1["b2"], r0["b2"])


def _invariants(r, n, W):
    b1, b2, q = r["b1"].astype(np.int64), r["b2"].astype(np.int64), r["q"]
    assert np.all(b2 >= b1)
    assert np.all(b1[1:] >= b2[:-1])
    if n:
        assert b1[0] == 0 and b2[-1] == W - 1
    assert int(r["count"].sum()) == int((b2 - b1 + 1).sum())
    assert r["stats"]["F"] == int(q.sum(dtype=np.uint64))
    assert np.all(r["count"] >= 1)                       # the spans tile [0, F)
    cnt = np.bincount(np.concatenate([np.arange(a, b + 1) for a, b in zip(b1, b2)]), minlength=W)
    assert np.array_equal(cnt, r["count"])


def test_invariants_small_config():
    import synth
    a = synth.make("small")
    _, perm, lev, fl = oracle.sorted_inputs(a.lower, a.level, a.fields, oracle.SFC_MORTON)
    alpha = synth.random_tfs(11)
    for P, W in [(1.0, 1024), (2.0, 4096), (0.5, 333)]:
        r = oracle.update(fl, lev, alpha, per_cell=True, P=P, width=W)
        _invariants(r, a.n, W)
        assert r["stats"]["Q"] > 0 and not r["stats"]["linear"]
        assert np.all(r["min"] <= r["mean"]) and np.all(r["mean"] <= r["max"])


def test_zero_width_cells_and_wide_plot():
    rng = np.random.default_rng(9)
    n, W = 300, 5000                      # W > N: cells span several pixels
    fields = np.repeat(rng.lognormal(size=(1, n)).astype(np.float32), 4, axis=0)
    alpha = np.repeat(rng.uniform(size=(1, 256)).astype(np.float32), 4, axis=0)
    fields[1, ::7] *= 3.0                 # a few cells get V > 0, the rest V = 0
    alpha[1, 255] = 1.0 - alpha[0, 255]   # max V > 0 (the top entry is in range)
    level = rng.integers(0, 3, n).astype(np.uint8)
    dom = [0.0] * 4, [float(fields.max())] * 4     # one domain: unscaled cells have V = 0
    r = oracle.update(fields, level, alpha, dom[0], dom[1], per_cell=True, P=8.0,
                      min_importance=1e-4, width=W)
    assert np.any(r["q"] == 0)            # (1e-4)^8 underflows the fixed-point quantum
    _invariants(r, n, W)


def test_all_zero_widths_fall_back_to_linear():
    n, W = 50, 20
    fields = np.ones((2, n), np.float32)
    alpha = np.zeros((2, 16), np.float32)
    r = oracle.update(fields, np.zeros(n, np.uint8), alpha, per_cell=True, P=1, min_importance=0.0, width=W)
    assert r["stats"]["linear"] == 1 and r["stats"]["F"] == n
    assert np.all(r["q"] == 1)


def test_empty_input():
    r = oracle.update(np.zeros((2, 0), np.float32), np.zeros(0, np.uint8), np.zeros((2, 8), np.float32),
                      width=16)
    assert np.all(r["count"] == 0) and np.all(r["sum"] == 0) and r["stats"]["F"] == 0


def test_vmax_exact_mode_is_max_of_variation():
    rng = np.random.default_rng(4)
    n = 2000
    fields = rng.normal(size=(3, n)).astype(np.float32)
    alpha = rng.uniform(size=(3, 64)).astype(np.float32)
    level = np.zeros(n, np.uint8)
    r = oracle.update(fields, level, alpha, per_cell=True, P=1, min_importance=0.0, width=10, vmax_mode=1)
    # with P = 1, no minimum and one level, q is proportional to V / max V:
    # the largest width is exactly rint(1 * 2^Q)
    assert int(r["q"].max()) == 2 ** r["stats"]["Q"]
    # brute force over the cells: the largest spread of the looked-up alphas
    lo, hi = fields.min(1), fields.max(1)
    s = (np.float32(1) / (hi - lo)).astype(np.float32)
    t = np.clip(((fields - lo[:, None]).astype(np.float32) * s[:, None]).astype(np.float32), 0, 1)
    e = np.minimum(np.floor(t * np.float32(64)).astype(np.int64), 63)
    a = np.take_along_axis(alpha, e, 1)
    assert np.float32(r["stats"]["vmax"]) == np.max(a.max(0) - a.min(0))
    # Eq. 6 pairs the fields' entries by index: when every field has the same
    # values (so every cell looks up one entry index in all tables) and all
    # entries between the data minimum's and maximum's are reached, the
    # approximation equals the exact maximum
    same = np.repeat(np.linspace(-1, 1, 64 * 8, dtype=np.float32)[None], 3, axis=0)
    lv = np.zeros(same.shape[1], np.uint8)
    ex = oracle.update(same, lv, alpha, P=1, min_importance=0.0, width=10, vmax_mode=1)["stats"]
    ap = oracle.update(same, lv, alpha, P=1, min_importance=0.0, width=10, vmax_mode=0)["stats"]
    assert (ap["i"], ap["j"]) == (0, 63) and ap["vmax"] == ex["vmax"] == np.max(alpha.max(0) - alpha.min(0))


def test_user_domain_clamps():
    fields = np.array([[-5.0, 0.0, 0.5, 1.0, 7.0]], np.float32)
    alpha = np.linspace(0, 1, 4, dtype=np.float32)[None]
    r = oracle.update(fields, np.zeros(5, np.uint8), alpha, dom_lo=[0.0], dom_hi=[1.0], per_cell=True,
                      width=5, P=0)
    # one cell per pixel: min = max = the clamped normalised value
    assert r["min"][0].tolist() == [0.0, 0.0, 0.5, 1.0, 1.0]
    assert r["y"][0].tolist() == [alpha[0, 0], alpha[0, 0], alpha[0, 2], alpha[0, 3], alpha[0, 3]]


@pytest.mark.parametrize("seed", range(6))
def test_widths_of_sampled_cells_equal_update(seed):
    # the one-by-one widths (for full-size sampled checks) equal the widths the
    # whole-data-set update assigns, given the data set's range and deepest level
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(50, 3000))
    M = int(rng.integers(1, 5))
    fields = rng.lognormal(0, 1.5, (M, n)).astype(np.float32)
    level = rng.integers(0, 6, n).astype(np.uint8)
    alpha = rng.uniform(0, 1, (M, 256)).astype(np.float32)
    kw = dict(P=float(rng.choice([1.0, 2.0, 0.5])), min_importance=0.025)
    r = oracle.update(fields, level, alpha, per_cell=True, width=64, **kw)
    pick = rng.choice(n, min(n, 200), replace=False)
    q, Q, vmax = oracle.widths(n, fields.min(1), fields.max(1), int(level.max()), alpha, fields[:, pick],
                               level[pick], **kw)
    assert Q == r["stats"]["Q"] and np.float32(vmax) == np.float32(r["stats"]["vmax"])
    assert np.array_equal(q, r["q"][pick])
