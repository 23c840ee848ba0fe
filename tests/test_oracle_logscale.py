"""Pins of the oracle's per-field log10 value scale (CPU only).

The log10 is pinned to float64's log10 (numpy) within 1.5 ulp on a stratified
sample of every binade of positive floats (subnormals included), on the
neighbourhoods of the places where its argument reduction switches (the
sqrt(2) boundary of the mantissa, the subnormal/normal boundary) and on all
powers of two and exact powers of ten; log10(1) is exactly 0.  The field
transform is pinned by hand-built fields: values <= 0 take the field's
smallest positive value, unflagged fields stay untouched, and a field without
a positive value is refused.
"""
import numpy as np
import pytest

import oracle

ULP_BOUND = 1.5


def _ulp_err(x):
    x = np.asarray(x, np.float32)
    y = oracle.log_fields(x[None, :], 1)[0].astype(np.float64)
    ref = np.log10(x.astype(np.float64))
    rf = np.abs(ref).astype(np.float32)
    ulp = np.spacing(np.where(rf == 0, np.float32(1e-45), rf)).astype(np.float64)
    return np.abs(y - ref) / ulp, y


def test_log10_stratified_sample():
    # every 1021st bit pattern of the positive finite floats plus random ones
    bits = np.arange(1, 0x7F800000, 1021 * 2 + 1, dtype=np.uint64).astype(np.uint32)
    rnd = np.random.default_rng(7).integers(1, 0x7F800000, 200_000, dtype=np.uint32)
    x = np.concatenate([bits, rnd]).view(np.float32)
    err, _ = _ulp_err(x)
    assert err.max() <= ULP_BOUND, (err.max(), x[np.argmax(err)])


def test_log10_reduction_boundaries():
    s2 = np.float32(np.sqrt(2.0))
    b = []
    for e in range(-149, 128):
        for c in (np.float32(1.0), s2):
            base = np.ldexp(np.float64(c), e)
            if base <= 0 or base >= 3.4e38 or base < 1.4e-45:
                continue
            cb = np.float32(base).view(np.uint32)
            b.append(np.arange(max(1, int(cb) - 40), min(0x7F7FFFFF, int(cb) + 40), dtype=np.uint32))
    b.append(np.arange(0x007FFF00, 0x00800100, dtype=np.uint32))     # subnormal / normal
    x = np.concatenate(b).view(np.float32)
    err, _ = _ulp_err(x)
    assert err.max() <= ULP_BOUND, (err.max(), x[np.argmax(err)])


def test_log10_exact_points():
    assert oracle.log10f(np.float32(1.0)) == 0.0
    e = np.arange(-149, 128)
    x = np.ldexp(np.float32(1.0), e).astype(np.float32)
    err, y = _ulp_err(x)
    assert err.max() <= 1.0
    assert np.all(np.sign(y) == np.sign(e))
    p10 = np.array([10.0 ** k for k in range(0, 11)], np.float32)      # exact in float32
    err, y = _ulp_err(p10)
    assert err.max() <= ULP_BOUND
    assert np.all(np.abs(y - np.arange(11)) <= 4e-6 * np.maximum(1, np.arange(11)))


def test_log10_monotone_on_decades():
    # strictly increasing across decades and ordered within a sorted sample
    x = np.sort(np.random.default_rng(3).uniform(1e-30, 1e30, 50_000).astype(np.float32))
    y = oracle.log10f(x)
    d = np.diff(y.astype(np.float64))
    assert np.all(d >= -2 * np.spacing(np.abs(y[1:])).astype(np.float64))


def test_log_fields_clamp_and_mask():
    f = np.array([[-1.0, 0.0, 2.0, 4.0, 0.5, 1e-3],
                  [3.0, -2.0, 0.0, 1.0, 7.0, 8.0],
                  [1.0, 10.0, 100.0, 0.0, 1000.0, 1e-6]], np.float32)
    out = oracle.log_fields(f, 0b101)
    # field 1 is not flagged: untouched
    assert np.array_equal(out[1], f[1])
    # field 0: -1 and 0 take the smallest positive value 1e-3
    clamp0 = np.array([1e-3, 1e-3, 2.0, 4.0, 0.5, 1e-3], np.float32)
    assert np.array_equal(out[0], oracle.log10f(clamp0))
    assert out[0][0] == out[0][1] == out[0][5] == out[0].min()
    # field 2: the zero takes 1e-6; exact decades land on their exponent
    clamp2 = np.array([1.0, 10.0, 100.0, 1e-6, 1000.0, 1e-6], np.float32)
    assert np.array_equal(out[2], oracle.log10f(clamp2))
    assert np.allclose(out[2], [0, 1, 2, -6, 3, -6], atol=4e-6)
    assert out[2].argmax() == 4


def test_log_fields_needs_a_positive_value():
    f = np.array([[0.0, -1.0, -3.0]], np.float32)
    with pytest.raises(oracle.OracleError):
        oracle.log_fields(f, 1)
    # an unflagged non-positive field is fine
    assert np.array_equal(oracle.log_fields(f, 0), f)


def test_log_fields_subnormal_minimum():
    tiny = np.float32(1e-44)                    # subnormal, the smallest positive value
    f = np.array([[tiny, 0.0, 1.0]], np.float32)
    out = oracle.log_fields(f, 1)[0]
    assert out[0] == out[1]
    assert abs(out[0] - np.log10(np.float64(tiny))) <= 1.5 * np.spacing(np.float32(44.0))
