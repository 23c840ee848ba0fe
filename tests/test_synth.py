"""The synthetic-input generator's sub-box cut (CPU only).

Serving and the benchmark cut sub-boxes of base cells out of a data set that
is already generated instead of evaluating the noise again; the cut must give
exactly what the generator gives for that box (same cells, fields, order),
and the serving sizes must span the stated range.
"""
import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def diff_full():
    return synth.make("diff")


@pytest.mark.parametrize("box", [((5, 17, 30), 20), ((0, 0, 0), 64), ((63, 63, 63), 1), ((10, 0, 40), 24)])
def test_sub_box_equals_generated_box(diff_full, box):
    sub = synth.make("diff", box=box)
    cut = synth.sub_box(diff_full, box)
    assert cut.n == sub.n
    assert np.array_equal(cut.lower, sub.lower) and np.array_equal(cut.level, sub.level)
    assert np.array_equal(cut.fields.view(np.uint32), sub.fields.view(np.uint32))


def test_serving_sizes_span_one_to_two_hundred_million():
    sizes = [c for _, c in synth.SERVING]
    assert len(sizes) == 8
    assert min(sizes) < 1.5e6 and max(sizes) > 1.8e8
    # stratified log-uniform: consecutive sizes about a factor 200^(1/7) apart
    r = np.diff(np.log(sorted(sizes)))
    assert np.all(np.abs(r - np.log(200) / 7) < 0.25)
