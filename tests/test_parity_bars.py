"""The parity bars themselves (CPU): a result within rounding of the oracle
passes, and plausible mistakes of a GPU path fail -- a dropped plinth, a
plinth removed twice, one line's contribution missing, a small systematic
scale error.  The 'GPU' results here are the oracle's own, perturbed on the
CPU."""
import numpy as np
import pytest

import oracle
from parity import assert_plinth_close, assert_sigma_close
from paper_2101_02005_gb300 import synth

Q = synth.partition_function
QREF = float(Q(296.0))


@pytest.fixture(scope="module")
def arrays():
    L = synth.make_lines(400, 0.0, 400.0, synth.SEED_BASE + 21, 18.0)
    grid = (0.0, 0.1, 4000)
    st = (1000.0, 1.0, float(Q(1000.0)), QREF)
    base = oracle.cross_section(L.as_oracle(), grid, st, 25.0)
    ref = oracle.cross_section(L.as_oracle(), grid, st, 25.0, plinth=True)
    one = L.subset(slice(0, 1))
    single = oracle.cross_section(one.as_oracle(), grid, st, 25.0, plinth=True)
    return base, ref, single


def test_rounding_passes(arrays):
    base, ref, _ = arrays
    rng = np.random.default_rng(5)
    # a float-like error on every term: relative 1e-7 of the terms summed
    got = ref + 1e-7 * base * rng.standard_normal(base.size)
    got[ref == 0] = 0.0
    assert_plinth_close(got, ref, base)
    assert_sigma_close(base * (1 + 1e-7 * rng.standard_normal(base.size)), base)


def test_plinth_mistakes_fail(arrays):
    base, ref, single = arrays
    plinths = base - ref
    assert np.max(plinths) > 0
    with pytest.raises(AssertionError):
        assert_plinth_close(base, ref, base, "plinth not removed")
    with pytest.raises(AssertionError):
        assert_plinth_close(ref - plinths, ref, base, "plinth removed twice")
    with pytest.raises(AssertionError):
        assert_plinth_close(ref - single, ref, base, "one line missing")
    with pytest.raises(AssertionError):
        assert_plinth_close(ref * (1 + 3e-5), ref, base, "scale error 3e-5")


def test_sigma_mistakes_fail(arrays):
    base, _, _ = arrays
    with pytest.raises(AssertionError):
        assert_sigma_close(base * (1 + 2e-5), base, "scale error 2e-5")
    bad = base.copy()
    bad[np.argmax(base)] *= 1.0002
    with pytest.raises(AssertionError):
        assert_sigma_close(bad, base, "one bin off by 2e-4")
