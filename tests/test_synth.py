"""Host-side checks of the seeded synthetic workloads (no method arithmetic)."""
import numpy as np

from paper_2101_02005_gb300 import synth


def test_lognormal_counts_sum_and_determinism():
    c = synth.lognormal_window_counts(1_000_003, 300, 123)
    assert c.sum() == 1_000_003 and c.min() >= 0 and c.size == 300
    assert np.array_equal(c, synth.lognormal_window_counts(1_000_003, 300, 123))
    assert c.max() / np.median(c) > 10          # uneven density, sigma = 1.5


def test_lines_sorted_in_range_and_distributions():
    L = synth.make_lines(200_000, 0.0, 30000.0, 77, 18.0, windows=300)
    assert L.nu0.dtype == np.float64 and L.S_ref.dtype == np.float32
    assert np.all(np.diff(L.nu0) >= 0) and L.nu0.min() >= 0 and L.nu0.max() < 30000
    lS = np.log10(L.S_ref.astype(np.float64))
    assert -30.001 <= lS.min() and lS.max() <= -18.999 and abs(lS.mean() + 24.5) < 0.05
    assert abs(L.E_low.mean() / 3000 - 1) < 0.02
    assert 0.01 <= L.gamma_ref.min() and L.gamma_ref.max() <= 0.1
    assert 0.3 <= L.n_T.min() and L.n_T.max() <= 0.8
    # same seed, same lists; unsorted variant has the same other fields
    L2 = synth.make_lines(200_000, 0.0, 30000.0, 77, 18.0, windows=300)
    assert np.array_equal(L.nu0, L2.nu0) and np.array_equal(L.S_ref, L2.S_ref)
    U = synth.make_lines(200_000, 0.0, 30000.0, 77, 18.0, windows=300, sort=False)
    assert np.array_equal(U.S_ref, L.S_ref) and not np.all(np.diff(U.nu0) >= 0)


def test_configs_small_scale():
    w0 = synth.config(0)
    assert w0.species[0].n == 10_000 and w0.grid.nbins == 30000 and w0.cut == 25.0
    w3 = synth.config(3, scale=1e-4)
    assert len(w3.species) == 4 and len(w3.states()) == 200
    assert [s.mass_amu for s in w3.species] == [18.0, 16.0, 44.0, 28.0]
    w4 = synth.config(4, scale=1e-3)
    assert len(w4.states()) == 16
    g = synth.upstream_grad(16, 100, synth.SEED_BASE + 4)
    assert g.shape == (16, 100) and abs(g.mean()) < 0.1
