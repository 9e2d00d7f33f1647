"""CUDA path (through the C ABI) against the FP64 oracle, element by element.

Bar: relative L1 <= 1e-5 and per-bin relative error <= 1e-4 over bins with
sigma > 1e-10 max(sigma) (benchmark tolerance), for both the FP32-compensated
and the FP64 GPU forms.  Inputs are the seeded synthetic workloads; sizes are
chosen so the oracle finishes in seconds while spanning many tiles and a
ragged tail.
"""
import math

import numpy as np
import pytest

import oracle
from parity import (assert_plinth_close, assert_sigma_close, oracle_sigma_max, record,
                    round_series_case, sigma_errors)
from paper_2101_02005_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

Q = synth.partition_function
QREF = float(Q(296.0))


@pytest.fixture(scope="module")
def hk():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2101_02005_gb300 import build
    build.build()
    from paper_2101_02005_gb300 import hk
    hk.lib()
    return hk


def oracle_sigma(L, grid, T, P, cut, bin_lo=0, bin_hi=None, per_gram=False):
    return oracle.cross_section(L.as_oracle(), grid.astuple(), (T, P, float(Q(T)), QREF), cut,
                                bin_lo, bin_hi, per_gram=per_gram)


def gpu_sigma(hk, L, grid, T, P, cut, precision, flags=0):
    D = hk.DeviceLines.from_host(L)
    s = hk.hk_cross_section(D, hk.make_grid(*grid.astuple()),
                            hk.make_state(T, P, float(Q(T)), float(synth.dlnQ_dT(T))),
                            hk.make_opts(QREF, cut, precision, flags=flags))
    hk.hk_sync_status()
    return s.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("prec", [0, 1])
def test_config0_full(hk, prec):
    w = synth.config(0)
    L = w.species[0]
    T, P = w.states()[0]
    ref = oracle_sigma(L, w.grid, T, P, w.cut)
    got = gpu_sigma(hk, L, w.grid, T, P, w.cut, prec)
    e = assert_sigma_close(got, ref, f"c0 prec={prec}")
    record(f"c0 {'fp64' if prec else 'fp32c'} (whole array)", e)
    # at 1000 K a few high-E'' lines dominate max(sigma); a few % of bins pass the mask
    assert e["n_mask"] > 500


@pytest.mark.parametrize("prec", [0, 1])
def test_ragged_grid_off_grid_lines_and_cut_variants(hk, prec):
    rng = np.random.default_rng(17)
    n = 700
    nu0 = np.sort(np.concatenate([rng.uniform(-3.0, 103.0, n - 4), [-2.5, 0.0, 99.95, 102.7]]))
    L = synth.LineList(nu0, (10 ** rng.uniform(-24, -20, n)).astype(np.float32),
                       rng.exponential(2000, n).astype(np.float32),
                       rng.uniform(0.01, 0.1, n).astype(np.float32),
                       rng.uniform(0.3, 0.8, n).astype(np.float32), 18.0)
    for nbins, cut in [(1037, 2.5), (2048 + 513, 0.05), (1000, 0.0), (333, 500.0)]:
        grid = synth.Grid(0.0, 100.0 / nbins, nbins)
        ref = oracle_sigma(L, grid, 700.0, 0.3, cut)
        got = gpu_sigma(hk, L, grid, 700.0, 0.3, cut, prec)
        assert_sigma_close(got, ref, f"nbins={nbins} cut={cut} prec={prec}")
        # bins outside every line's cut are exactly zero on both sides
        assert np.array_equal(ref == 0, got == 0)


def test_cut_ties_match_oracle(hk):
    """Line centres on and a hair off bin centres and half-bins, with cuts
    whose W = cut / dnu is an integer, a hair above one, and fractional: the
    cut bounds (FP32 fast path with the exact FP64 walk near ties) give the
    oracle's pair total exactly, the same zero pattern, and parity."""
    deltas = [0.0, 1e-12, -1e-12, 1e-9, -1e-9, 2e-6, -2e-6, 9e-6, -9e-6, 0.5, 0.5 + 1e-9,
              0.5 - 1e-9, 0.25, 0.999999, 1e-5, -1e-5]
    for dnu, cut in [(0.1, 25.0), (0.1, 2.5), (0.01, 1.0), (0.1, 25.0 + 1e-10), (0.1, 0.35),
                     (0.05, 0.125), (0.03, 0.3)]:
        nbins = 1800
        base = np.arange(40, nbins - 40, 97)
        nu0 = np.sort(np.array([(i + d) * dnu for i in base for d in deltas], dtype=np.float64))
        n = nu0.size
        rng = np.random.default_rng(int(cut * 1000) + int(1 / dnu))
        L = synth.LineList(nu0, (10 ** rng.uniform(-22, -20, n)).astype(np.float32),
                           rng.exponential(1000, n).astype(np.float32),
                           rng.uniform(0.01, 0.1, n).astype(np.float32),
                           rng.uniform(0.3, 0.8, n).astype(np.float32), 18.0)
        grid = synth.Grid(0.0, dnu, nbins)
        D = hk.DeviceLines.from_host(L)
        counts = hk.hk_count_pairs(D, hk.make_grid(*grid.astuple()),
                                   hk.make_state(900.0, 0.5, float(Q(900.0))),
                                   hk.make_opts(QREF, cut))
        assert counts[0] == oracle.count_pairs(L.nu0, *grid.astuple(), cut), (dnu, cut)
        ref = oracle_sigma(L, grid, 900.0, 0.5, cut)
        for prec in (0, 1):
            got = gpu_sigma(hk, L, grid, 900.0, 0.5, cut, prec)
            assert_sigma_close(got, ref, f"ties dnu={dnu} cut={cut} prec={prec}")
            assert np.array_equal(ref == 0, got == 0), (dnu, cut, prec)


def test_host_streamed_matches_oracle(hk):
    """hk_cross_section_host: the config-0 list in host memory, streamed in
    ragged blocks (1e4 lines in blocks of 1500), against the oracle and the
    device-resident call; FP64, unsorted and pageable inputs; empty list."""
    w = synth.config(0)
    L = w.species[0]
    T, P = w.states()[0]
    grid = hk.make_grid(*w.grid.astuple())
    st = hk.make_state(T, P, float(Q(T)))
    ref = oracle_sigma(L, w.grid, T, P, w.cut)
    H = hk.HostLines.from_host(L)
    o32 = hk.make_opts(QREF, w.cut)
    got = hk.hk_cross_section_host(H, grid, st, o32, chunk_lines=1500)
    hk.hk_sync_status()
    assert got.dtype == torch.float32 and not got.is_cuda
    assert_sigma_close(got.numpy(), ref, "host fp32c")
    dev = hk.hk_cross_section(hk.DeviceLines.from_host(L), grid, st, o32)
    hk.hk_sync_status()
    e = sigma_errors(got.numpy(), dev.cpu().numpy())
    assert e["max_bin"] <= 1e-6, e
    for prec, flags in ((hk.HK_FP64, 0), (hk.HK_FP32C, hk.HK_SIGMA_F64)):
        g64 = hk.hk_cross_section_host(H, grid, st, hk.make_opts(QREF, w.cut, prec, flags=flags),
                                       chunk_lines=4096)
        hk.hk_sync_status()
        assert g64.dtype == torch.float64
        assert_sigma_close(g64.numpy(), ref, f"host prec={prec}")
    perm = np.random.default_rng(5).permutation(L.n)
    U = L.subset(perm)
    U.sorted = False
    gu = hk.hk_cross_section_host(hk.HostLines.from_host(U, pin=False), grid, st,
                                  hk.make_opts(QREF, w.cut, flags=hk.HK_SIGMA_F64),
                                  chunk_lines=3000)
    hk.hk_sync_status()
    assert_sigma_close(gu.numpy(), ref, "host unsorted pageable")
    gd = hk.hk_cross_section_host(H, grid, st, o32)          # default block size
    hk.hk_sync_status()
    assert_sigma_close(gd.numpy(), ref, "host default chunk")
    E = hk.HostLines.from_host(synth.make_lines(0, 0, 10, 1, 18.0))
    ge = hk.hk_cross_section_host(E, grid, st, o32)
    hk.hk_sync_status()
    assert np.all(ge.numpy() == 0)


def _oracle_ext(L, grid, T, P, cut, cut_mode, plinth):
    return oracle.cross_section(L.as_oracle(), grid.astuple(), (T, P, float(Q(T)), QREF), cut,
                                cut_mode=cut_mode, plinth=plinth)


@pytest.mark.parametrize("prec", [0, 1])
def test_plinth_and_per_line_cuts(hk, prec):
    """Doppler- and Lorentz-multiple cuts (Sect. 2.4.3 item 4) and plinth
    removal (Sect. 2.1) on the config-0 list: pair totals equal the oracle's,
    the same zero pattern, and parity.  With the plinth removed a bin near a
    cut edge is a difference of two nearly equal values: the bar is taken
    relative to the terms summed (the un-removed sigma), and relative to the
    removed value itself where the difference is well conditioned
    (assert_plinth_close)."""
    w = synth.config(0, scale=0.3)
    L = w.species[0]
    T, P = 1000.0, 1.0
    grid = w.grid
    D = hk.DeviceLines.from_host(L)
    st = hk.make_state(T, P, float(Q(T)))
    cases = [(hk.HK_CUT_FIXED, 25.0, True), (hk.HK_CUT_DOPPLER, 500.0, False),
             (hk.HK_CUT_DOPPLER, 500.0, True), (hk.HK_CUT_LORENTZ, 150.0, False),
             (hk.HK_CUT_LORENTZ, 150.0, True)]
    for mode, cut, plinth in cases:
        flags = (hk.HK_REMOVE_PLINTH if plinth else 0) | hk.HK_SIGMA_F64
        opts = hk.make_opts(QREF, cut, prec, cut_mode=mode, flags=flags)
        got = hk.hk_cross_section(D, hk.make_grid(*grid.astuple()), st, opts)
        hk.hk_sync_status()
        got = got.cpu().numpy()
        ref = _oracle_ext(L, grid, T, P, cut, mode, plinth)
        what = f"mode={mode} cut={cut} plinth={plinth} prec={prec}"
        if mode != hk.HK_CUT_FIXED:
            GLo = oracle.widths(L.nu0, L.gamma_ref, L.n_T, T, P, L.mass_amu)[1]
            cl = oracle.line_cuts(L.nu0, GLo, mode, cut, T, L.mass_amu)
            pairs = hk.hk_count_pairs(D, hk.make_grid(*grid.astuple()), st, opts)[0]
            assert pairs == oracle.count_pairs_percut(L.nu0, cl, *grid.astuple()), what
        # bins outside every cut are exactly zero on both sides (with the plinth
        # removed an edge bin may also round to zero in FP32)
        assert np.all(got[ref == 0] == 0) and (plinth or np.all(ref[got == 0] == 0)), what
        if not plinth:
            assert_sigma_close(got, ref, what)
            continue
        base = _oracle_ext(L, grid, T, P, cut, mode, False)
        assert_plinth_close(got, ref, base, what)


@pytest.mark.parametrize("prec", [0, 1])
def test_line_profiles(hk, prec):
    """Lorentzian, Doppler and binned-Gaussian profiles (Sect. 2.1) on the
    config-0 list, with and without the plinth and with a Doppler-multiple
    cut, against the oracle (same bars as test_plinth_and_per_line_cuts)."""
    w = synth.config(0, scale=0.3)
    L = w.species[0]
    T, P = 1000.0, 1.0
    grid = w.grid
    D = hk.DeviceLines.from_host(L)
    st = hk.make_state(T, P, float(Q(T)))
    cases = []
    for prof in (hk.HK_PROFILE_LORENTZ, hk.HK_PROFILE_DOPPLER, hk.HK_PROFILE_BINNED_GAUSS):
        cases += [(prof, hk.HK_CUT_FIXED, 25.0, False), (prof, hk.HK_CUT_FIXED, 25.0, True)]
    cases += [(hk.HK_PROFILE_DOPPLER, hk.HK_CUT_DOPPLER, 40.0, True)]
    for prof, mode, cut, plinth in cases:
        flags = (hk.HK_REMOVE_PLINTH if plinth else 0) | hk.HK_SIGMA_F64
        opts = hk.make_opts(QREF, cut, prec, cut_mode=mode, flags=flags, profile=prof)
        got = hk.hk_cross_section(D, hk.make_grid(*grid.astuple()), st, opts)
        hk.hk_sync_status()
        got = got.cpu().numpy()
        args = (L.as_oracle(), grid.astuple(), (T, P, float(Q(T)), QREF), cut)
        ref = oracle.cross_section(*args, cut_mode=mode, plinth=plinth, profile=prof)
        what = f"profile={prof} mode={mode} plinth={plinth} prec={prec}"
        # outside every cut zero; far tails (exp(-x^2) ~ 1e-300) may underflow on one
        # side only, far below the mask
        assert np.all(np.isfinite(got)), what
        assert np.all(np.abs(got[ref == 0]) <= 1e-14 * ref.max()), what
        if not plinth:
            assert_sigma_close(got, ref, what)
            continue
        base = oracle.cross_section(*args, cut_mode=mode, plinth=False, profile=prof)
        assert_plinth_close(got, ref, base, what)


def test_wide_lines_whole_tiles(hk):
    """Lines 20001 bins wide (and uncut) on a grid of ~100 tiles, so that
    most tiles lie wholly inside one one-node segment of a line (the peeled
    instance's one-pass tiles), next to tiles holding a line's edge groups,
    its centre, and the grid's ragged end: Voigt, Voigt with the plinth, the
    Lorentzian (one-node everywhere) with and without the plinth, and no cut,
    in FP32C against the oracle."""
    L = synth.make_lines(300, 0.0, 1000.0, synth.SEED_BASE + 11, 18.0)
    grid = synth.Grid(0.0, 0.01, 100003)
    T, P = 1000.0, 1.0
    D = hk.DeviceLines.from_host(L)
    st = hk.make_state(T, P, float(Q(T)))
    V, LZ = hk.HK_PROFILE_VOIGT, hk.HK_PROFILE_LORENTZ
    cases = [(V, hk.HK_CUT_FIXED, 100.0, False), (V, hk.HK_CUT_FIXED, 100.0, True),
             (LZ, hk.HK_CUT_FIXED, 100.0, False), (LZ, hk.HK_CUT_FIXED, 100.0, True),
             (V, hk.HK_CUT_NONE, 0.0, False)]
    for prof, mode, cut, plinth in cases:
        flags = (hk.HK_REMOVE_PLINTH if plinth else 0) | hk.HK_SIGMA_F64
        opts = hk.make_opts(QREF, cut, hk.HK_FP32C, cut_mode=mode, flags=flags, profile=prof)
        got = hk.hk_cross_section(D, hk.make_grid(*grid.astuple()), st, opts)
        hk.hk_sync_status()
        got = got.cpu().numpy()
        args = (L.as_oracle(), grid.astuple(), (T, P, float(Q(T)), QREF), cut)
        ref = oracle.cross_section(*args, cut_mode=mode, plinth=plinth, profile=prof)
        what = f"profile={prof} mode={mode} cut={cut} plinth={plinth}"
        assert np.all(np.isfinite(got)), what
        assert np.all(got[ref == 0] == 0), what
        if not plinth:
            assert_sigma_close(got, ref, what)
            continue
        base = oracle.cross_section(*args, cut_mode=mode, plinth=False, profile=prof)
        assert_plinth_close(got, ref, base, what)


@pytest.mark.parametrize("prec", [0, 1])
def test_hitran_widths_and_pressure_shift(hk, prec):
    """HITRAN air/self widths (Eq. gammaL) and pressure-shifted positions on a
    config-0-shaped list: device-resident (sorted and unsorted) and streamed
    from host memory, against the oracle; pair totals on the shifted
    positions equal the oracle's."""
    L = synth.make_lines(3000, 0.0, 3000.0, synth.SEED_BASE + 7, 18.0, hitran=True)
    grid = synth.Grid(0.0, 0.1, 30000)
    T, P, Ps, cut = 900.0, 3.0, 0.8, 25.0
    ref = oracle.cross_section(L.as_oracle(), grid.astuple(), (T, P, float(Q(T)), QREF), cut,
                               P_self=Ps)
    st = hk.make_state(T, P, float(Q(T)), P_self=Ps)
    g = hk.make_grid(*grid.astuple())
    opts = hk.make_opts(QREF, cut, prec, flags=hk.HK_SIGMA_F64)
    D = hk.DeviceLines.from_host(L)
    pos = oracle.shift(L.nu0, L.delta, P)
    assert hk.hk_count_pairs(D, g, st, opts)[0] == oracle.count_pairs(pos, *grid.astuple(), cut)
    got = hk.hk_cross_section(D, g, st, opts)
    hk.hk_sync_status()
    assert_sigma_close(got.cpu().numpy(), ref, f"hitran prec={prec}")
    perm = np.random.default_rng(9).permutation(L.n)
    U = L.subset(perm)
    U.sorted = False
    got = hk.hk_cross_section(hk.DeviceLines.from_host(U), g, st, opts)
    hk.hk_sync_status()
    assert_sigma_close(got.cpu().numpy(), ref, f"hitran unsorted prec={prec}")
    got = hk.hk_cross_section_host(hk.HostLines.from_host(L), g, st, opts, chunk_lines=700)
    hk.hk_sync_status()
    assert_sigma_close(got.numpy(), ref, f"hitran host prec={prec}")


def test_batched_with_profiles_plinth_and_per_line_cuts(hk):
    """The batched launch with a non-Voigt profile, the plinth and a per-line
    cut: every (species, T, P) array equals the single-problem call on the
    same options (same kernels, one launch), and one array against the
    oracle."""
    w = synth.config(3, scale=1e-4)
    grid = synth.Grid(0.0, 0.01, 100000)
    species = [hk.DeviceLines.from_host(s_) for s_ in w.species]
    pts = [(float(t), float(p)) for t in w.T[::10] for p in w.P[::5]]
    states = [hk.make_state(t, p, float(Q(t))) for t, p in pts]
    g = hk.make_grid(*grid.astuple())
    for prof, mode, cut in [(hk.HK_PROFILE_DOPPLER, hk.HK_CUT_DOPPLER, 400.0),
                            (hk.HK_PROFILE_VOIGT, hk.HK_CUT_LORENTZ, 300.0)]:
        opts = hk.make_opts(QREF, cut, cut_mode=mode, profile=prof,
                            flags=hk.HK_SIGMA_F64 | hk.HK_REMOVE_PLINTH)
        out = hk.hk_cross_section_batched(species, states, g, opts)
        hk.hk_sync_status()
        out = out.cpu().numpy()
        for si, D in enumerate(species):
            for k, st in enumerate(states):
                one = hk.hk_cross_section(D, g, st, opts)
                hk.hk_sync_status()
                e = sigma_errors(out[si, k], one.cpu().numpy())
                assert e["max_bin"] <= 1e-6, (prof, si, k, e)
        t, p = pts[-1]
        L = w.species[-1]
        ref = oracle.cross_section(L.as_oracle(), grid.astuple(), (t, p, float(Q(t)), QREF), cut,
                                   cut_mode=mode, plinth=True, profile=prof)
        base = oracle.cross_section(L.as_oracle(), grid.astuple(), (t, p, float(Q(t)), QREF), cut,
                                    cut_mode=mode, plinth=False, profile=prof)
        assert_plinth_close(out[-1, -1], ref, base, f"batched profile={prof}")


def test_backward_rejects_plinth_and_per_line_cuts(hk):
    L = synth.make_lines(50, 0.0, 10.0, 3, 18.0)
    D = hk.DeviceLines.from_host(L)
    grid = hk.make_grid(0.0, 0.01, 1000)
    g = torch.zeros((1, 1000), dtype=torch.float32, device="cuda")
    st = [hk.make_state(500.0, 1.0, float(Q(500.0)), float(synth.dlnQ_dT(500.0)))]
    for opts in (hk.make_opts(QREF, 5.0, cut_mode=hk.HK_CUT_DOPPLER),
                 hk.make_opts(QREF, 2.0, flags=hk.HK_REMOVE_PLINTH),
                 hk.make_opts(QREF, 2.0, profile=hk.HK_PROFILE_LORENTZ)):
        with pytest.raises(hk.HKError) as e:
            hk.hk_cross_section_backward(D, grid, st, opts, g)
        assert e.value.status == hk.HK_ENOTSUP
    H = hk.DeviceLines.from_host(synth.make_lines(50, 0.0, 10.0, 3, 18.0, hitran=True))
    with pytest.raises(hk.HKError) as e:
        hk.hk_cross_section_backward(H, grid, st, hk.make_opts(QREF, 2.0), g)
    assert e.value.status == hk.HK_ENOTSUP


def test_pool_limit_gives_enomem_and_recovers(hk, monkeypatch):
    """Host-side allocation failure: with the scratch pool released and its
    limit (HK_POOL_LIMIT_MB) below what a call needs, the call returns
    HK_ENOMEM before any device work; with the limit lifted the same call
    succeeds and matches the oracle (the context stays usable)."""
    w = synth.config(0, scale=0.1)
    L = w.species[0]
    T, P = w.states()[0]
    D = hk.DeviceLines.from_host(L)
    grid = hk.make_grid(*w.grid.astuple())
    st = hk.make_state(T, P, float(Q(T)))
    opts = hk.make_opts(QREF, w.cut)
    torch.cuda.synchronize()
    hk.hk_release()
    monkeypatch.setenv("HK_POOL_LIMIT_MB", "0.001")
    with pytest.raises(hk.HKError) as ei:
        hk.hk_cross_section(D, grid, st, opts)
    assert ei.value.status == hk.HK_ENOMEM
    monkeypatch.delenv("HK_POOL_LIMIT_MB")
    got = hk.hk_cross_section(D, grid, st, opts)
    hk.hk_sync_status()
    assert_sigma_close(got.cpu().numpy(), oracle_sigma(L, w.grid, T, P, w.cut), "after ENOMEM")


def test_zero_lines_and_single_line(hk):
    L0 = synth.make_lines(0, 0, 10, 1, 18.0)
    grid = synth.Grid(0.0, 0.01, 1000)
    got = gpu_sigma(hk, L0, grid, 500.0, 1.0, 1.0, 0)
    assert np.all(got == 0)
    L1 = synth.make_lines(1, 4.0, 6.0, 2, 18.0)
    ref = oracle_sigma(L1, grid, 500.0, 1.0, 1.0)
    for prec in (0, 1):
        assert_sigma_close(gpu_sigma(hk, L1, grid, 500.0, 1.0, 1.0, prec), ref, f"1 line {prec}")


def test_unsorted_input_matches_oracle(hk):
    L = synth.make_lines(3000, 0.0, 300.0, 5, 18.0, sort=False)
    grid = synth.Grid(0.0, 0.05, 6000)
    ref = oracle_sigma(L, grid, 1200.0, 2.0, 5.0)
    assert_sigma_close(gpu_sigma(hk, L, grid, 1200.0, 2.0, 5.0, 0), ref, "unsorted")


def test_einstein_A_mode_per_gram(hk):
    rng = np.random.default_rng(3)
    L = synth.make_lines(2000, 100.0, 400.0, 9, 56.0, A_range=(1e6, 1e9))
    L.g_up = rng.integers(1, 20, L.n).astype(np.float32)
    L.s_mode = 1
    grid = synth.Grid(100.0, 0.02, 15000)
    ref = oracle_sigma(L, grid, 2500.0, 0.1, 10.0, per_gram=True)
    for prec in (0, 1):
        got = gpu_sigma(hk, L, grid, 2500.0, 0.1, 10.0, prec, flags=1)
        assert_sigma_close(got, ref, f"A-mode prec={prec}")


def test_float_overflow_reports_erange_and_double_output_is_exact(hk):
    """One line of large E'' at high T: S(T) ~ 1e56, sigma beyond the float
    range.  Float output must be reported (HK_ERANGE), double output must match."""
    L = synth.make_lines(3, 10.0, 20.0, 8, 18.0)
    L.E_low[:] = np.float32(60000.0)
    L.S_ref[:] = np.float32(1e-19)
    grid = synth.Grid(0.0, 0.01, 3000)
    T, P, cut = 2500.0, 1.0, 5.0
    D = hk.DeviceLines.from_host(L)
    args = (hk.make_grid(*grid.astuple()), hk.make_state(T, P, float(Q(T))))
    hk.hk_sync_status()
    hk.hk_cross_section(D, *args, hk.make_opts(QREF, cut))
    with pytest.raises(hk.HKError) as ei:
        hk.hk_sync_status()
    assert ei.value.status == hk.HK_ERANGE
    hk.hk_sync_status()                                  # the status word was cleared
    s = hk.hk_cross_section(D, *args, hk.make_opts(QREF, cut, flags=hk.HK_SIGMA_F64))
    hk.hk_sync_status()
    ref = oracle_sigma(L, grid, T, P, cut)
    assert ref.max() > 1e45
    assert_sigma_close(s.cpu().numpy(), ref, "double output of FP32C")


def test_line_strength_and_widths(hk):
    L = synth.config(0).species[0]
    D = hk.DeviceLines.from_host(L)
    T, P = 1777.0, 0.37
    st = hk.make_state(T, P, float(Q(T)))
    op = hk.make_opts(QREF, 25.0)
    S = hk.hk_line_strength(D, st, op).cpu().numpy()
    aDinv, y = (t.cpu().numpy() for t in hk.hk_widths(D, st, op))
    So = oracle.line_strength(L.nu0, L.E_low, T, float(Q(T)), QREF, 18.0, S_ref=L.S_ref)
    aD, GL = oracle.widths(L.nu0, L.gamma_ref, L.n_T, T, P, 18.0)
    m = So > 1e-300
    assert np.allclose(S[m], So[m], rtol=1e-11, atol=0)
    assert np.allclose(aDinv, 1 / aD, rtol=2e-7)
    assert np.allclose(y, GL / aD, rtol=2e-7)


@pytest.mark.parametrize("prec", [0, 1])
def test_voigt_accumulate_adds(hk, prec):
    L = synth.make_lines(1500, 0.0, 150.0, 21, 18.0)
    grid = synth.Grid(0.0, 0.01, 15000)
    T, P, cut = 900.0, 0.5, 3.0
    S = oracle.line_strength(L.nu0, L.E_low, T, float(Q(T)), QREF, 18.0, S_ref=L.S_ref)
    aD, GL = oracle.widths(L.nu0, L.gamma_ref, L.n_T, T, P, 18.0)
    ref = oracle.sigma(L.nu0, S, aD, GL, *grid.astuple(), cut)
    dt = torch.float64 if prec else torch.float32
    # a non-zero starting sigma of the same magnitude (so the float difference
    # after - before is well conditioned)
    start_np = 0.37 * ref
    start_np[::7] = 0.0
    base = torch.from_numpy(start_np).to(dt).cuda()
    start = base.clone()
    hk.hk_voigt_accumulate(torch.from_numpy(L.nu0).cuda(), torch.from_numpy(S).cuda(),
                           torch.from_numpy((1 / aD).astype(np.float32)).cuda(),
                           torch.from_numpy((GL / aD).astype(np.float32)).cuda(),
                           hk.make_grid(*grid.astuple()), cut, base, prec)
    hk.hk_sync_status()
    got = (base - start).cpu().numpy().astype(np.float64)
    assert_sigma_close(got, ref, "voigt_accumulate")


def test_config1_shape_windows(hk):
    """Config 1 shape (log-normal density, 0.1 grid, cut 25, 1500 K) at 1/100 of
    its line count: whole array on the GPU, windows (dense, sparse, edges) on
    the oracle."""
    w = synth.config(1, scale=1e-2)
    L = w.species[0]
    T, P = w.states()[0]
    D = hk.DeviceLines.from_host(L)
    # at 1500 K lines of large E'' reach S(T) ~ 1e40: sigma needs double output
    got = hk.hk_cross_section(D, hk.make_grid(*w.grid.astuple()),
                              hk.make_state(T, P, float(Q(T))),
                              hk.make_opts(QREF, w.cut, flags=hk.HK_SIGMA_F64))
    hk.hk_sync_status()
    got = got.cpu().numpy().astype(np.float64)
    counts = synth.lognormal_window_counts(L.n, 300, synth.SEED_BASE + 1)
    dense = int(np.argmax(counts))
    sparse = int(np.argmin(counts))
    gmax = oracle_sigma_max(oracle, L, w.grid.astuple(), (T, P, float(Q(T)), QREF), w.cut)
    assert gmax <= got.max() * (1 + 1e-4)
    for lo in [0, dense * 1000 + 300, sparse * 1000 + 300, w.grid.nbins - 1500]:
        hi = lo + 1500
        ref = oracle_sigma(L, w.grid, T, P, w.cut, lo, hi)
        assert_sigma_close(got[lo:hi], ref, f"c1/100 window {lo}", ref_max=gmax)


def test_batched_matches_single(hk):
    """Config 3 shape at reduced line counts; every (species, T, P) array of the
    batched launch against the oracle on two windows."""
    w = synth.config(3, scale=2e-4)
    grid = synth.Grid(0.0, 0.01, 200000)          # 0-2000 cm^-1 slice of the grid
    species = [hk.DeviceLines.from_host(s) for s in w.species]
    Ts = w.T[::6]
    Ps = w.P[::3]
    states = [hk.make_state(t, p, float(Q(t))) for t in Ts for p in Ps]
    out = hk.hk_cross_section_batched(species, states, hk.make_grid(*grid.astuple()),
                                      hk.make_opts(QREF, w.cut, flags=hk.HK_SIGMA_F64))
    hk.hk_sync_status()
    out = out.cpu().numpy()
    k = 0
    for t in Ts:
        for p in Ps:
            for s, L in enumerate(w.species):
                gmax = oracle_sigma_max(oracle, L, grid.astuple(), (t, p, float(Q(t)), QREF), w.cut)
                for lo in (1000, 150000):
                    ref = oracle_sigma(L, grid, t, p, w.cut, lo, lo + 400)
                    assert_sigma_close(out[s, k, lo:lo + 400], ref,
                                       f"batched s={s} T={t:.0f} P={p:.1e}", ref_max=gmax)
            k += 1


def test_backward_matches_oracle_gradient(hk):
    """Config 4 shape (cut 25, 0.01 grid, paired T-P points) at reduced size."""
    rng = np.random.default_rng(44)
    L = synth.make_lines(300, 0.0, 100.0, synth.SEED_BASE + 4, 18.0)
    grid = synth.Grid(0.0, 0.01, 10000)
    Ts = np.array([300.0, 800.0, 2500.0])
    Ps = np.array([1e-3, 0.3, 10.0])
    cut = 25.0
    g = rng.standard_normal((3, grid.nbins)).astype(np.float32)
    D = hk.DeviceLines.from_host(L)
    states = [hk.make_state(t, p, float(Q(t)), float(synth.dlnQ_dT(t))) for t, p in zip(Ts, Ps)]
    dT, dP, dS, dG = hk.hk_cross_section_backward(D, hk.make_grid(*grid.astuple()), states,
                                                  hk.make_opts(QREF, cut),
                                                  torch.from_numpy(g).cuda())
    hk.hk_sync_status()
    dT, dP, dS, dG = (x.cpu().numpy() for x in (dT, dP, dS, dG))
    oS = np.zeros(L.n)
    oG = np.zeros(L.n)
    for k, (t, p) in enumerate(zip(Ts, Ps)):
        _, _, oT, oP = oracle.backward(L.as_oracle(), grid.astuple(),
                                       (t, p, float(Q(t)), QREF, float(synth.dlnQ_dT(t))), cut,
                                       g[k].astype(np.float64), oS, oG)
        assert abs(dT[k] - oT) <= 1e-4 * abs(oT), (k, dT[k], oT)
        assert abs(dP[k] - oP) <= 1e-4 * abs(oP), (k, dP[k], oP)
    assert np.linalg.norm(dS - oS) <= 1e-4 * np.linalg.norm(oS)
    assert np.linalg.norm(dG - oG) <= 1e-4 * np.linalg.norm(oG)


def test_batched_graph_capture_replay(hk):
    """The batched call is a plain sequence of kernel launches and memsets:
    captured once into a CUDA graph and replayed, it gives the direct result."""
    w = synth.config(3, scale=1e-4)
    grid = hk.make_grid(0.0, 0.01, 100000)
    species = [hk.DeviceLines.from_host(s) for s in w.species]
    states = [hk.make_state(t, p, float(Q(t))) for t in w.T[::10] for p in w.P[::5]]
    opts = hk.make_opts(QREF, w.cut, flags=hk.HK_SIGMA_F64)
    need = hk.hk_workspace_size(0, species, len(states), grid, opts)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    out = torch.empty((len(species), len(states), grid.nbins), dtype=torch.float64, device="cuda")
    direct = hk.hk_cross_section_batched(species, states, grid, opts, out, ws).clone()
    hk.hk_sync_status()
    out.zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            hk.hk_cross_section_batched(species, states, grid, opts, out, ws, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(2):
        out.zero_()
        g.replay()
    torch.cuda.synchronize()
    a, b = out.cpu().numpy(), direct.cpu().numpy()
    assert np.allclose(a, b, rtol=1e-12, atol=0)
    assert np.count_nonzero(a) > 0.5 * a.size


def test_autotune_keeps_results(hk):
    L = synth.config(1, scale=2e-4).species[0]
    w = synth.config(1, scale=2e-4)
    D = hk.DeviceLines.from_host(L)
    T, P = w.states()[0]
    args = (D, hk.make_grid(*w.grid.astuple()), hk.make_state(T, P, float(Q(T))),
            hk.make_opts(QREF, w.cut, flags=hk.HK_SIGMA_F64))
    before = hk.hk_cross_section(*args).cpu().numpy()
    hk.hk_autotune(*args)
    lmax, tile = hk.hk_tuning_full(hk.HK_FP32C)
    assert lmax in (1024, 2048, 4096, 16384, 65536) and tile in (1024, 2048)
    after = hk.hk_cross_section(*args).cpu().numpy()
    hk.hk_sync_status()
    assert_sigma_close(after, before, "after autotune")
    hk.hk_set_tuning(hk.HK_FP32C, 2048, 1024)


@pytest.mark.parametrize("tile", [1024, 2048])
def test_tile_widths_match_oracle(hk, tile):
    """Both tile widths the autotuner chooses from, for short lines (501 bins,
    tiles with a halo) and wide ones (2001 bins, peeled sweeps), at two
    lines-per-item settings: parity with the oracle."""
    try:
        for lmax in (1024, 65536):
            hk.hk_set_tuning(hk.HK_FP32C, lmax, tile)
            for cut in (25.0, 100.0):
                L = synth.make_lines(6000, 0.0, 800.0, 93, 18.0, windows=8)
                grid = synth.Grid(0.0, 0.05 if cut > 50 else 0.1, 16000 if cut > 50 else 8000)
                ref = oracle_sigma(L, grid, 1200.0, 0.7, cut)
                got = gpu_sigma(hk, L, grid, 1200.0, 0.7, cut, 0, flags=hk.HK_SIGMA_F64)
                assert_sigma_close(got, ref, f"tile {tile} lmax {lmax} cut {cut}")
                assert np.array_equal(ref == 0, got == 0)
    finally:
        hk.hk_set_tuning(hk.HK_FP32C, 2048, 1024)


def test_dense_line_batches(hk):
    """Short lines (cut 25 at 0.1 cm^-1: 501 bins) in clusters that share a
    nearest bin, so consecutive lines form batches with one group structure
    (the multi-line sweep), mixed with clusters that straddle a half-bin (two
    nearest bins in one batch: per-line path), lines so narrow in Doppler
    width that no bin is in their four-node band, lines near the tile edges
    (1024-bin tiles), and a ragged last cluster; FP32C against the oracle,
    with the oracle's zero pattern; also lines a hair either side of the
    half-bins where the halo tiles' ownership changes."""
    rng = np.random.default_rng(2101)
    dnu, nbins = 0.1, 12000
    centres = np.sort(rng.uniform(40.0, 1160.0, 420))
    nu0 = []
    for i, c in enumerate(centres):
        k = int(round(c / dnu))
        if i % 7 == 3:                       # a half-bin straddled inside the cluster
            base = (k + 0.5) * dnu
            offs = np.linspace(-3e-3, 3e-3, 9)
        elif i % 11 == 5:                    # on a tile edge
            base = (1024 * (1 + i % 10)) * dnu
            offs = rng.uniform(-1e-3, 1e-3, 12)
        elif i % 13 == 6:                    # where tile ownership changes (a half-bin
            base = (512 * (1 + i % 20) - 0.5) * dnu   # before a multiple of 512 bins)
            offs = np.linspace(-2e-9, 2e-9, 8)
        else:                                # one shared nearest bin
            base = k * dnu + rng.uniform(-0.04, 0.04)
            offs = rng.uniform(-2e-3, 2e-3, int(rng.integers(4, 17)))
        nu0.extend((base + np.sort(offs)).tolist())
    nu0 = np.sort(np.asarray(nu0))
    n = nu0.size
    gam = rng.uniform(0.01, 0.1, n).astype(np.float32)
    gam[rng.uniform(size=n) < 0.05] = 40.0   # y >> 50: no four-node band, all two-node
    L = synth.LineList(nu0, (10 ** rng.uniform(-24, -20, n)).astype(np.float32),
                       rng.exponential(1500.0, n).astype(np.float32), gam,
                       rng.uniform(0.3, 0.8, n).astype(np.float32), 18.0)
    grid = synth.Grid(0.0, dnu, nbins)
    for T, P in [(1500.0, 1.0), (300.0, 0.05)]:
        ref = oracle_sigma(L, grid, T, P, 25.0)
        got = gpu_sigma(hk, L, grid, T, P, 25.0, 0, flags=hk.HK_SIGMA_F64)
        assert_sigma_close(got, ref, f"dense batches T={T}")
        assert np.array_equal(ref == 0, got == 0), T


@pytest.mark.parametrize("cut", [1.5, 15.0])
def test_voigt_bands_per_pair_accuracy(hk, cut):
    """Per-pair accuracy of the FP32 Faddeeva evaluation, through
    hk_voigt_accumulate: clusters of four identical lines (one batch), each
    cluster alone on its bins, with alpha_D and y chosen so that the bins sweep
    every band (the core r2 < 64 down to y = 1e-6, the four-, two- and
    one-node bands out to r2 ~ 1e10); cut 1.5 takes the short-line instance,
    cut 15 the wide-line one.  Every bin above 1e-15 of the peak against the
    oracle's FP64 value on the same float inputs: FP32C at most 1e-5 relative
    (the Gaussian tail inherits 2 x^2 times the relative rounding of x),
    median below 1e-6; the FP64 GPU form (same bands) at most 3e-6.""" 
    dnu = 0.01
    spacing = 2.0 * cut + 1.0
    params = [(y, a) for y in [1e-6, 1e-3, 0.05, 0.5, 2.0, 7.0, 40.0]
              for a in [0.1, 0.02, 0.003, 1e-4]]
    k = np.arange(len(params))
    centre = spacing * (k + 1) + 0.00371 * k                  # off-bin centres
    nu0 = np.repeat(centre, 4)
    aDinv = np.repeat(np.array([1.0 / a for _, a in params], np.float32), 4)
    yv = np.repeat(np.array([y for y, _ in params], np.float32), 4)
    S = np.full(nu0.size, 1e-20)
    aD = 1.0 / aDinv.astype(np.float64)                        # the kernel's inputs, exactly
    GL = yv.astype(np.float64) * aD
    nbins = int(round(spacing * (len(params) + 1) / dnu))
    grid = synth.Grid(0.0, dnu, nbins)
    ref = oracle.sigma(nu0, S, aD, GL, *grid.astuple(), cut)
    out = torch.zeros(nbins, dtype=torch.float64, device="cuda")
    hk.hk_voigt_accumulate(torch.from_numpy(nu0).cuda(), torch.from_numpy(S).cuda(),
                           torch.from_numpy(aDinv).cuda(), torch.from_numpy(yv).cuda(),
                           hk.make_grid(*grid.astuple()), cut, out, hk.HK_FP64)
    hk.hk_sync_status()
    out32 = torch.zeros(nbins, dtype=torch.float32, device="cuda")
    hk.hk_voigt_accumulate(torch.from_numpy(nu0).cuda(), torch.from_numpy(S).cuda(),
                           torch.from_numpy(aDinv).cuda(), torch.from_numpy(yv).cuda(),
                           hk.make_grid(*grid.astuple()), cut, out32, hk.HK_FP32C)
    hk.hk_sync_status()
    m = ref > 1e-15 * ref.max()
    # both GPU forms use the same truncated bands (~1e-6 by design); FP32C adds
    # its rounding
    for name, got, tol_max, tol_med in [("fp64", out.cpu().numpy(), 3e-6, 1e-6),
                                        ("fp32c", out32.cpu().numpy().astype(np.float64), 1e-5,
                                         1e-6)]:
        rel = np.abs(got[m] - ref[m]) / ref[m]
        i = int(np.argmax(rel))
        assert rel.max() <= tol_max and np.median(rel) <= tol_med, (
            name, cut, float(rel.max()), float(np.median(rel)), int(np.flatnonzero(m)[i]))
    assert np.array_equal(ref == 0, out32.cpu().numpy() == 0)


def test_dense_wide_lines(hk):
    """Dense wide lines (cut 25 at 0.01 cm^-1: 5001 bins, the peeled instance)
    in clusters, so that batches of lines dealt 8 apart still lie within a
    few groups of each other: tiles in one band for every line (one-node
    runs from the tile origin, shared reciprocals), tiles across lines'
    one-/two-node boundaries (the two-node rule for every line), tiles where
    lines start or end (masked two-node spans), tiles with lines' four-node
    and core groups (line by line), and lines with y >> 50 (no four-node
    band).  Voigt and Lorentzian, with and without the plinth, at two (T, P)
    points; FP32C against the oracle over the whole array."""
    rng = np.random.default_rng(2102)
    dnu, nbins = 0.01, 40000
    centres = np.sort(rng.uniform(30.0, 370.0, 60))
    nu0 = np.sort(np.concatenate([c + rng.uniform(-0.05, 0.05, int(rng.integers(20, 80)))
                                  for c in centres]))
    n = nu0.size
    gam = rng.uniform(0.01, 0.1, n).astype(np.float32)
    gam[rng.uniform(size=n) < 0.05] = 40.0
    L = synth.LineList(nu0, (10 ** rng.uniform(-24, -20, n)).astype(np.float32),
                       rng.exponential(1500.0, n).astype(np.float32), gam,
                       rng.uniform(0.3, 0.8, n).astype(np.float32), 18.0)
    grid = synth.Grid(0.0, dnu, nbins)
    D = hk.DeviceLines.from_host(L)
    g = hk.make_grid(*grid.astuple())
    V, LZ = hk.HK_PROFILE_VOIGT, hk.HK_PROFILE_LORENTZ
    for T, P in [(1000.0, 1.0), (300.0, 20.0)]:
        st = hk.make_state(T, P, float(Q(T)))
        args = (L.as_oracle(), grid.astuple(), (T, P, float(Q(T)), QREF), 25.0)
        base = {}
        for prof in (V, LZ):
            for plinth in (False, True):
                flags = (hk.HK_REMOVE_PLINTH if plinth else 0) | hk.HK_SIGMA_F64
                opts = hk.make_opts(QREF, 25.0, hk.HK_FP32C, flags=flags, profile=prof)
                got = hk.hk_cross_section(D, g, st, opts)
                hk.hk_sync_status()
                got = got.cpu().numpy()
                ref = oracle.cross_section(*args, plinth=plinth, profile=prof)
                what = f"dense wide profile={prof} plinth={plinth} T={T} P={P}"
                assert np.all(got[ref == 0] == 0), what
                if not plinth:
                    base[prof] = ref
                    record(what, assert_sigma_close(got, ref, what))
                else:
                    record(what, assert_plinth_close(got, ref, base[prof], what))


def test_ring_pair_count(hk):
    """hk_count_ring_pairs (instrumentation for the cost model): on the
    config-0 list (short lines, cut 25 at 0.1 cm^-1) the pairs with
    R8(y) <= r2 < 64, R8 = max(26, ln(1.13e9 / y)) at most 64, against a count
    from the oracle's widths and the exact cut range (a few edge pairs may fall
    either side in float geometry); a subset of the core count; 0 for the FP64
    form and for wide lines."""
    w = synth.config(0)
    L = w.species[0]
    T, P = w.states()[0]
    D = hk.DeviceLines.from_host(L)
    g = hk.make_grid(*w.grid.astuple())
    st = hk.make_state(T, P, float(Q(T)))
    ring = hk.hk_count_ring_pairs(D, g, st, hk.make_opts(QREF, w.cut))
    core = hk.hk_count_pairs(D, g, st, hk.make_opts(QREF, w.cut))[5]
    aD, GL = oracle.widths(L.nu0, L.gamma_ref, L.n_T, T, P, L.mass_amu)
    nu_min, dnu, nbins = w.grid.astuple()
    want = 0
    for l in range(L.n):
        if not (L.nu0[l] > 0.0):
            continue
        y = GL[l] / aD[l]
        R8 = min(64.0, max(26.0, math.log(1.13e9) - math.log(y)))
        i = np.arange(max(0, int((L.nu0[l] - w.cut - nu_min) / dnu) - 2),
                      min(nbins, int((L.nu0[l] + w.cut - nu_min) / dnu) + 3))
        d = nu_min + i * dnu - L.nu0[l]
        r2 = (d / aD[l]) ** 2 + y * y
        want += int(np.count_nonzero((np.abs(d) <= w.cut) & (r2 >= R8) & (r2 < 64.0)))
    assert 0 < ring < core
    assert abs(ring - want) <= 1e-3 * want + 20, (ring, want)
    assert hk.hk_count_ring_pairs(D, g, st, hk.make_opts(QREF, w.cut, hk.HK_FP64)) == 0
    assert hk.hk_count_ring_pairs(D, g, st, hk.make_opts(QREF, 600.0)) == 0   # 12001 bins


@pytest.mark.parametrize("plinth", [False, True])
def test_round_series_parity(hk, plinth):
    """Short lines in dense clusters of 128 lines within 0.02 bins of a bin
    centre, so that whole 32-line rounds share their centre bin and take the
    round series, with Lorentz widths chosen per cluster for each form: y near
    0.4 (four nodes), 1.8 (two nodes, 7 terms), 5 (two nodes, 12 terms) and 21
    (no series), at nu0 ~ 14500 cm^-1 (x step ~1.7 per bin, as at config 1);
    modest strengths and lower-state energies keep the whole array above the
    mask, so every bin is held to the bar.  FP32C against the oracle
    (tests/test_series_rules.py checks on the CPU that each cluster kind meets
    its form's conditions)."""
    L, grid = round_series_case(31 + plinth)
    T, P = 1500.0, 1.0
    flags = hk.HK_SIGMA_F64 | (hk.HK_REMOVE_PLINTH if plinth else 0)
    got = gpu_sigma(hk, L, grid, T, P, 25.0, 0, flags=flags)
    ref = oracle.cross_section(L.as_oracle(), grid.astuple(), (T, P, float(Q(T)), QREF), 25.0,
                               plinth=plinth)
    if plinth:
        raw = oracle_sigma(L, grid, T, P, 25.0)
        assert_plinth_close(got, ref, raw, "round series, plinth")
    else:
        assert_sigma_close(got, ref, "round series")
        m = ref > 1e-10 * ref.max()
        assert m.mean() > 0.5, m.mean()
    assert np.array_equal(ref == 0, got == 0)


def test_wide_round_series_parity(hk):
    """Wide lines (cut 100 at 0.01 cm^-1: 20001 bins) packed ten to a bin, so
    that a round's lines lie within a few bins and its far tiles take the
    wide-line series; Lorentz widths from small to large.  FP32C against the
    oracle over the whole array."""
    rng = np.random.default_rng(41)
    dnu, nu_min, nbins = 0.01, 14900.0, 30000
    n = 6000
    nu0 = np.sort(nu_min + (15000 + rng.uniform(-300, 300, n)) * dnu)
    L = synth.LineList(nu0, (10 ** rng.uniform(-22, -20, n)).astype(np.float32),
                       rng.exponential(300.0, n).astype(np.float32),
                       (10 ** rng.uniform(-3, 0, n)).astype(np.float32),
                       rng.uniform(0.3, 0.8, n).astype(np.float32), 18.0)
    grid = synth.Grid(nu_min, dnu, nbins)
    for T, P in [(1000.0, 0.1), (2000.0, 10.0)]:
        got = gpu_sigma(hk, L, grid, T, P, 100.0, 0, flags=hk.HK_SIGMA_F64)
        ref = oracle_sigma(L, grid, T, P, 100.0)
        assert_sigma_close(got, ref, f"wide round series T={T} P={P}")
        assert np.array_equal(ref == 0, got == 0), (T, P)
