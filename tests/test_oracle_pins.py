"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every check here uses an independent source: mpmath at 40-50 digits, scipy's
wofz (the reference the paper itself compares against, Sect. 2.2.3), special
values of the Faddeeva function, exact rational arithmetic, closed-form
integrals, limits of the Voigt profile, or finite differences.  None of them
re-types the oracle's own formula for the quantity under test.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

mp = pytest.importorskip("mpmath")
sp = pytest.importorskip("scipy.special")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")
SQPI = math.sqrt(math.pi)


def w_mp(x, y, dps=50):
    with mp.workdps(dps):
        z = mp.mpc(x, y)
        return mp.exp(-z * z) * mp.erfc(-1j * z)


# ---------------------------------------------------------------- Faddeeva --

XS = [0.0, 1e-3, 0.3, 0.9, 1.7, 2.5, 3.9, 4.0, 5.5, 6.2, 7.7, 7.99, 8.01, 9.5, 12.0, 30.0,
      141.0, 1e3, 4.2e4, 1e6]
YS = [0.0, 1e-12, 1e-8, 1e-5, 1e-2, 0.2, 1.0, 3.0, 7.99, 8.01, 30.0, 1e3, 1e4]


@pytest.mark.parametrize("y", YS)
def test_faddeeva_vs_mpmath(y):
    xs = np.array(XS)
    w = oracle.faddeeva(xs, y)
    for x, wo in zip(XS, w):
        ref = w_mp(x, y)
        re, im = float(ref.real), float(ref.imag)
        if re > 1e-290:
            assert abs(wo.real - re) <= 3e-13 * re, (x, y, wo, ref)
        assert abs(wo.imag - im) <= 3e-13 * abs(complex(ref)), (x, y, wo, ref)


def test_faddeeva_vs_scipy_wofz():
    rng = np.random.default_rng(7)
    x = np.concatenate([rng.uniform(-12, 12, 20000), 10 ** rng.uniform(-4, 6, 20000)])
    y = np.concatenate([10 ** rng.uniform(-12, 1, 20000), 10 ** rng.uniform(-12, 4, 20000)])
    w = oracle.faddeeva(x, y)
    r = sp.wofz(x + 1j * y)
    m = r.real > 1e-280
    assert np.max(np.abs(w.real - r.real)[m] / r.real[m]) < 1e-12
    assert np.max(np.abs(w.imag - r.imag) / np.abs(r)) < 1e-12


def test_faddeeva_special_values():
    x = np.linspace(-26, 26, 5001)
    w = oracle.faddeeva(x, 0.0)
    assert np.allclose(w.real, np.exp(-x * x), rtol=3e-16, atol=0)  # Re w(x) = exp(-x^2)
    # Im w(x) = 2 D(x) / sqrt(pi), D = Dawson's integral
    assert np.allclose(w.imag, 2 / SQPI * sp.dawsn(x), rtol=1e-13, atol=1e-15)
    y = np.logspace(-10, 4, 300)
    w0 = oracle.faddeeva(0.0, y)
    assert np.allclose(w0.real, sp.erfcx(y), rtol=1e-13, atol=0)  # Re w(iy) = erfcx(y)
    assert np.max(np.abs(w0.imag)) < 1e-15
    xr = np.linspace(0.01, 40, 777)
    for yy in [1e-9, 0.5, 9.0]:
        a = oracle.faddeeva(xr, yy)
        b = oracle.faddeeva(-xr, yy)
        assert np.array_equal(a.real, b.real) and np.array_equal(a.imag, -b.imag)


@pytest.mark.parametrize("y", [1e-3, 0.1, 1.0, 10.0])
def test_faddeeva_area(y):
    """int Re w(x+iy) dx = sqrt(pi) (the Voigt profile is normalised)."""
    X = 2000.0
    n = 800001
    x = np.linspace(-X, X, n)
    h = x[1] - x[0]
    f = oracle.faddeeva(x, y).real
    simpson = h / 3 * (f[0] + f[-1] + 4 * f[1:-1:2].sum() + 2 * f[2:-1:2].sum())
    # tails beyond |x| = X: Re w ~ y / (sqrt(pi) (x^2 + y^2)) (1 + O(1/x^2))
    tail = 2 * (math.pi / 2 - math.atan(X / y)) / SQPI
    assert abs(simpson + tail - SQPI) < 2e-9


@pytest.mark.parametrize("y", [1e-9, 1e-3, 0.7, 5.0, 12.0])
def test_faddeeva_derivative_vs_mpmath(y):
    xs = [0.0, 0.4, 2.2, 5.0, 7.9, 8.1, 15.0, 300.0, 5e4]
    d = oracle.faddeeva_deriv(np.array(xs), y)
    def wz(z):
        return mp.exp(-z * z) * mp.erfc(-1j * z)

    for x, do in zip(xs, d):
        with mp.workdps(50):
            # numerical derivative along x at fixed y equals w'(z) for analytic w
            ref = complex(mp.diff(lambda t: wz(mp.mpc(t, y)), x))
            dre_dy = float(mp.diff(lambda t: wz(mp.mpc(x, t)).real, y)) if y > 1e-6 else None
        assert abs(do - ref) <= 1e-11 * abs(ref) + 1e-300, (x, y, do, ref)
        # d Re w / d y = -Im w' : pins the sign convention used by the adjoint
        if dre_dy is not None:
            assert abs(-do.imag - dre_dy) <= 1e-10 * abs(dre_dy) + 1e-12


# ------------------------------------------------------- constants, S, widths --

def test_constants_are_the_papers():
    g = json.load(open(GOLDEN))
    c = oracle.constants()
    assert c["k_B"] == g["k_B"]["value"]
    assert c["c"] == g["c"]["value"]
    # c2 = h c / k_B with CODATA-2010 h (reading: the paper prints no h)
    assert abs(c["c2"] - 1.4387770) < 2e-7


def _lines(n=64, seed=3):
    rng = np.random.default_rng(seed)
    return dict(nu0=rng.uniform(5, 3000, n), S_ref=10 ** rng.uniform(-30, -19, n),
                E_low=rng.exponential(3000, n), gamma_ref=rng.uniform(0.01, 0.1, n),
                n_T=rng.uniform(0.3, 0.8, n), A=rng.uniform(1e-3, 1e3, n),
                g_up=rng.integers(1, 30, n).astype(float), mass_amu=18.0)


def Q(T):
    return 0.1 * T ** 1.5


def test_strength_at_reference_temperature_is_S_ref():
    L = _lines()
    S = oracle.line_strength(L["nu0"], L["E_low"], 296.0, Q(296.0), Q(296.0), 18.0,
                             S_ref=L["S_ref"])
    assert np.allclose(S, L["S_ref"], rtol=2e-15, atol=0)


def test_strength_modes_agree():
    """S-mode with S_ref taken from A-mode at T_ref reproduces A-mode at any T:
    pins the Boltzmann and stimulated-emission factors of Eq. S/S1."""
    L = _lines()
    Sref = oracle.line_strength(L["nu0"], L["E_low"], 296.0, Q(296.0), Q(296.0), 18.0,
                                A=L["A"], g_up=L["g_up"], s_mode=1)
    for T in [100.0, 700.0, 3000.0]:
        a = oracle.line_strength(L["nu0"], L["E_low"], T, Q(T), Q(296.0), 18.0, A=L["A"],
                                 g_up=L["g_up"], s_mode=1)
        s = oracle.line_strength(L["nu0"], L["E_low"], T, Q(T), Q(296.0), 18.0, S_ref=Sref)
        m = a > 1e-300
        assert np.allclose(s[m], a[m], rtol=1e-12, atol=0)


def test_strength_A_mode_vs_mpmath_eqS():
    """Eq. S of Sect. 2.2.2 evaluated in mpmath with the paper's constants."""
    L = _lines(8)
    T = 1234.0
    cst = oracle.constants()
    S = oracle.line_strength(L["nu0"], L["E_low"], T, Q(T), Q(296.0), 18.0, A=L["A"],
                             g_up=L["g_up"], s_mode=1, per_gram=True)
    with mp.workdps(40):
        hc_k = mp.mpf(cst["h"]) * mp.mpf(cst["c"]) / mp.mpf(cst["k_B"])
        m = mp.mpf(18.0) * mp.mpf(cst["amu"])
        for l in range(8):
            nu = mp.mpf(L["nu0"][l])
            ref = (mp.mpf(L["A"][l]) / (8 * mp.pi * mp.mpf(cst["c"]) * m) * mp.mpf(L["g_up"][l]) /
                   (nu ** 2 * mp.mpf(Q(T))) * mp.exp(-hc_k * mp.mpf(L["E_low"][l]) / T) *
                   (1 - mp.exp(-hc_k * nu / T)))
            assert abs(S[l] - float(ref)) <= 1e-13 * float(ref)


def test_widths():
    L = _lines(16)
    cst = oracle.constants()
    # at T_ref, P_ref: Gamma_L = gamma_ref + A / (4 pi c)
    aD, GL = oracle.widths(L["nu0"], L["gamma_ref"], L["n_T"], 296.0, 1.0, 18.0, A=L["A"])
    assert np.allclose(GL, L["gamma_ref"] + L["A"] / (4 * math.pi * cst["c"]), rtol=1e-15)
    # pressure is linear, temperature exponent n
    _, GL2 = oracle.widths(L["nu0"], L["gamma_ref"], L["n_T"], 592.0, 3.0, 18.0)
    assert np.allclose(GL2, L["gamma_ref"] * 3.0 * 2.0 ** (-L["n_T"]), rtol=1e-14)
    # Doppler HWHM of Eq. gammaD equals sqrt(ln 2) alpha_D (Sect. 2.4.2)
    T = 1500.0
    aD, _ = oracle.widths(L["nu0"], L["gamma_ref"], L["n_T"], T, 1.0, 18.0)
    with mp.workdps(30):
        m = 18 * mp.mpf(cst["amu"])
        for l in range(16):
            GD = mp.mpf(L["nu0"][l]) / mp.mpf(cst["c"]) * mp.sqrt(2 * mp.log(2) * mp.mpf(cst["k_B"]) * T / m)
            assert abs(math.sqrt(math.log(2)) * aD[l] - float(GD)) <= 1e-14 * float(GD)


# ------------------------------------------------------------- cut predicate --

def test_cut_ranges_vs_exact_rationals():
    """Random centres: the FP64 predicate equals the exact rational decision
    |nu_min + i dnu - nu0| <= cut (ties have probability zero).  Centres placed
    on decimal ties: the decision equals the decimal (intended) one, inclusive."""
    rng = np.random.default_rng(11)
    nu_min, dnu, nbins, cut = 0.0, 0.1, 3000, 2.5

    def check(nu0, exact):
        lo, hi = oracle.line_ranges(nu0, nu_min, dnu, nbins, cut)
        for l in range(nu0.size):
            if nu0[l] <= 0:              # reading: no Doppler width, the line adds nothing
                assert hi[l] < lo[l]
                continue
            v = exact(nu0[l])
            c = int(nu0[l] / dnu)
            inside = [i for i in range(max(0, c - 40), min(nbins, c + 40))
                      if abs(exact(nu_min) + i * exact(dnu) - v) <= exact(cut)]
            if inside:
                assert (lo[l], hi[l]) == (inside[0], inside[-1]), (l, nu0[l])
            else:
                assert hi[l] < lo[l]

    check(rng.uniform(-3, 303, 300), lambda v: Fraction(float(v)))
    check(np.array([0.0, 299.9, 10.0, 150.05, 7.5]), lambda v: Fraction(repr(float(v))))


def test_cut_tie_is_inclusive_and_no_cut_is_full_grid():
    lo, hi = oracle.line_ranges(np.array([10.0]), 0.0, 0.5, 100, 2.0)
    assert (lo[0], hi[0]) == (16, 24)           # bins at 8.0 .. 12.0 inclusive
    lo, hi = oracle.line_ranges(np.array([10.0]), 0.0, 0.5, 100, 0.0)
    assert (lo[0], hi[0]) == (0, 99)


# ------------------------------------------- plinth and per-line cuts (Sect. 2.1, 2.4.3) --

def test_plinth_vanishes_at_the_cut_edge():
    """A line on a bin centre with a cut of a whole number of bins: the bins at
    +-cut sit exactly at the cutting length, so with the plinth removed they
    are exactly zero; inside the cut the profile stays positive and equals the
    un-removed one minus a constant."""
    nu_min, dnu, nbins = 0.0, 0.125, 200                # binary-exact grid
    nu0, S, aD, GL, cut = 10.0, 3e-21, 0.21, 0.07, 2.5    # u = 80, W = 20 exactly
    a = oracle.sigma(np.array([nu0]), np.array([S]), np.array([aD]), np.array([GL]), nu_min,
                     dnu, nbins, cut)
    b = oracle.sigma(np.array([nu0]), np.array([S]), np.array([aD]), np.array([GL]), nu_min,
                     dnu, nbins, cut, plinth=True)
    assert b[60] == 0.0 and b[100] == 0.0
    assert np.all(b[61:100] > 0) and np.all(b[:60] == 0) and np.all(b[101:] == 0)
    d = a[60:101] - b[60:101]          # rounding of a - h is ~1e-16 of a, a up to 1e3 h
    assert np.all(np.abs(d - d[0]) <= 4e-16 * a[60:101]) and d[0] > 0


def test_plinth_area_lorentz_and_gauss_limits():
    """Area of the plinth-removed profile against closed forms: Lorentzian
    (alpha_D << Gamma_L) (2/pi) atan(c/G) - 2 c G / (pi (c^2 + G^2)); Gaussian
    (Gamma_L = 0) erf(c/alpha_D) - 2 c exp(-c^2/alpha_D^2) / (alpha_D sqrt(pi))."""
    dnu = 0.0005
    grid = (0.0, dnu, 40000)
    nu0 = 10.00025                                      # halfway between bins
    S = 1.0
    G, aD, c = 0.1, 1e-5, 2.0                            # Lorentzian limit, (aD/G)^2 = 1e-8
    sig = oracle.sigma(np.array([nu0]), np.array([S]), np.array([aD]), np.array([G]), *grid, c,
                       plinth=True)
    # the cut edges fall on half-bins: midpoint rule, whose leading error for the
    # kinked profile is (dnu^2 / 12) |phi'(c)| (Euler-Maclaurin)
    exact = 2 / math.pi * math.atan(c / G) - 2 * c * G / (math.pi * (c * c + G * G))
    exact += dnu ** 2 / 12 * (G / math.pi) * 2 * c / (c * c + G * G) ** 2
    assert abs(sig.sum() * dnu - exact) < 2e-8 * exact
    aD, c = 0.05, 0.1
    sig = oracle.sigma(np.array([nu0]), np.array([S]), np.array([aD]), np.array([0.0]), *grid, c,
                       plinth=True)
    phic = math.exp(-(c / aD) ** 2) / (aD * SQPI)
    exact = math.erf(c / aD) - 2 * c * phic
    exact += dnu ** 2 / 12 * 2 * c / aD ** 2 * phic
    assert abs(sig.sum() * dnu - exact) < 1e-9 * exact


def test_per_line_cuts_doppler_and_lorentz():
    """Doppler-multiple cuts: factor * sqrt(ln 2) * alpha_D with alpha_D from
    Eq. gammaD in mpmath; Lorentz-multiple cuts: factor * Gamma_L.  The pair
    count equals the exact rational count of bins with |nu_i - nu0| <= cut_l."""
    rng = np.random.default_rng(31)
    n = 200
    nu0 = np.sort(rng.uniform(1.0, 300.0, n))
    T, m = 1700.0, 18.0
    g = json.load(open(GOLDEN))
    c, kB, amu = g["c"]["value"], g["k_B"]["value"], 1.660538921e-24   # amu: CODATA 2010
    aD, GL = oracle.widths(nu0, rng.uniform(0.01, 0.1, n), rng.uniform(0.3, 0.8, n), T, 0.7, m)
    f = 37.0
    cd = oracle.line_cuts(nu0, GL, oracle.CUT_DOPPLER, f, T, m)
    with mp.workdps(40):
        for l in range(0, n, 17):
            ref = f * mp.sqrt(mp.log(2)) * mp.mpf(nu0[l]) / mp.mpf(c) * mp.sqrt(
                2 * mp.mpf(kB) * T / (m * mp.mpf(amu)))
            assert abs(cd[l] - float(ref)) <= 4e-16 * float(ref)
    cl = oracle.line_cuts(nu0, GL, oracle.CUT_LORENTZ, 3.0, T, m)
    assert np.allclose(cl, 3.0 * GL, rtol=1e-15, atol=0)
    nu_min, dnu, nbins = 0.0, 0.01, 30000
    for cuts in (cd, cl):
        exact = 0
        for l in range(n):
            v, cf = Fraction(float(nu0[l])), Fraction(float(cuts[l]))
            i0 = int(nu0[l] / dnu)
            k = int(cuts[l] / dnu) + 3
            exact += sum(1 for i in range(max(0, i0 - k), min(nbins, i0 + k + 1))
                         if abs(Fraction(nu_min) + i * Fraction(dnu) - v) <= cf)
        assert oracle.count_pairs_percut(nu0, cuts, nu_min, dnu, nbins) == exact


# ----------------------------------- HITRAN broadening and pressure shift (Sect. 2.2) --

def test_hitran_width_reduces_to_the_exomol_form():
    """Eq. gammaL: with P_self = 0 it is the ExoMol form with gamma_air, with
    P_self = P the ExoMol form with gamma_self, and it is affine in P_self."""
    rng = np.random.default_rng(41)
    n = 50
    nu0 = rng.uniform(10, 3000, n)
    ga, gs, nT = rng.uniform(0.01, 0.1, n), rng.uniform(0.1, 0.5, n), rng.uniform(0.3, 0.8, n)
    A = rng.uniform(1e6, 1e8, n)
    T, P, m = 700.0, 2.5, 18.0
    _, e_air = oracle.widths(nu0, ga, nT, T, P, m, A=A)
    _, e_self = oracle.widths(nu0, gs, nT, T, P, m, A=A)
    aD, h0 = oracle.widths_hitran(nu0, ga, gs, nT, T, P, 0.0, m, A=A)
    _, h1 = oracle.widths_hitran(nu0, ga, gs, nT, T, P, P, m, A=A)
    _, hh = oracle.widths_hitran(nu0, ga, gs, nT, T, P, 0.5 * P, m, A=A)
    assert np.allclose(h0, e_air, rtol=1e-14, atol=0) and np.allclose(h1, e_self, rtol=1e-14, atol=0)
    assert np.allclose(hh, 0.5 * (h0 + h1), rtol=1e-14, atol=0)
    assert np.array_equal(aD, oracle.widths(nu0, ga, nT, T, P, m)[0])


def test_pressure_shift_translates_the_line():
    """A shift delta P / P_ref of exactly k bins moves sigma by k bins and
    changes nothing else (the strength and width keep nu0)."""
    dnu = 0.125
    grid = (0.0, dnu, 400)
    L = dict(nu0=np.array([20.0625]), S_ref=np.array([1e-20]), E_low=np.array([500.0]),
             gamma_ref=np.array([0.07]), n_T=np.array([0.6]), mass_amu=18.0, s_mode=0)
    state = (800.0, 2.0, 0.1 * 800 ** 1.5, 0.1 * 296 ** 1.5)
    base = oracle.cross_section(L, grid, state, 5.0)
    Ls = dict(L, delta=np.array([0.375]))                  # 0.375 * 2 bar = 0.75 = 6 bins
    shifted = oracle.cross_section(Ls, grid, state, 5.0)
    assert np.array_equal(shifted[6:], base[:-6]) and np.all(shifted[:6] == 0)


# -------------------------------------------------- line profiles (Sect. 2.1) --

def _prof(profile, nu0, S, aD, GL, grid, cut, plinth=False):
    return oracle.sigma(np.array([nu0]), np.array([S]), np.array([aD]), np.array([GL]), *grid,
                        cut, profile=profile, plinth=plinth)


def test_lorentz_and_doppler_profiles():
    """Lorentzian: half maximum at Gamma_L, arctan area, and the Voigt's
    alpha_D -> 0 limit (the Voigt path is pinned to mpmath).  Doppler: half
    maximum at Gamma_D = sqrt(ln 2) alpha_D, erf area, and the Voigt at
    Gamma_L = 0."""
    dnu = 0.01
    grid = (0.0, dnu, 20000)
    nu0, S, GL = 100.0, 1.0, 0.25                          # on bin 10000; Gamma_L = 25 bins
    lor = _prof(oracle.PROFILE_LORENTZ, nu0, S, 1e-3, GL, grid, 50.0)
    assert abs(lor[10025] / lor[10000] - 0.5) < 1e-12
    # the cut edges fall on bin centres: the point sum is the trapezoid rule plus
    # half an end value at each edge
    exact = 2 / math.pi * math.atan(50.0 / GL) + dnu * (GL / math.pi) / (50.0 ** 2 + GL ** 2)
    assert abs(lor.sum() * dnu - exact) < 1e-8
    voi = _prof(oracle.PROFILE_VOIGT, nu0, S, 1e-6, GL, grid, 50.0)
    m = lor > 0
    assert np.allclose(voi[m], lor[m], rtol=1e-9, atol=0)
    aD = 0.3 / math.sqrt(math.log(2))                       # Gamma_D = 30 bins
    dop = _prof(oracle.PROFILE_DOPPLER, nu0, S, aD, 0.0, grid, 5.0)
    assert abs(dop[10030] / dop[10000] - 0.5) < 1e-12
    assert abs(dop.sum() * dnu - math.erf(5.0 / aD)) < 1e-12
    voi = _prof(oracle.PROFILE_VOIGT, nu0, S, aD, 0.0, grid, 5.0)
    assert np.array_equal(voi, dop) or np.allclose(voi, dop, rtol=1e-14, atol=0)


def test_binned_gaussian_telescopes_and_limits():
    """Bin averages of the Gaussian telescope: the sum of sigma_i dnu over any
    run of bins is S/2 [erf(right edge / alpha_D) - erf(left edge / alpha_D)]
    (mpmath); for alpha_D >> dnu the binned values approach the point Doppler
    profile to O((dnu / alpha_D)^2)."""
    dnu = 0.05
    grid = (0.0, dnu, 4000)
    nu0, S, aD = 100.0123, 2.0, 0.037                        # narrower than a bin
    b = _prof(oracle.PROFILE_BINNED_GAUSS, nu0, S, aD, 0.0, grid, 0.0)
    for lo, hi in [(1990, 2010), (2000, 2001), (1998, 2000), (1000, 3000)]:
        with mp.workdps(30):
            left = mp.mpf(lo) * mp.mpf(dnu) - mp.mpf(dnu) / 2 - mp.mpf(nu0)
            right = mp.mpf(hi) * mp.mpf(dnu) + mp.mpf(dnu) / 2 - mp.mpf(nu0)
            ref = float(S / 2 * (mp.erf(right / aD) - mp.erf(left / aD)))
        assert abs(b[lo:hi + 1].sum() * dnu - ref) <= 1e-13 * S, (lo, hi)
    aD = 1.5                                                # 30 bins wide
    b = _prof(oracle.PROFILE_BINNED_GAUSS, nu0, S, aD, 0.0, grid, 20.0)
    d = _prof(oracle.PROFILE_DOPPLER, nu0, S, aD, 0.0, grid, 20.0)
    m = d > 1e-6 * d.max()
    # bin average of f = exp(-x^2), h = dnu/aD: f + (h^2/24) f2 + (h^4/1920) f4 + ...
    # with f2/f = 4x^2 - 2 and f4/f = 16x^4 - 48x^2 + 12 (second, fourth derivatives)
    x = (grid[0] + dnu * np.arange(grid[2]) - nu0) / aD
    h = dnu / aD
    X = x * x
    pred = d * (1 + h ** 2 / 24 * (4 * X - 2) + h ** 4 / 1920 * (16 * X * X - 48 * X + 12))
    assert np.max(np.abs(b[m] - pred[m]) / d[m]) < 2e-8


# ------------------------------------------------------------ sigma: limits --

def _single(nu0, S, aD, GL, grid, cut):
    nu_min, dnu, nbins = grid
    return oracle.sigma(np.array([nu0]), np.array([S]), np.array([aD]), np.array([GL]), nu_min,
                        dnu, nbins, cut)


def test_gaussian_limit_and_area():
    grid = (0.0, 0.005, 4000)
    nu0, S, aD = 10.00123, 2.5e-21, 0.031
    sig = _single(nu0, S, aD, 0.0, grid, 10 * aD)
    nu = grid[0] + grid[1] * np.arange(grid[2])
    d = nu - nu0
    ref = np.where(np.abs(d) <= 10 * aD, S * np.exp(-(d / aD) ** 2) / (aD * SQPI), 0.0)
    m = ref > 0
    tol = 1e-13 * (1 + (d[m] / aD) ** 2)  # x carries ~3e-14 absolute error from u = nu0/dnu
    assert np.all(np.abs(sig[m] - ref[m]) <= tol * ref[m]) and np.all(sig[~m] == 0)
    # sum sigma dnu / S = erf(10) = 1 to 1e-44; the point-sum error ~ 2 exp(-pi^2 aD^2/dnu^2)
    assert abs(sig.sum() * grid[1] / S - 1.0) < 1e-13
    # half maximum at the Doppler HWHM sqrt(ln2) alpha_D
    G = math.sqrt(math.log(2)) * aD
    w = oracle.faddeeva(np.array([0.0, G / aD]), 0.0).real
    assert abs(w[1] / w[0] - 0.5) < 1e-15


def test_lorentzian_limit_and_arctan_area():
    dnu = 0.01
    grid = (0.0, dnu, 20000)
    nu0 = 100.005                                # halfway between bins
    GL, aD, S = 1.0, 1e-5, 1e-20
    cut = 25.0                                   # cut edges fall on half-bins: midpoint rule
    sig = _single(nu0, S, aD, GL, grid, cut)
    nu = grid[0] + dnu * np.arange(grid[2])
    d = nu - nu0
    lor = S * GL / (math.pi * (d * d + GL * GL))
    m = np.abs(d) <= cut
    assert np.allclose(sig[m], lor[m], rtol=2e-10)
    area = sig.sum() * dnu / S
    exact = 2 / math.pi * math.atan(cut / GL)
    # midpoint-rule error (dnu^2 / 24) * [phi'] ~ 1e-9
    assert abs(area - exact) < 1e-8


def test_voigt_wide_cut_area_vs_mpmath_tail():
    dnu, aD, GL, S = 0.01, 0.05, 0.02, 1.0
    grid = (0.0, dnu, 40000)
    nu0, cut = 200.005, 150.0
    sig = _single(nu0, S, aD, GL, grid, cut)
    area = sig.sum() * dnu
    y = GL / aD
    X = 4e4                       # in units of alpha_D
    with mp.workdps(30):
        near = mp.quad(lambda x: w_mp(x, y, 30).real, [cut / aD, 1e4, X]) / mp.sqrt(mp.pi)
    # beyond X: Re w = y / (sqrt(pi)(x^2 + y^2)) (1 + O(x^-2)), integral in closed form
    far = (math.pi / 2 - math.atan(X / y)) / math.pi
    tail = 2 * (float(near) + far)
    assert abs(area - (1 - tail)) < 2e-9


def test_sigma_linearity_and_permutation():
    rng = np.random.default_rng(5)
    n = 300
    nu0 = rng.uniform(0, 100, n)
    S = 10 ** rng.uniform(-25, -20, n)
    aD = rng.uniform(0.01, 0.2, n)
    GL = rng.uniform(0.0, 0.3, n)
    grid = (0.0, 0.05, 2000)
    full = oracle.sigma(nu0, S, aD, GL, *grid, 5.0)
    a = oracle.sigma(nu0[:120], S[:120], aD[:120], GL[:120], *grid, 5.0)
    b = oracle.sigma(nu0[120:], S[120:], aD[120:], GL[120:], *grid, 5.0)
    assert np.allclose(full, a + b, rtol=1e-14, atol=0)
    p = rng.permutation(n)
    perm = oracle.sigma(nu0[p], S[p], aD[p], GL[p], *grid, 5.0)
    assert np.allclose(full, perm, rtol=1e-13, atol=0)
    # window evaluation equals the slice of the full array, sorted or not
    o = np.argsort(nu0)
    win = oracle.sigma(nu0[o], S[o], aD[o], GL[o], *grid, 5.0, bin_lo=700, bin_hi=913,
                       sorted_nu0=True)
    assert np.allclose(win, full[700:913], rtol=1e-13, atol=0)


def test_sigma_brute_force_mpmath():
    """Whole path for 5 lines x 200 bins at 40 digits from the paper's
    equations (S-mode scaling, Eq. alphaD, ExoMol Gamma_L, w = exp(-z^2) erfc(-iz))."""
    rng = np.random.default_rng(2)
    n = 5
    L = dict(nu0=np.sort(rng.uniform(1.0, 9.0, n)), S_ref=10 ** rng.uniform(-22, -19, n),
             E_low=rng.exponential(2000, n), gamma_ref=rng.uniform(0.01, 0.1, n),
             n_T=rng.uniform(0.3, 0.8, n), mass_amu=18.0)
    grid = (0.0, 0.05, 200)
    T, P, cut = 900.0, 0.3, 1.5
    sig = oracle.cross_section(L, grid, (T, P, Q(T), Q(296.0)), cut)
    cst = oracle.constants()
    with mp.workdps(40):
        c2 = mp.mpf(cst["h"]) * mp.mpf(cst["c"]) / mp.mpf(cst["k_B"])
        m = 18 * mp.mpf(cst["amu"])
        ref = [mp.mpf(0)] * grid[2]
        for l in range(n):
            nu = mp.mpf(L["nu0"][l])
            E = mp.mpf(L["E_low"][l])
            S = (mp.mpf(L["S_ref"][l]) * mp.mpf(Q(296.0)) / mp.mpf(Q(T)) *
                 mp.exp(-c2 * E / T) / mp.exp(-c2 * E / 296) *
                 (1 - mp.exp(-c2 * nu / T)) / (1 - mp.exp(-c2 * nu / 296)))
            aD = nu / mp.mpf(cst["c"]) * mp.sqrt(2 * mp.mpf(cst["k_B"]) * T / m)
            GL = mp.mpf(L["gamma_ref"][l]) * (mp.mpf(296) / T) ** mp.mpf(L["n_T"][l]) * P
            for i in range(grid[2]):
                d = mp.mpf(i) * mp.mpf(grid[1]) - nu
                if abs(d) <= cut:
                    z = mp.mpc(d / aD, GL / aD)
                    ref[i] += S * (mp.exp(-z * z) * mp.erfc(-1j * z)).real / (aD * mp.sqrt(mp.pi))
    ref = np.array([float(r) for r in ref])
    m = ref > 0
    assert np.array_equal(m, sig > 0)
    assert np.allclose(sig[m], ref[m], rtol=1e-12, atol=0)


# ---------------------------------------------------------------- gradients --

def test_backward_vs_central_differences():
    rng = np.random.default_rng(9)
    n = 12
    L = dict(nu0=np.sort(rng.uniform(2, 18, n)), S_ref=10 ** rng.uniform(-22, -20, n),
             E_low=rng.exponential(1500, n), gamma_ref=rng.uniform(0.01, 0.1, n),
             n_T=rng.uniform(0.3, 0.8, n), mass_amu=18.0)
    grid = (0.0, 0.02, 1000)
    cut = 3.0
    g = rng.standard_normal(grid[2])
    T, P = 800.0, 0.5

    def loss(T, P, Sref=None, gam=None):
        LL = dict(L)
        if Sref is not None:
            LL["S_ref"] = Sref
        if gam is not None:
            LL["gamma_ref"] = gam
        return float(g @ oracle.cross_section(LL, grid, (T, P, Q(T), Q(296.0)), cut))

    dS, dG, dT, dP = oracle.backward(L, grid, (T, P, Q(T), Q(296.0), 1.5 / T), cut, g)

    def cdiff(f, x0, h):  # Richardson-extrapolated central difference
        d1 = (f(x0 + h) - f(x0 - h)) / (2 * h)
        d2 = (f(x0 + h / 2) - f(x0 - h / 2)) / h
        return (4 * d2 - d1) / 3

    # Q(T) = 0.1 T^1.5 also moves with T: the loss closure re-evaluates it
    fdT = cdiff(lambda t: loss(t, P), T, T * 1e-3)
    fdP = cdiff(lambda p: loss(T, p), P, P * 1e-3)
    assert abs(dT - fdT) <= 1e-7 * abs(fdT)
    assert abs(dP - fdP) <= 1e-7 * abs(fdP)
    for l in [0, 5, 11]:
        e = np.zeros(n)
        e[l] = 1.0
        h = L["S_ref"][l] * 1e-3
        fdS = cdiff(lambda s: loss(T, P, Sref=L["S_ref"] + (s - L["S_ref"][l]) * e), L["S_ref"][l], h)
        assert abs(dS[l] - fdS) <= 1e-7 * abs(fdS) + 1e-300
        h = L["gamma_ref"][l] * 1e-2  # Richardson: O(h^4); smaller steps hit roundoff
        fdG = cdiff(lambda s: loss(T, P, gam=L["gamma_ref"] + (s - L["gamma_ref"][l]) * e),
                    L["gamma_ref"][l], h)
        assert abs(dG[l] - fdG) <= 1e-7 * abs(fdG)
