"""Plain FP64 CPU oracle for the HELIOS-K 2.0 opacity hot path.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only users.  The product library never imports,
links or calls anything here, and nothing here imports the product library.

All arithmetic lives in ``hk_oracle.c`` (plain C, FP64, OpenMP over bins);
this module only marshals numpy arrays through ctypes.  Each function states
the passage of arXiv:2101.02005 it follows.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = ctypes.CDLL(path)
        d = ctypes.POINTER(ctypes.c_double)
        i64 = ctypes.c_int64
        _lib.hko_constants.argtypes = [d]
        _lib.hko_faddeeva.argtypes = [i64, d, d, d, d]
        _lib.hko_faddeeva_deriv.argtypes = [i64, d, d, d, d]
        _lib.hko_line_strength.argtypes = [i64, d, d, d, d, d, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_int, d]
        _lib.hko_widths.argtypes = [i64, d, d, d, d, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_double, d, d]
        _lib.hko_line_ranges.argtypes = [i64, d, ctypes.c_double, ctypes.c_double, i64,
                                         ctypes.c_double, ctypes.POINTER(i64),
                                         ctypes.POINTER(i64)]
        _lib.hko_count_pairs.argtypes = [i64, d, ctypes.c_double, ctypes.c_double, i64,
                                         ctypes.c_double]
        _lib.hko_count_pairs.restype = i64
        _lib.hko_sigma.argtypes = [i64, d, d, d, d, ctypes.c_int, ctypes.c_double,
                                   ctypes.c_double, i64, ctypes.c_double, i64, i64, d,
                                   ctypes.c_int]
        _lib.hko_line_cuts.argtypes = [i64, d, d, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, d]
        _lib.hko_count_pairs_percut.argtypes = [i64, d, d, ctypes.c_double, ctypes.c_double,
                                                i64]
        _lib.hko_count_pairs_percut.restype = i64
        _lib.hko_sigma_ext.argtypes = [i64, d, d, d, d, d, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_double, i64, ctypes.c_double,
                                       i64, i64, d, ctypes.c_int]
        _lib.hko_sigma_prof.argtypes = [i64, d, d, d, d, d, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_double, ctypes.c_double, i64,
                                        ctypes.c_double, i64, i64, d, ctypes.c_int]
        _lib.hko_widths_hitran.argtypes = [i64, d, d, d, d, d] + [ctypes.c_double] * 6 + [d, d]
        _lib.hko_shift.argtypes = [i64, d, d, ctypes.c_double, ctypes.c_double, d]
        _lib.hko_backward.argtypes = [i64, d, d, d, d, d, d] + [ctypes.c_double] * 10 + [
            i64, ctypes.c_double, d, d, d, d, d, ctypes.c_int]
    return _lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, n=None):
    if a is None:
        return None
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None:
        assert a.shape == (n,), (a.shape, n)
    return a


# Defaults used by every config of the benchmark (T_ref, P_ref: reading of
# Sect. 2.2, ExoMol form; P in bar).
T_REF = 296.0
P_REF = 1.0


def constants():
    """(c, k_B, h, amu, c2, pi) as the oracle uses them (Sect. 2.2, Eq. S)."""
    out = np.zeros(6)
    lib().hko_constants(_d(out))
    return dict(zip(["c", "k_B", "h", "amu", "c2", "pi"], out.tolist()))


def faddeeva(x, y):
    """w(x + iy) for y >= 0: trapezoid with pole correction (|z|^2 < 64) or
    Laplace continued fraction; returns a complex128 array."""
    x, y = np.broadcast_arrays(np.asarray(x, np.float64), np.asarray(y, np.float64))
    x = np.ascontiguousarray(x).ravel()
    y = np.ascontiguousarray(y).ravel()
    re = np.empty_like(x)
    im = np.empty_like(x)
    lib().hko_faddeeva(x.size, _d(x), _d(y), _d(re), _d(im))
    return re + 1j * im


def faddeeva_deriv(x, y):
    """w'(x + iy) (Faddeeva ODE / asymptotic series)."""
    x, y = np.broadcast_arrays(np.asarray(x, np.float64), np.asarray(y, np.float64))
    x = np.ascontiguousarray(x).ravel()
    y = np.ascontiguousarray(y).ravel()
    re = np.empty_like(x)
    im = np.empty_like(x)
    lib().hko_faddeeva_deriv(x.size, _d(x), _d(y), _d(re), _d(im))
    return re + 1j * im


def line_strength(nu0, E_low, T, Q_T, Q_Tref, mass_amu, S_ref=None, A=None, g_up=None,
                  s_mode=0, T_ref=T_REF, per_gram=False):
    """S(T) per line (Sect. 2.2.2 Eq. S; split form of Sect. 2.4.3)."""
    nu0 = _f64(nu0)
    n = nu0.size
    E_low = _f64(E_low, n)
    S_ref = _f64(S_ref, n) if S_ref is not None else np.zeros(n)
    A = _f64(A, n) if A is not None else np.zeros(n)
    g_up = _f64(g_up, n) if g_up is not None else np.zeros(n)
    out = np.empty(n)
    lib().hko_line_strength(n, _d(nu0), _d(S_ref), _d(A), _d(g_up), _d(E_low), int(s_mode),
                            T, Q_T, T_ref, Q_Tref, mass_amu, int(bool(per_gram)), _d(out))
    return out


def widths(nu0, gamma_ref, n_T, T, P, mass_amu, A=None, T_ref=T_REF, P_ref=P_REF):
    """(alpha_D, Gamma_L) per line: Eq. gammaD / Eq. alphaD and the ExoMol
    Lorentz form of Sect. 2.2 with the natural term A/(4 pi c)."""
    nu0 = _f64(nu0)
    n = nu0.size
    g = _f64(gamma_ref, n)
    nT = _f64(n_T, n)
    Ap = _f64(A, n) if A is not None else None
    aD = np.empty(n)
    GL = np.empty(n)
    lib().hko_widths(n, _d(nu0), _d(g), _d(nT), _d(Ap) if Ap is not None else None, T, P,
                     T_ref, P_ref, mass_amu, _d(aD), _d(GL))
    return aD, GL


def widths_hitran(nu0, gamma_air, gamma_self, n_T, T, P, P_self, mass_amu, A=None, T_ref=T_REF,
                  P_ref=P_REF):
    """(alpha_D, Gamma_L) with the HITRAN air/self-broadened Lorentz width (Eq. gammaL)."""
    nu0 = _f64(nu0)
    n = nu0.size
    ga, gs, nT = _f64(gamma_air, n), _f64(gamma_self, n), _f64(n_T, n)
    A = _f64(A, n) if A is not None else None
    aD, GL = np.empty(n), np.empty(n)
    lib().hko_widths_hitran(n, _d(nu0), _d(ga), _d(gs), _d(nT), _d(A) if A is not None else None,
                            T, P, P_self, T_ref, P_ref, mass_amu, _d(aD), _d(GL))
    return aD, GL


def shift(nu0, delta, P, P_ref=P_REF):
    """Pressure-shifted positions nu0 + delta P / P_ref."""
    nu0 = _f64(nu0)
    out = np.empty(nu0.size)
    lib().hko_shift(nu0.size, _d(nu0), _d(_f64(delta, nu0.size)), P, P_ref, _d(out))
    return out


def line_ranges(nu0, nu_min, dnu, nbins, cut):
    """Inclusive bin range [lo, hi] of each line inside the cut (cut <= 0: all)."""
    nu0 = _f64(nu0)
    lo = np.empty(nu0.size, np.int64)
    hi = np.empty(nu0.size, np.int64)
    p = ctypes.POINTER(ctypes.c_int64)
    lib().hko_line_ranges(nu0.size, _d(nu0), nu_min, dnu, nbins, cut,
                          lo.ctypes.data_as(p), hi.ctypes.data_as(p))
    return lo, hi


def count_pairs(nu0, nu_min, dnu, nbins, cut):
    """Number of (line, bin) pairs the cut admits: the algorithmic Voigt count."""
    nu0 = _f64(nu0)
    return int(lib().hko_count_pairs(nu0.size, _d(nu0), nu_min, dnu, nbins, cut))


CUT_FIXED, CUT_NONE, CUT_DOPPLER, CUT_LORENTZ = 0, 1, 2, 3
PROFILE_VOIGT, PROFILE_LORENTZ, PROFILE_DOPPLER, PROFILE_BINNED_GAUSS = 0, 1, 2, 3


def line_cuts(nu0, gammaL, mode, factor, T, mass_amu):
    """Per-line cutting lengths (Sect. 2.4.3 item 4): mode CUT_DOPPLER = factor
    times Gamma_D = sqrt(ln 2) alpha_D (Eq. gammaD), CUT_LORENTZ = factor times
    Gamma_L."""
    nu0 = _f64(nu0)
    n = nu0.size
    GL = _f64(gammaL, n)
    out = np.empty(n)
    lib().hko_line_cuts(n, _d(nu0), _d(GL), int(mode), float(factor), float(T),
                        float(mass_amu), _d(out))
    return out


def count_pairs_percut(nu0, cut_l, nu_min, dnu, nbins):
    nu0 = _f64(nu0)
    c = _f64(cut_l, nu0.size)
    return int(lib().hko_count_pairs_percut(nu0.size, _d(nu0), _d(c), nu_min, dnu, nbins))


def sigma(nu0, S, alphaD, gammaL, nu_min, dnu, nbins, cut, bin_lo=0, bin_hi=None,
          sorted_nu0=False, nthreads=0, cut_l=None, plinth=False, profile=PROFILE_VOIGT):
    """sigma_i for bins [bin_lo, bin_hi): the direct FP64 sum of S * Re w / (alpha_D sqrt(pi)).
    cut_l: per-line cutting lengths (overrides `cut`); plinth: subtract each
    line's value at its cutting length inside its cut (Sect. 2.1); profile:
    PROFILE_* (Voigt, Lorentzian, Doppler, binned Gaussian; Sect. 2.1)."""
    nu0 = _f64(nu0)
    n = nu0.size
    S = _f64(S, n)
    aD = _f64(alphaD, n)
    GL = _f64(gammaL, n)
    cl = _f64(cut_l, n)
    if bin_hi is None:
        bin_hi = nbins
    out = np.zeros(max(bin_hi - bin_lo, 0))
    lib().hko_sigma_prof(n, _d(nu0), _d(S), _d(aD), _d(GL), _d(cl) if cl is not None else None,
                         int(bool(plinth)), int(profile), int(bool(sorted_nu0)), nu_min, dnu,
                         nbins, cut, bin_lo, bin_hi, _d(out), int(nthreads))
    return out


def cross_section(lines, grid, state, cut, bin_lo=0, bin_hi=None, nthreads=0,
                  T_ref=T_REF, P_ref=P_REF, per_gram=False, cut_mode=CUT_FIXED, plinth=False,
                  profile=PROFILE_VOIGT, P_self=0.0):
    """Full path for one (T, P): S(T), widths, then the direct sum.

    ``lines``: mapping with nu0, E_low, gamma_ref, n_T and S_ref (s_mode 0) or
    A + g_up (s_mode 1), optional A for the natural term, mass_amu, s_mode,
    sorted.  ``grid``: (nu_min, dnu, nbins).  ``state``: (T, P, Q_T, Q_Tref).
    cut_mode CUT_DOPPLER / CUT_LORENTZ: ``cut`` is the factor of the per-line
    half width; CUT_NONE: no cut.  plinth: remove the plinth (Sect. 2.1).
    HITRAN lists: ``gamma_self`` in ``lines`` selects the air/self width of
    Eq. gammaL (gamma_ref is then gamma_air; P_self the self partial pressure),
    ``delta`` the pressure shift of the positions.
    """
    nu_min, dnu, nbins = grid
    T, P, Q_T, Q_Tref = state[:4]
    s_mode = int(lines.get("s_mode", 0))
    S = line_strength(lines["nu0"], lines["E_low"], T, Q_T, Q_Tref, lines["mass_amu"],
                      S_ref=lines.get("S_ref"), A=lines.get("A"), g_up=lines.get("g_up"),
                      s_mode=s_mode, T_ref=T_ref, per_gram=per_gram)
    if lines.get("gamma_self") is not None:
        aD, GL = widths_hitran(lines["nu0"], lines["gamma_ref"], lines["gamma_self"],
                               lines["n_T"], T, P, P_self, lines["mass_amu"], A=lines.get("A"),
                               T_ref=T_ref, P_ref=P_ref)
    else:
        aD, GL = widths(lines["nu0"], lines["gamma_ref"], lines["n_T"], T, P, lines["mass_amu"],
                        A=lines.get("A"), T_ref=T_ref, P_ref=P_ref)
    pos = lines["nu0"]
    sorted_pos = bool(lines.get("sorted", False))
    if lines.get("delta") is not None:
        pos = shift(lines["nu0"], lines["delta"], P, P_ref)
        sorted_pos = False
    cut_l = None
    if cut_mode == CUT_NONE:
        cut = 0.0
    elif cut_mode in (CUT_DOPPLER, CUT_LORENTZ):
        cut_l = line_cuts(lines["nu0"], GL, cut_mode, cut, T, lines["mass_amu"])
    return sigma(pos, S, aD, GL, nu_min, dnu, nbins, cut, bin_lo, bin_hi,
                 sorted_nu0=sorted_pos, nthreads=nthreads, cut_l=cut_l,
                 plinth=plinth, profile=profile)


def backward(lines, grid, state, cut, grad_sigma, dL_dSref=None, dL_dgamma=None, nthreads=0,
             T_ref=T_REF, P_ref=P_REF):
    """Adjoint of L = sum_i g_i sigma_i for one (T, P) point, S-mode.

    ``state``: (T, P, Q_T, Q_Tref, dlnQ_dT).  Per-line gradients accumulate
    into the given arrays; returns (dL_dSref, dL_dgamma, dL_dT, dL_dP)."""
    nu_min, dnu, nbins = grid
    T, P, Q_T, Q_Tref, dlnQ_dT = state
    nu0 = _f64(lines["nu0"])
    n = nu0.size
    if dL_dSref is None:
        dL_dSref = np.zeros(n)
    if dL_dgamma is None:
        dL_dgamma = np.zeros(n)
    g = _f64(grad_sigma, nbins)
    A = lines.get("A")
    A = _f64(A, n) if A is not None else None
    dT = ctypes.c_double(0.0)
    dP = ctypes.c_double(0.0)
    lib().hko_backward(n, _d(nu0), _d(_f64(lines["S_ref"], n)), _d(_f64(lines["E_low"], n)),
                       _d(_f64(lines["gamma_ref"], n)), _d(_f64(lines["n_T"], n)),
                       _d(A) if A is not None else None, T, P, Q_T, dlnQ_dT, T_ref, P_ref,
                       Q_Tref, lines["mass_amu"], nu_min, dnu, nbins, cut, _d(g),
                       _d(dL_dSref), _d(dL_dgamma), ctypes.byref(dT), ctypes.byref(dP),
                       int(nthreads))
    return dL_dSref, dL_dgamma, dT.value, dP.value
