"""The accuracy claims of the FP32C kernel's band rules, checked in FP64 on the
CPU (no GPU): the one- to four-node Gauss-Hermite bands, the float core's
18-node trapezoid with its pole term, the 8-node Gauss-Hermite ring of the
short-line core, and the
series in 1/x that sums a warp's 32 lines at once (two-node form over the
short-line interiors, four-node form over everything outside the r2 < 64
union, the wide-line form with 12 and 4 terms).  Each rule is written here
from its definition -- Gauss-Hermite nodes from numpy, the Lorentzian
expansion 1/((x-a)^2 + c^2) = Im(1/(x - z))/c, 1/(x - z) = sum z^m / x^(m+1)
-- and compared with the direct sums (scipy's wofz for the core and the ring),
on seeded rounds built like the kernel's, with the bounds the kernel uses to
choose them; three tests check that the kernel source takes the same bounds.
The GPU parity tests compare the kernel itself with the oracle."""
import os
import re

import numpy as np
import pytest

scipy_special = pytest.importorskip("scipy.special")

SQPI = np.sqrt(np.pi)

# The bounds each rule is held to below, and that the kernel must use.
RING_MIN, RING_C = 26.0, 1.13e9      # R8(y) = min(64, max(26, ln(1.13e9) - ln y))
K2, Z2 = 7, 3.0                       # two nodes: 7 terms when every |z| <= 3
K3, Z3 = 12, 7.0                      # two nodes: 12 terms when every |z| <= 7
K4, Y4, D4 = 12, 1.2, 0.2             # four nodes: y <= 1.2, |d| <= 0.2
KW, KWF, WNEAR, WFAR, WZMAX = 12, 4, 5.0, 100.0, 1000.0   # wide lines


def gh_pairs(n):
    """Positive Gauss-Hermite nodes t_k of an n-node rule and the normalised
    weights of the node pairs (sum of all weights 1)."""
    t, w = np.polynomial.hermite.hermgauss(n)
    w = w / SQPI
    keep = t > 0
    return t[keep], 2.0 * w[keep]


def ring_r2(y):
    return np.minimum(64.0, np.maximum(RING_MIN, np.log(RING_C) - np.log(y)))


def test_ring_rule_meets_its_bound():
    """8 nodes over R8(y) <= r2 < 64: within 2e-7 of Re w (y from 1e-9 to 8)."""
    t, W = gh_pairs(8)
    rng = np.random.default_rng(11)
    y = np.concatenate([10 ** rng.uniform(-9, np.log10(8), 200000), rng.uniform(0, 8, 100000)])
    R = ring_r2(y)
    r2 = R + rng.uniform(0, 1, y.size) * (64.0 - R)
    ok = (r2 < 64.0) & (r2 > y * y)
    y, r2 = y[ok], r2[ok]
    x = np.sqrt(r2 - y * y)
    X, Y = x * x, y * y
    F = sum(Wj * (r2 + tj * tj) / ((X - Y - tj * tj) ** 2 + 4 * X * Y) for tj, Wj in zip(t, W))
    got = y / SQPI * F
    ref = scipy_special.wofz(x + 1j * y).real
    assert np.max(np.abs(got - ref) / ref) <= 2e-7


def lorentz_direct(bins, lines, nodes):
    """sum over lines and nodes of s W / (sqrt(pi)) * y / ((x_j - t)^2 + y^2),
    x_j = (bin - centre_j) b_j: the lines' Gauss-Hermite values."""
    v = np.zeros(bins.size)
    for b, cen, y, s in lines:
        x = (bins - cen) * b
        for t, W in nodes:
            v += s * y / SQPI * W / ((x - t) ** 2 + y * y)
    return v


def series(bins, lines, nodes, K, kuse=None):
    """The round's series about line 0: B_m = sum s W Im(z^m) / (sqrt(pi) beta),
    z = ((t - d) + i y) / beta, evaluated as sum_m B_m / x^(m+1)."""
    b0, c0 = lines[0][0], lines[0][1]
    B = np.zeros(K + 1)
    zmax = 0.0
    for b, cen, y, s in lines:
        beta = b / b0
        d = (c0 - cen) * b
        for t, W in nodes:
            z = complex((t - d) / beta, y / beta)
            zmax = max(zmax, abs(z))
            zk = 1.0 + 0j
            for m in range(1, K + 1):
                zk *= z
                B[m] += s * W / (SQPI * beta) * zk.imag
    k = kuse or K
    x = (bins - c0) * b0
    w = 1.0 / x
    h = np.full(x.size, B[k])
    for m in range(k - 1, 0, -1):
        h = h * w + B[m]
    return h * w * w, zmax


def two_nodes():
    t = 1.0 / np.sqrt(2.0)
    return [(t, 0.5), (-t, 0.5)]


def four_nodes():
    t, W = gh_pairs(4)
    return [(tj, Wj / 2) for tj, Wj in zip(t, W)] + [(-tj, Wj / 2) for tj, Wj in zip(t, W)]


def short_round(rng, spread, ymax):
    b0 = rng.uniform(0.8, 3.0)
    c0 = rng.uniform(-0.5, 0.5)
    return [(b0 * (1 + rng.uniform(-2e-7, 2e-7)), c0 + rng.uniform(-spread, spread),
             10 ** rng.uniform(-4, np.log10(ymax)), 10 ** rng.uniform(-3, 0)) for _ in range(32)]


def test_two_node_round_series():
    """7 terms over the two-node band (every line's r2 >= 2500) when |z| <= 3."""
    rng = np.random.default_rng(12)
    worst, used = 0.0, 0
    for _ in range(300):
        lines = short_round(rng, 0.5, 2.2)
        bins = lines[0][1] + np.concatenate([np.arange(-300, -10), np.arange(10, 300)])
        ok = np.ones(bins.size, bool)
        for b, cen, y, s in lines:
            ok &= ((bins - cen) * b) ** 2 + y * y >= 2500.0
        got, zmax = series(bins[ok], lines, two_nodes(), K2)
        if zmax > Z2 or not ok.any():
            continue
        used += 1
        ref = lorentz_direct(bins[ok], lines, two_nodes())
        worst = max(worst, np.max(np.abs(got - ref) / ref))
    assert used > 100 and worst <= 1e-7


def test_two_node_round_series_twelve_terms():
    """12 terms over the two-node band when 3 < |z| <= 7 (larger y)."""
    rng = np.random.default_rng(15)
    worst, used = 0.0, 0
    for _ in range(300):
        lines = short_round(rng, 0.5, 6.5)
        bins = lines[0][1] + np.concatenate([np.arange(-300, -10), np.arange(10, 300)])
        ok = np.ones(bins.size, bool)
        for b, cen, y, s in lines:
            ok &= ((bins - cen) * b) ** 2 + y * y >= 2500.0
        got, zmax = series(bins[ok], lines, two_nodes(), K3)
        if zmax > Z3 or zmax <= Z2 or not ok.any():
            continue
        used += 1
        ref = lorentz_direct(bins[ok], lines, two_nodes())
        worst = max(worst, np.max(np.abs(got - ref) / ref))
    assert used > 100 and worst <= 1e-7


def test_four_node_round_series():
    """12 terms over every bin where each line has r2 >= 64, lines with
    y <= 1.2 and offsets |d| <= 0.2."""
    rng = np.random.default_rng(13)
    worst = 0.0
    for _ in range(300):
        b0 = rng.uniform(0.8, 3.0)
        lines = [(b0 * (1 + rng.uniform(-2e-7, 2e-7)), rng.uniform(-D4, D4) / b0,
                  10 ** rng.uniform(-4, np.log10(Y4)), 10 ** rng.uniform(-3, 0))
                 for _ in range(32)]
        bins = np.arange(-300, 301, dtype=float)
        ok = np.ones(bins.size, bool)
        for b, cen, y, s in lines:
            ok &= ((bins - cen) * b) ** 2 + y * y >= 64.0
        got, _ = series(bins[ok], lines, four_nodes(), K4)
        ref = lorentz_direct(bins[ok], lines, four_nodes())
        worst = max(worst, np.max(np.abs(got - ref) / ref))
    assert worst <= 1e-7


def test_wide_round_series():
    """Wide lines: 12 terms where |x| >= 5 |z|max, 4 terms where |x| >= 100
    |z|max, centre offsets up to 300 bins, every line in its two-node band."""
    rng = np.random.default_rng(14)
    worst = {KW: 0.0, KWF: 0.0}
    for _ in range(200):
        b0 = rng.uniform(0.1, 3.0)
        c0 = rng.uniform(0, 1)
        span = rng.choice([2, 25, 300])
        lines = [(b0 * (1 + rng.uniform(-1e-3, 1e-3)) if j else b0,
                  c0 + (rng.uniform(-span, span) if j else 0.0),
                  10 ** rng.uniform(-6, 1.5), 10 ** rng.uniform(-3, 0)) for j in range(32)]
        _, zmax = series(np.array([1e9]), lines, two_nodes(), KW)
        if zmax > WZMAX:
            continue
        for lo, hi, K in [(WNEAR, WFAR, KW), (WFAR, 30 * WFAR, KWF)]:
            xs = np.concatenate([np.linspace(lo * zmax, hi * zmax, 200),
                                 -np.linspace(lo * zmax, hi * zmax, 200)])
            bins = c0 + xs / b0
            ok = np.ones(bins.size, bool)
            for b, cen, y, s in lines:
                ok &= ((bins - cen) * b) ** 2 + y * y >= 2500.0
            if not ok.any():
                continue
            got, _ = series(bins[ok], lines, two_nodes(), KW, K)
            ref = lorentz_direct(bins[ok], lines, two_nodes())
            worst[K] = max(worst[K], np.max(np.abs(got - ref) / ref))
    assert worst[KW] <= 1e-7 and worst[KWF] <= 1e-7, worst


def test_kernel_uses_the_tested_bounds():
    """The FP32C kernel's series and ring constants are the ones the tests
    above hold to their bounds (read from its source, so that a change to
    either side without the other fails here)."""
    src = open(os.path.join(os.path.dirname(__file__), "..", "paper_2101_02005_gb300", "csrc",
                            "hk_gather_f32.cu")).read()

    def has(pattern):
        assert re.search(pattern, src), pattern

    def num(x):
        return r"%s(?:\.0*)?f" % re.escape(repr(float(x)).rstrip("0").rstrip("."))

    has(r"constexpr int KMP2 = %d, KMP4 = %d;" % (K2, K4))
    assert K3 == K4   # the 12-term two-node form reuses KMP4
    has(r"const bool ok4 = base & \(q\.y <= %s\) & \(fabsf\(d\) <= %s\);" % (num(Y4), num(D4)))
    has(r"ok2 = base & \(zz <= %s\), ok3 = base & \(zz <= %s\);" % (num(Z2 ** 2), num(Z3 ** 2)))
    has(r"mode == 3 \? KMP4 : KMP2")
    has(r"constexpr int KW = %d, KWF = %d;" % (KW, KWF))
    has(r"!\(zm <= %s\)" % num(WZMAX))
    has(r"left_of\(%s \* zm\), gr = right_of\(%s \* zm\)" % (num(WNEAR), num(WNEAR)))
    has(r"left_of\(%s \* zm\), gr4 = right_of\(%s \* zm\)" % (num(WFAR), num(WFAR)))
    m = re.search(r"fmaxf\(([0-9.]+)f, ([0-9.]+)f - __logf\(y\)\)", src)
    assert m and float(m.group(1)) == RING_MIN
    assert abs(float(m.group(2)) - np.log(RING_C)) < 1e-6


# The float core rule: the trapezoid rule of step h = 1/2 with the pole
# correction (Chiarella and Reichel 1968; Matta and Reichel 1971), on the
# nodes n = -8 .. 9 of the lattice chosen so that no node lies within h/4 of x.
CORE_N0, CORE_N1, CORE_H, CORE_YCORR = -8, 9, 0.5, 2.0


def core_rule(x, y):
    """Re w(x + iy) by the truncated trapezoid rule with its pole term, in
    complex FP64: w(z) ~ (i h / pi) sum_n e^{-t_n^2} / (z - t_n)
    + 2 e^{-z^2} / (1 -+ e^{-2 pi i z / h}) (minus on the lattice t_n = n h,
    plus on t_n = (n + 1/2) h; the pole term only for y < 2)."""
    z = x + 1j * y
    fr = (x / CORE_H) % 1.0
    shift = ~((fr > 0.25) & (fr < 0.75))
    off = np.where(shift, 0.5, 0.0)
    s = np.zeros(x.shape, complex)
    for n in range(CORE_N0, CORE_N1 + 1):
        t = (n + off) * CORE_H
        s += np.exp(-t * t) / (z - t)
    w = 1j * CORE_H / np.pi * s
    e = np.exp(-2j * np.pi * z / CORE_H)
    pole = 2.0 * np.exp(-z * z) / np.where(shift, 1.0 + e, 1.0 - e)
    w = w + np.where(y < CORE_YCORR, pole, 0.0)
    return w.real


def test_core_rule_meets_its_bound():
    """18 nodes over r2 < 64 (x >= 0, y from 1e-6 to 8): within 2e-8 of Re w."""
    rng = np.random.default_rng(16)
    r2 = rng.uniform(0, 64, 400000)
    y = np.concatenate([10 ** rng.uniform(-6, np.log10(8), 200000), rng.uniform(0, 8, 200000)])
    ok = y * y < r2
    y, r2 = y[ok], r2[ok]
    x = np.sqrt(r2 - y * y)
    got = core_rule(x, y)
    ref = scipy_special.wofz(x + 1j * y).real
    assert np.max(np.abs(got - ref) / ref) <= 2e-8


def test_core_rule_matches_the_kernel_source():
    """The float core loop takes the nodes, step, lattice rule and pole-term
    range that the test above holds to its bound."""
    src = open(os.path.join(os.path.dirname(__file__), "..", "paper_2101_02005_gb300", "csrc",
                            "hk_internal.cuh")).read()
    body = src[src.index("core_re(R x, R y)"):src.index("// Re w for any band")]
    fl = body[body.index("if constexpr (sizeof(R) == 4)"):body.index("} else {")]
    assert "for (int n = %d; n <= %d; ++n)" % (CORE_N0, CORE_N1) in fl
    assert "R u = ax * R(%d);" % round(1 / CORE_H) in body
    assert "bool sh = !(fr > R(0.25) && fr < R(0.75));" in body
    assert "if (y < R(%d)) {" % CORE_YCORR in body


# The Gauss-Hermite bands by r2 = x^2 + y^2: (nodes, lower r2 bound, upper
# r2 bound, the relative error each is held to).
GH_BANDS = [(1, 1.5e6, 1e12, 1.0e-6), (2, 2500.0, 1.5e6, 4.1e-7), (3, 200.0, 2500.0, 7e-7),
            (4, 64.0, 200.0, 1.0e-6)]


def test_gauss_hermite_bands_meet_their_bounds():
    """Each band's n-node Gauss-Hermite rule for w = (i/pi) int e^{-t^2}/(z - t) dt
    (nodes and weights from numpy) is within its stated relative error of
    scipy's Re w over the band, y from 1e-9 sqrt(r2) to sqrt(r2)."""
    rng = np.random.default_rng(17)
    for n, lo, hi, bound in GH_BANDS:
        t, w = np.polynomial.hermite.hermgauss(n)
        # log-uniform over the band, plus dense points on its lower edge, where
        # each rule's error peaks
        r2 = np.concatenate([np.exp(rng.uniform(np.log(lo), np.log(hi), 180000)),
                             np.full(20000, lo)])
        f = np.concatenate([10 ** rng.uniform(-9, 0, 100000), rng.uniform(0, 1, 100000)])
        rng.shuffle(f)
        y = np.sqrt(r2) * f
        x = np.sqrt(np.maximum(r2 - y * y, 0.0))
        z = x + 1j * y
        got = (1j / np.pi * sum(wj / (z - tj) for tj, wj in zip(t, w))).real
        ref = scipy_special.wofz(z).real
        keep = ref > 0
        err = np.max(np.abs(got[keep] - ref[keep]) / ref[keep])
        assert err <= bound * (1 + 1e-3), (n, err)


def test_band_limits_match_the_kernel_source():
    src = open(os.path.join(os.path.dirname(__file__), "..", "paper_2101_02005_gb300", "csrc",
                            "hk_internal.cuh")).read()
    m = re.search(r"core = R\(([0-9.e]+)\), gh4 = R\(([0-9.e]+)\), gh3 = R\(([0-9.e]+)\), "
                  r"gh2 = R\(([0-9.e]+)\);", src)
    assert m, "BandLimits"
    core, gh4, gh3, gh2 = (float(v) for v in m.groups())
    assert (gh2, gh3, gh4, core) == tuple(b[1] for b in GH_BANDS)


def test_round_series_case_takes_each_form():
    """The GPU parity case for the round series (tests/parity.py) builds, in
    each cluster kind, 32-line rounds that meet exactly one form's conditions
    as the kernel decides them: a shared centre bin, then four nodes (every
    y <= 1.2 and |d| <= 0.2), else two nodes with 7 terms (every |z| <= 3),
    else 12 terms (every |z| <= 7), else no series."""
    import oracle
    from parity import ROUND_SERIES_GAMMA, round_series_case
    L, grid = round_series_case(31)
    nu_min, dnu, _ = grid.astuple()
    aD, GL = oracle.widths(L.nu0, L.gamma_ref, L.n_T, 1500.0, 1.0, L.mass_amu)
    y_all = GL / aD
    b_all = dnu / aD                           # x step per bin
    u = (L.nu0 - nu_min) / dnu
    c_all = np.rint(u)
    rn_all = u - c_all                         # centre offset from the nearest bin
    t = 1.0 / np.sqrt(2.0)
    forms = []
    for r in range(L.n // 32):
        s = slice(32 * r, 32 * r + 32)
        c, y, b, rn = c_all[s], y_all[s], b_all[s], rn_all[s]
        assert np.all(c == c[0])
        d = (rn[0] - rn) * b
        beta = b / b[0]
        zz = np.maximum(((t - d) / beta) ** 2, ((-t - d) / beta) ** 2) + (y / beta) ** 2
        if np.all(y <= Y4) and np.all(np.abs(d) <= D4):
            forms.append(4)
        elif np.all(zz <= Z2 * Z2):
            forms.append(2)
        elif np.all(zz <= Z3 * Z3):
            forms.append(3)
        else:
            forms.append(0)
    # clusters of 4 rounds cycle through the widths: four nodes, 7 terms, 12 terms, none
    assert len(ROUND_SERIES_GAMMA) == 4
    assert forms == ([4] * 4 + [2] * 4 + [3] * 4 + [0] * 4) * 4
