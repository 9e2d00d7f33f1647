"""Parity metrics between a GPU result and the FP64 oracle.

The bar (benchmark statement): relative L1 error <= 1e-5 and per-bin relative
error <= 1e-4 over the bins where the oracle's sigma exceeds 1e-10 * max(sigma).
"""
import concurrent.futures as cf
import json
import os

import numpy as np

L1_TOL = 1e-5
BIN_TOL = 1e-4
MASK_REL = 1e-10


def sigma_errors(gpu, ref, mask_rel=MASK_REL, ref_max=None):
    """ref_max: max(sigma) of the whole array when gpu/ref are a window of it."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert gpu.shape == ref.shape
    mx = np.max(np.abs(ref)) if ref.size else 0.0
    if ref_max is not None:
        mx = max(mx, ref_max)
    m = ref > mask_rel * mx
    if not np.any(m):
        return dict(l1=0.0, max_bin=0.0, n_mask=0, frac_mask=0.0)
    d = np.abs(gpu[m] - ref[m])
    return dict(l1=float(d.sum() / np.abs(ref[m]).sum()),
                max_bin=float(np.max(d / np.abs(ref[m]))),
                n_mask=int(m.sum()), frac_mask=float(m.mean()))


def assert_sigma_close(gpu, ref, what="", l1=L1_TOL, per_bin=BIN_TOL, ref_max=None):
    e = sigma_errors(gpu, ref, ref_max=ref_max)
    assert np.all(np.isfinite(np.asarray(gpu, dtype=np.float64))), what
    if not (e["l1"] <= l1 and e["max_bin"] <= per_bin):
        g = np.asarray(gpu, dtype=np.float64)
        r = np.asarray(ref, dtype=np.float64)
        m = r > MASK_REL * max(np.max(np.abs(r)), ref_max or 0.0)
        rel = np.where(m, np.abs(g - r) / np.where(m, np.abs(r), 1.0), 0.0)
        i = int(np.argmax(rel))
        e["worst_bin"] = i
        e["worst"] = (float(g[i]), float(r[i]))
        e["rel_pct"] = [float(np.percentile(rel[m], q)) for q in (50, 90, 99)]
        raise AssertionError((what, e))
    return e


def oracle_sigma_max(oracle, L, grid, state, cut, top=24, halfwidth=3):
    """max(sigma) of the whole array from the oracle, evaluated only around the
    centres of the `top` lines of largest S / alpha_D (the peaks), for windowed
    comparisons of arrays too large for the oracle.  Never larger than the true
    maximum, so the mask it gives is at least as strict as the global one."""
    nu_min, dnu, nbins = grid
    T, P, Q_T, Q_ref = state
    S = oracle.line_strength(L.nu0, L.E_low, T, Q_T, Q_ref, L.mass_amu, S_ref=L.S_ref,
                             A=L.A, g_up=L.g_up, s_mode=L.s_mode)
    aD, _ = oracle.widths(L.nu0, L.gamma_ref, L.n_T, T, P, L.mass_amu, A=L.A)
    ok = (L.nu0 > 0) & (L.nu0 >= nu_min) & (L.nu0 < nu_min + nbins * dnu)
    score = np.where(ok, S / np.where(aD > 0, aD, np.inf), -1.0)
    idx = np.argsort(-score)[:top]
    best = 0.0
    for j in idx:
        c = int(round((L.nu0[j] - nu_min) / dnu))
        lo, hi = max(0, c - halfwidth), min(nbins, c + halfwidth + 1)
        if hi > lo:
            best = max(best, float(np.max(oracle.cross_section(L.as_oracle(), grid, state, cut,
                                                                lo, hi))))
    return best


def record(what, err):
    """Appends a measured error to the JSON-lines file named by HK_ERRORS_JSON
    (unset: nothing is written), for the per-configuration error table."""
    path = os.environ.get("HK_ERRORS_JSON")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"what": what, **err}) + "\n")


def assert_plinth_close(gpu, ref, base, what="", l1=L1_TOL, per_bin=BIN_TOL):
    """Parity of a plinth-removed sigma (Sect. 2.1).

    The plinth-removed value of a bin is a difference: the sum of the line
    profiles `base` (the un-removed sigma) less the sum of the lines'
    plinths, base - ref >= 0.  Each side carries the relative rounding error
    of the terms it sums, so the error of the difference is bounded relative
    to the terms, that is relative to `base`: per bin and in L1 over the
    mask base > 1e-10 max(base).  Where the difference is well conditioned
    (ref >= base / 2, condition number at most 2) the removed value is also
    held to the bar itself, per bin and in L1, relative to ref.  Returns the
    errors of both regions."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    base = np.asarray(base, dtype=np.float64)
    assert np.all(np.isfinite(gpu)), what
    m = base > MASK_REL * base.max()
    d = np.abs(gpu - ref)
    e = {"terms_l1": float(d[m].sum() / base[m].sum()),
         "terms_max_bin": float(np.max(d[m] / base[m]))}
    far = m & (ref >= 0.5 * base)
    if np.any(far):
        e["l1"] = float(d[far].sum() / ref[far].sum())
        e["max_bin"] = float(np.max(d[far] / ref[far]))
        e["n_far"] = int(far.sum())
    ok = (e["terms_l1"] <= l1 and e["terms_max_bin"] <= per_bin
          and e.get("l1", 0.0) <= l1 and e.get("max_bin", 0.0) <= per_bin)
    assert ok, (what, e)
    return e


def sample_bins(sig, seed, n_rand=16, n_above=24):
    """Seeded bins of a whole sigma array: uniform over the grid, uniform over
    the bins above the mask, the argmax, and the first and last bins (where
    to compare; the expected values come from the oracle alone)."""
    rng = np.random.default_rng(seed)
    n = sig.size
    b = set(rng.integers(0, n, n_rand).tolist())
    above = np.flatnonzero(sig > MASK_REL * sig.max())
    if above.size:
        b |= set(rng.choice(above, min(n_above, above.size), replace=False).tolist())
    b |= {0, n - 1, int(np.argmax(sig))}
    return np.array(sorted(b), dtype=np.int64)


def oracle_bins(L, grid, state, cut, bins, per_gram=False):
    """Oracle sigma at each bin of `bins`, from the lines within cut + 2 bins
    of it (all lines if there is no cut; the oracle's cut predicate still
    decides each pair); bins in parallel threads."""
    import oracle
    nu_min, dnu, nbins = grid

    def one(i):
        if cut > 0:
            nu = nu_min + i * dnu
            a = int(np.searchsorted(L.nu0, nu - cut - 2 * dnu, "left"))
            b = int(np.searchsorted(L.nu0, nu + cut + 2 * dnu, "right"))
            sub = L.subset(slice(a, b))
        else:
            sub = L
        if sub.n == 0:
            return 0.0
        return float(oracle.cross_section(sub.as_oracle(), grid, state, cut, int(i), int(i) + 1,
                                          nthreads=1, per_gram=per_gram)[0])

    with cf.ThreadPoolExecutor(max(1, min(16, os.cpu_count() or 1))) as ex:
        return np.array(list(ex.map(one, bins.tolist())))


def sampled_errors(gpu_full, L, grid, state, cut, seed):
    """Errors of a whole sigma array (host, f64) on a seeded sample of bins
    (sample_bins) against the oracle bin by bin: relative L1 and per-bin
    relative error over the sampled bins above 1e-10 of the oracle's value at
    the array's maximum, and the largest absolute error below that mask."""
    gpu_full = np.asarray(gpu_full, dtype=np.float64)
    assert np.all(np.isfinite(gpu_full))
    bins = sample_bins(gpu_full, seed)
    ref = oracle_bins(L, grid, state, cut, bins)
    g = gpu_full[bins]
    ref_max = float(ref[bins == int(np.argmax(gpu_full))][0])
    assert ref_max > 0
    m = ref > MASK_REL * ref_max
    d = np.abs(g - ref)
    return dict(n=int(bins.size), n_mask=int(m.sum()),
                max_bin=float(np.max(d[m] / ref[m])) if m.any() else 0.0,
                l1=float(d[m].sum() / ref[m].sum()) if m.any() else 0.0,
                below_mask_abs=float(d[~m].max()) if (~m).any() else 0.0, ref_max=ref_max)


# Lorentz widths gamma_ref (cm^-1) of the four cluster kinds of the round-series
# case, at 1500 K and 1 bar: y near 0.4 (the four-node series), 1.8 (two nodes,
# 7 terms), 5 (two nodes, 12 terms) and 21 (no series).
ROUND_SERIES_GAMMA = (0.05, 0.25, 0.7, 3.0)


def round_series_case(seed):
    """Short lines in 16 clusters of 128 lines within 0.02 bins of a bin centre
    (0.1 cm^-1 bins from 14000 cm^-1, 9000 bins), the clusters cycling through
    ROUND_SERIES_GAMMA, so that whole 32-line rounds share their centre bin;
    modest strengths and lower-state energies.  Returns (lines, grid)."""
    from paper_2101_02005_gb300 import synth
    rng = np.random.default_rng(seed)
    dnu, nu_min, nbins = 0.1, 14000.0, 9000
    nu0, gam = [], []
    for i, k in enumerate(np.linspace(400, nbins - 400, 16).astype(int)):
        base = nu_min + k * dnu
        nu0.extend((base + np.sort(rng.uniform(-2e-3, 2e-3, 128))).tolist())
        g = ROUND_SERIES_GAMMA[i % 4]
        gam.extend((g * rng.uniform(0.85, 1.0, 128)).tolist())
    nu0 = np.asarray(nu0)
    n = nu0.size
    L = synth.LineList(nu0, (10 ** rng.uniform(-22, -20, n)).astype(np.float32),
                       rng.exponential(300.0, n).astype(np.float32),
                       np.asarray(gam, np.float32), np.full(n, 0.5, np.float32), 18.0)
    return L, synth.Grid(nu_min, dnu, nbins)
