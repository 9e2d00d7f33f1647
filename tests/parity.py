"""Parity metrics between a GPU result and the FP64 oracle.

The bar (benchmark statement): relative L1 error <= 1e-5 and per-bin relative
error <= 1e-4 over the bins where the oracle's sigma exceeds 1e-10 * max(sigma).
"""
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
