"""Parity at the full benchmark sizes, on sampled outputs.

Each workload runs at its full line count through the same call and options
the benchmark uses (FP32-compensated, FP64 output, one launch per (T, P) or
one batched launch).  The oracle then computes sigma one bin at a time at a
seeded sample of bins (plus the bin of the array's maximum), summing only
the lines whose centres lie within the cut of that bin (the oracle's cut
predicate still decides each pair).  The per-bin bar is the benchmark's:
relative error <= 1e-4 on bins above 1e-10 of the array's maximum; the
relative L1 bar (1e-5) is applied to the sample.

Gradients (config 4, 16 (T, P) points) are checked per line against the
oracle's adjoint of single-line lists (a line's gradient depends only on
that line and the upstream gradient), and dL/dT, dL/dP against central
finite differences (h = 1e-3 relative, with one Richardson step) of
L = sum g sigma computed by the FP64 GPU forward, itself checked against the
oracle on sampled bins.
"""
import concurrent.futures as cf
import gc
import os

import numpy as np
import pytest

import oracle
from parity import BIN_TOL, L1_TOL, MASK_REL, record, sampled_errors, sigma_errors
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


def _free():
    gc.collect()
    torch.cuda.empty_cache()




def check_sampled(gpu_full, L, grid, state, cut, seed, what):
    """gpu_full: the whole sigma array (host, f64).  Returns the sample's errors."""
    err = sampled_errors(gpu_full, L, grid, state, cut, seed)
    record(what, err)
    assert err["n_mask"] >= 8, (what, err)
    assert err["max_bin"] <= BIN_TOL and err["l1"] <= L1_TOL, (what, err)
    # bins under the mask: absolute error within the per-bin bar at the mask level
    assert err["below_mask_abs"] <= BIN_TOL * MASK_REL * err["ref_max"], (what, err)
    return err


def check_local(gpu_full, L, grid, state, cut, seed, what, nb=30, floor=1e-25):
    """The per-bin bar relative to each bin's own value, on bins far below the
    array-wide mask but far above the FP32C floor (contributions ~2^-126 below
    the largest line value are flushed): seeded bins with sigma > floor x the
    array's maximum.  The array-wide mask of the configurations at high T
    (maxima ~1e80) leaves most of the array to the loose absolute check; this
    holds every part of the sums (every series, band and batch path) to 1e-4."""
    from parity import oracle_bins
    g = np.asarray(gpu_full, dtype=np.float64)
    cand = np.flatnonzero(g > floor * g.max())
    if cand.size == 0:
        return
    rng = np.random.default_rng(seed)
    bins = np.sort(rng.choice(cand, size=min(nb, cand.size), replace=False))
    ref = oracle_bins(L, grid, state, cut, bins)
    rel = np.abs(g[bins] - ref) / ref
    record(what + " (bins above 1e-25 of the maximum, own value)",
           dict(n=int(bins.size), max_bin=float(rel.max())))
    assert np.all(ref > 0) and rel.max() <= BIN_TOL, (what, float(rel.max()),
                                                      int(bins[np.argmax(rel)]))


def test_config1_full(hk):
    """5e8 lines, 0-30000 cm^-1 at 0.1, cut 25, T = 1500 K, P = 1 bar: the
    benchmark's own launch; plus the FP64 GPU form on every 10th line."""
    w = synth.config(1)
    L = w.species[0]
    T, P = w.states()[0]
    state = (T, P, float(Q(T)), QREF)
    D = hk.DeviceLines.from_host(L)
    grid = hk.make_grid(*w.grid.astuple())
    st = hk.make_state(T, P, float(Q(T)))
    sig = hk.hk_cross_section(D, grid, st, hk.make_opts(QREF, w.cut, hk.HK_FP32C,
                                                        flags=hk.HK_SIGMA_F64))
    hk.hk_sync_status()
    sig = sig.cpu().numpy()
    check_sampled(sig, L, w.grid.astuple(), state, w.cut, 11, "c1 fp32c")
    check_local(sig, L, w.grid.astuple(), state, w.cut, 21, "c1 fp32c")
    # the benchmark's end-to-end call: the list streamed from page-locked host
    # memory in the default blocks (2^23 .. 2^26 lines, a ragged last one)
    del D
    _free()
    H = hk.HostLines.from_host(L)
    sh = hk.hk_cross_section_host(H, grid, st, hk.make_opts(QREF, w.cut, hk.HK_FP32C,
                                                            flags=hk.HK_SIGMA_F64))
    hk.hk_sync_status()
    del H
    e = sigma_errors(sh.numpy(), sig)
    assert e["max_bin"] <= 1e-6, ("c1 host-streamed vs device-resident", e)
    check_sampled(sh.numpy(), L, w.grid.astuple(), state, w.cut, 13, "c1 fp32c host-streamed")
    L10 = L.subset(np.arange(0, L.n, 10))
    D10 = hk.DeviceLines.from_host(L10)
    s64 = hk.hk_cross_section(D10, grid, st, hk.make_opts(QREF, w.cut, hk.HK_FP64))
    hk.hk_sync_status()
    check_sampled(s64.cpu().numpy(), L10, w.grid.astuple(), state, w.cut, 12, "c1 fp64 1/10")
    del D10, L, L10, w
    _free()


def test_config2_full(hk):
    """1e8 lines at 0.01 over 0-30000 with a 100 cm^-1 cut (T = 2000 K,
    P = 0.1 bar), and the atom-like list: 1e5 lines with natural broadening,
    no cut, over the whole 0-1e5 cm^-1 grid at 0.01 (1e7 bins)."""
    w = synth.config(2)
    L = w.species[0]
    T, P = w.states()[0]
    state = (T, P, float(Q(T)), QREF)
    st = hk.make_state(T, P, float(Q(T)))
    D = hk.DeviceLines.from_host(L)
    sig = hk.hk_cross_section(D, hk.make_grid(*w.grid.astuple()), st,
                              hk.make_opts(QREF, w.cut, hk.HK_FP32C, flags=hk.HK_SIGMA_F64))
    hk.hk_sync_status()
    check_sampled(sig.cpu().numpy(), L, w.grid.astuple(), state, w.cut, 21, "c2 molecular")
    del D, sig
    _free()
    A = w.extra["atoms"]
    ag = w.extra["atom_grid"]
    DA = hk.DeviceLines.from_host(A)
    sa = hk.hk_cross_section(DA, hk.make_grid(*ag.astuple()), st,
                             hk.make_opts(QREF, 0.0, hk.HK_FP32C, flags=hk.HK_SIGMA_F64))
    hk.hk_sync_status()
    check_sampled(sa.cpu().numpy(), A, ag.astuple(), state, 0.0, 22, "c2 atoms")
    del DA, sa
    _free()


def test_config3_full_batched(hk):
    """4 species (1e5, 1e6, 5e6, 2e7 lines) x 20 T x 10 P = 800 sigma arrays of
    2e6 bins in one batched launch; sampled bins of the extreme and middle
    (T, P) points of every species."""
    w = synth.config(3)
    species = [hk.DeviceLines.from_host(s) for s in w.species]
    states_tp = [(t, p) for t in w.T for p in w.P]
    states = [hk.make_state(t, p, float(Q(t))) for t, p in states_tp]
    grid = hk.make_grid(*w.grid.astuple())
    out = hk.hk_cross_section_batched(species, states, grid,
                                      hk.make_opts(QREF, w.cut, hk.HK_FP32C,
                                                   flags=hk.HK_SIGMA_F64))
    hk.hk_sync_status()
    nP = len(w.P)
    picks = [0, nP - 1, len(states_tp) - nP, len(states_tp) - 1, 10 * nP + 5]
    for s, L in enumerate(w.species):
        for k in picks:
            t, p = states_tp[k]
            sig = out[s, k].cpu().numpy()
            check_sampled(sig, L, w.grid.astuple(), (t, p, float(Q(t)), QREF), w.cut,
                          300 + 10 * s + k, f"c3 species {s} T={t:.0f} P={p:.1e}")
    del out, species
    _free()


def test_config4_full_backward(hk):
    """1e6 lines, 0-5000 at 0.01, cut 25, 16 (T, P) points, upstream gradient
    N(0, 1) per bin: per-line dL/dS_ref, dL/dgamma_ref on sampled lines
    against the oracle's adjoint, dL/dT and dL/dP against central finite
    differences of the FP64 GPU forward at four of the points."""
    w = synth.config(4)
    L = w.species[0]
    pts = w.states()
    nTP = len(pts)
    grid = hk.make_grid(*w.grid.astuple())
    g = synth.upstream_grad(nTP, w.grid.nbins, synth.SEED_BASE + 4)
    D = hk.DeviceLines.from_host(L)
    states = [hk.make_state(t, p, float(Q(t)), float(synth.dlnQ_dT(t))) for t, p in pts]
    dT, dP, dS, dG = hk.hk_cross_section_backward(D, grid, states, hk.make_opts(QREF, w.cut),
                                                  torch.from_numpy(g).cuda())
    hk.hk_sync_status()
    dT, dP, dS, dG = (x.cpu().numpy() for x in (dT, dP, dS, dG))
    assert np.all(np.isfinite(dS)) and np.all(np.isfinite(dG))

    # per-line gradients on a seeded sample of lines (plus the largest |dS|)
    rng = np.random.default_rng(41)
    idx = np.unique(np.concatenate([rng.choice(L.n, 40, replace=False),
                                    np.argsort(-np.abs(dS))[:8]]))
    g64 = g.astype(np.float64)

    def one(l):
        sub = L.subset(slice(l, l + 1)).as_oracle()
        oS, oG = np.zeros(1), np.zeros(1)
        for k, (t, p) in enumerate(pts):
            oracle.backward(sub, w.grid.astuple(),
                            (t, p, float(Q(t)), QREF, float(synth.dlnQ_dT(t))), w.cut, g64[k],
                            oS, oG, nthreads=1)
        return oS[0], oG[0]

    with cf.ThreadPoolExecutor(max(1, min(16, os.cpu_count() or 1))) as ex:
        ref = np.array(list(ex.map(one, idx.tolist())))
    oS, oG = ref[:, 0], ref[:, 1]
    eS = float(np.linalg.norm(dS[idx] - oS) / np.linalg.norm(oS))
    eG = float(np.linalg.norm(dG[idx] - oG) / np.linalg.norm(oG))
    record("c4 dL/dS_ref, dL/dgamma_ref (sampled lines) vs oracle adjoint",
           dict(n=int(idx.size), rel_l2_dS=eS, rel_l2_dG=eG))
    assert eS <= 1e-4 and eG <= 1e-4, (eS, eG)

    # dL/dT, dL/dP against the oracle's FP64 gradient: with the upstream
    # gradient kept on a 1500-bin window (zero elsewhere) only the lines within
    # the cut of the window contribute, so the oracle's adjoint of that part of
    # the full list gives the exact reference at two of the points
    nu_min, dnu, nbins = w.grid.astuple()
    for k, lo in ((3, 120000), (12, 361000)):
        gw = np.zeros((1, nbins), np.float32)
        gw[0, lo:lo + 1500] = g[k, lo:lo + 1500]
        wT, wP, _, _ = hk.hk_cross_section_backward(D, grid, [states[k]], hk.make_opts(QREF, w.cut),
                                                    torch.from_numpy(gw).cuda())
        hk.hk_sync_status()
        a = int(np.searchsorted(L.nu0, nu_min + lo * dnu - w.cut - 2 * dnu, "left"))
        b = int(np.searchsorted(L.nu0, nu_min + (lo + 1500) * dnu + w.cut + 2 * dnu, "right"))
        sub = L.subset(slice(a, b)).as_oracle()
        t, p = pts[k]
        # the oracle on the window's own grid (bins outside it carry g = 0)
        _, _, oT, oP = oracle.backward(sub, (nu_min + lo * dnu, dnu, 1500),
                                       (t, p, float(Q(t)), QREF, float(synth.dlnQ_dT(t))),
                                       w.cut, gw[0, lo:lo + 1500].astype(np.float64),
                                       np.zeros(b - a), np.zeros(b - a))
        gT, gP = float(wT.cpu().numpy()[0]), float(wP.cpu().numpy()[0])
        record(f"c4 dL/dT, dL/dP point {k} (1500-bin window) vs oracle FP64 gradient",
               dict(lines=int(b - a), rel_dT=abs(gT - oT) / abs(oT), rel_dP=abs(gP - oP) / abs(oP)))
        assert abs(gT - oT) <= 1e-4 * abs(oT), (k, gT, oT)
        assert abs(gP - oP) <= 1e-4 * abs(oP), (k, gP, oP)

    # dL/dT, dL/dP: central differences of the FP64 forward
    o64 = hk.make_opts(QREF, w.cut, hk.HK_FP64)
    gd = torch.from_numpy(g64).cuda()

    def loss(k, t, p):
        s = hk.hk_cross_section(D, grid, hk.make_state(t, p, float(Q(t))), o64)
        return float(torch.dot(s, gd[k]).item())

    # Central differences at h = 1e-3 relative and h/2, combined by one
    # Richardson step: the Boltzmann factor's curvature (c2 E''/T^2 h up to
    # ~0.1 at 300 K) leaves the plain O(h^2) difference off by up to a few
    # per cent, the extrapolated one by O(h^4) ~ 1e-5.
    def fd(f, x, h):
        d1 = (f(x + h) - f(x - h)) / (2 * h)
        d2 = (f(x + h / 2) - f(x - h / 2)) / h
        return (4 * d2 - d1) / 3

    for k in (0, 5, 10, 15):
        t, p = pts[k]
        fdT = fd(lambda x: loss(k, x, p), t, 1e-3 * t)
        fdP = fd(lambda x: loss(k, t, x), p, 1e-3 * p)
        record(f"c4 dL/dT, dL/dP point {k} vs Richardson central differences",
               dict(rel_dT=abs(dT[k] - fdT) / abs(fdT), rel_dP=abs(dP[k] - fdP) / abs(fdP)))
        assert abs(dT[k] - fdT) <= 1e-4 * abs(fdT), (k, dT[k], fdT)
        assert abs(dP[k] - fdP) <= 1e-4 * abs(fdP), (k, dP[k], fdP)
    hk.hk_sync_status()

    # the FP64 forward used above, against the oracle at one point
    t, p = pts[5]
    s = hk.hk_cross_section(D, grid, hk.make_state(t, p, float(Q(t))), o64)
    hk.hk_sync_status()
    check_sampled(s.cpu().numpy(), L, w.grid.astuple(), (t, p, float(Q(t)), QREF), w.cut, 45,
                  "c4 fp64 forward")
    del s
    # the FP32C forward of all 16 points in one batched launch, at three points
    out = hk.hk_cross_section_batched([D], states, grid,
                                      hk.make_opts(QREF, w.cut, hk.HK_FP32C, flags=hk.HK_SIGMA_F64))
    hk.hk_sync_status()
    for k in (0, 5, 15):
        t, p = pts[k]
        check_sampled(out[0, k].cpu().numpy(), L, w.grid.astuple(), (t, p, float(Q(t)), QREF),
                      w.cut, 460 + k, f"c4 fp32c forward point {k} (batched)")
    del D, out
    _free()
