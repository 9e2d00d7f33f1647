"""Seeded synthetic line lists and workloads shaped like the paper's.

This module holds no arithmetic of the opacity method itself: it only draws
random line parameters and describes grids and (T, P) points.  Both the CUDA
path and the FP64 oracle take their inputs from here.

The paper's workloads (the ExoMol BT2 water list of Sect. 3.5, the DACE
molecule and atom tables) are not available; these draws stand in for them
with the distributions of the benchmark configurations:

* line centres nu0 uniform over a range, optionally in 100 cm^-1 windows whose
  line counts follow a log-normal (sigma = 1.5) so the line density is uneven;
* S_ref log-uniform, E'' exponential, gamma_ref and n_T uniform;
* for atom-like lists an Einstein A uniform on [1e6, 1e9] s^-1;
* Q(T) = 0.1 T^1.5 as the caller-supplied partition function.

Every field comes from its own counter-based (Philox) stream keyed by
(seed, field id), so any subset of fields can be redrawn identically.
Line centres are produced already sorted inside each window by the
order-statistics construction (normalised partial sums of exponential
spacings), so no sort of a 1e8-element array is needed; ``sort=False`` draws
independent uniforms instead (unsorted input).
"""
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

SEED_BASE = 2101020050
_FIELDS = {"nu0": 1, "S_ref": 2, "E_low": 3, "gamma_ref": 4, "n_T": 5, "A": 6, "g_up": 7,
           "counts": 8, "gamma_self": 9, "delta": 10, "grad": 100}


def stream(seed: int, fld: str) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[seed & 0xFFFFFFFFFFFFFFFF, _FIELDS[fld]]))


def partition_function(T):
    """Q(T) = 0.1 T^1.5, the configs' stand-in for a tabulated Q."""
    return 0.1 * np.power(T, 1.5)


def dlnQ_dT(T):
    return 1.5 / np.asarray(T, dtype=np.float64)


def lognormal_window_counts(n: int, nwin: int, seed: int, sigma: float = 1.5) -> np.ndarray:
    """Line counts per window: weights ~ LogNormal(0, sigma), rounded to sum
    exactly n by the largest-remainder rule."""
    w = stream(seed, "counts").lognormal(0.0, sigma, size=nwin)
    q = w / w.sum() * n
    base = np.floor(q).astype(np.int64)
    rem = n - int(base.sum())
    if rem > 0:
        order = np.argsort(-(q - base), kind="stable")
        base[order[:rem]] += 1
    return base


def _sorted_uniform_into(rng: np.random.Generator, out: np.ndarray, lo: float, hi: float):
    """Sorted U[lo, hi) sample of size out.size via normalised partial sums of
    k + 1 exponential spacings (Renyi's representation of order statistics)."""
    k = out.size
    if k == 0:
        return
    e = rng.standard_exponential(k + 1)
    np.cumsum(e, out=e)
    np.multiply(e[:k], (hi - lo) / e[k], out=out)
    out += lo


@dataclass
class LineList:
    nu0: np.ndarray          # f64 [n], cm^-1
    S_ref: np.ndarray        # f32 [n], cm/molecule at T_ref
    E_low: np.ndarray        # f32 [n], cm^-1
    gamma_ref: np.ndarray    # f32 [n], cm^-1 / bar at T_ref
    n_T: np.ndarray          # f32 [n]
    mass_amu: float
    A: Optional[np.ndarray] = None     # f32 [n], s^-1
    g_up: Optional[np.ndarray] = None  # f32 [n]
    s_mode: int = 0
    sorted: bool = True
    gamma_self: Optional[np.ndarray] = None  # f32 [n], HITRAN self broadening (gamma_ref = air)
    delta: Optional[np.ndarray] = None       # f32 [n], pressure shift, cm^-1 / P_ref

    @property
    def n(self) -> int:
        return int(self.nu0.size)

    def as_oracle(self) -> dict:
        d = dict(nu0=self.nu0, S_ref=self.S_ref, E_low=self.E_low, gamma_ref=self.gamma_ref,
                 n_T=self.n_T, mass_amu=self.mass_amu, s_mode=self.s_mode, sorted=self.sorted)
        if self.A is not None:
            d["A"] = self.A
        if self.g_up is not None:
            d["g_up"] = self.g_up
        if self.gamma_self is not None:
            d["gamma_self"] = self.gamma_self
        if self.delta is not None:
            d["delta"] = self.delta
        return d

    def subset(self, idx) -> "LineList":
        f = lambda a: None if a is None else a[idx]
        return LineList(self.nu0[idx], self.S_ref[idx], self.E_low[idx], self.gamma_ref[idx],
                        self.n_T[idx], self.mass_amu, f(self.A), f(self.g_up), self.s_mode,
                        self.sorted, f(self.gamma_self), f(self.delta))


def make_lines(n: int, nu_lo: float, nu_hi: float, seed: int, mass_amu: float,
               S_range: Tuple[float, float] = (1e-30, 1e-19), E_mean: float = 3000.0,
               gamma_range: Tuple[float, float] = (0.01, 0.1),
               nT_range: Tuple[float, float] = (0.3, 0.8),
               A_range: Optional[Tuple[float, float]] = None,
               windows: Optional[int] = None, window_sigma: float = 1.5,
               sort: bool = True, hitran: bool = False) -> LineList:
    """Draw a line list.  ``windows``: number of equal-width windows with
    log-normal line counts (None: one window)."""
    n = int(n)
    r_nu = stream(seed, "nu0")
    if windows:
        counts = lognormal_window_counts(n, windows, seed, window_sigma)
        edges = np.linspace(nu_lo, nu_hi, windows + 1)
    else:
        counts = np.array([n], np.int64)
        edges = np.array([nu_lo, nu_hi])
    nu0 = np.empty(n, np.float64)
    pos = 0
    for w, k in enumerate(counts.tolist()):
        if sort:
            _sorted_uniform_into(r_nu, nu0[pos:pos + k], edges[w], edges[w + 1])
        else:
            r_nu.random(out=nu0[pos:pos + k])
            nu0[pos:pos + k] *= edges[w + 1] - edges[w]
            nu0[pos:pos + k] += edges[w]
        pos += k
    f32 = np.float32
    # S_ref = 10^U[log10 S0, log10 S1], drawn in float32 in place
    S_ref = np.empty(n, f32)
    stream(seed, "S_ref").random(dtype=f32, out=S_ref)
    l0, l1 = np.log(S_range[0]), np.log(S_range[1])
    S_ref *= f32(l1 - l0)
    S_ref += f32(l0)
    np.exp(S_ref, out=S_ref)
    E_low = np.empty(n, f32)
    stream(seed, "E_low").standard_exponential(dtype=f32, out=E_low)
    E_low *= f32(E_mean)
    gamma = np.empty(n, f32)
    stream(seed, "gamma_ref").random(dtype=f32, out=gamma)
    gamma *= f32(gamma_range[1] - gamma_range[0])
    gamma += f32(gamma_range[0])
    n_T = np.empty(n, f32)
    stream(seed, "n_T").random(dtype=f32, out=n_T)
    n_T *= f32(nT_range[1] - nT_range[0])
    n_T += f32(nT_range[0])
    A = None
    if A_range is not None:
        A = np.empty(n, f32)
        stream(seed, "A").random(dtype=f32, out=A)
        A *= f32(A_range[1] - A_range[0])
        A += f32(A_range[0])
    gs = dl = None
    if hitran:   # HITRAN-like air/self widths and pressure shifts
        gs = np.empty(n, f32)
        stream(seed, "gamma_self").random(dtype=f32, out=gs)
        gs *= f32(0.4)
        gs += f32(0.1)
        dl = np.empty(n, f32)
        stream(seed, "delta").random(dtype=f32, out=dl)
        dl *= f32(0.03)
        dl -= f32(0.02)
    return LineList(nu0, S_ref, E_low, gamma, n_T, float(mass_amu), A=A, sorted=bool(sort),
                    gamma_self=gs, delta=dl)


@dataclass
class Grid:
    nu_min: float
    dnu: float
    nbins: int

    def astuple(self):
        return (self.nu_min, self.dnu, self.nbins)


@dataclass
class Workload:
    name: str
    species: List[LineList]
    grid: Grid
    cut: float
    T: np.ndarray
    P: np.ndarray
    paired: bool = False          # (T[k], P[k]) pairs instead of the T x P product
    extra: dict = field(default_factory=dict)

    def states(self) -> List[Tuple[float, float]]:
        if self.paired:
            return list(zip(self.T.tolist(), self.P.tolist()))
        return [(t, p) for t in self.T.tolist() for p in self.P.tolist()]


def config(k: int, scale: float = 1.0, sort: bool = True) -> Workload:
    """The five benchmark workloads; ``scale`` < 1 shrinks line counts (and
    nothing else) for quick runs."""
    seed = SEED_BASE + k
    s = lambda n: max(1, int(round(n * scale)))
    if k == 0:
        L = make_lines(s(1e4), 0.0, 3000.0, seed, 18.0, sort=sort)
        return Workload("c0: 1e4 lines, 0-3000 cm-1 @ 0.1, cut 25, T=1000 K, P=1 bar", [L],
                        Grid(0.0, 0.1, 30000), 25.0, np.array([1000.0]), np.array([1.0]),
                        paired=True)
    if k == 1:
        L = make_lines(s(5e8), 0.0, 30000.0, seed, 18.0, windows=300, sort=sort)
        return Workload("c1: 5e8 lines (log-normal density), 0-30000 cm-1 @ 0.1, cut 25, "
                        "T=1500 K, P=1 bar", [L], Grid(0.0, 0.1, 300000), 25.0,
                        np.array([1500.0]), np.array([1.0]), paired=True)
    if k == 2:
        L = make_lines(s(1e8), 0.0, 30000.0, seed, 18.0, windows=300, sort=sort)
        atoms = make_lines(s(1e5), 0.0, 1e5, seed + 1000, 56.0, S_range=(1e-25, 1e-15),
                           A_range=(1e6, 1e9), sort=sort)
        return Workload("c2: 1e8 lines 0-30000 @ 0.01, cut 100, T=2000 K, P=0.1 bar; "
                        "atoms 1e5 lines, no cut, 0-1e5 @ 0.01", [L],
                        Grid(0.0, 0.01, 3000000), 100.0, np.array([2000.0]),
                        np.array([0.1]), paired=True,
                        extra=dict(atoms=atoms, atom_grid=Grid(0.0, 0.01, 10000000),
                                   atom_cut=0.0))
    if k == 3:
        ns = [1e5, 1e6, 5e6, 2e7]
        ms = [18.0, 16.0, 44.0, 28.0]
        sp = [make_lines(s(n), 0.0, 20000.0, seed + 10 * j, m, sort=sort)
              for j, (n, m) in enumerate(zip(ns, ms))]
        return Workload("c3: 4 species (1e5/1e6/5e6/2e7 lines), 0-20000 @ 0.01, cut 100, "
                        "20 T x 10 P", sp, Grid(0.0, 0.01, 2000000), 100.0,
                        np.logspace(np.log10(100.0), np.log10(3000.0), 20),
                        np.logspace(-6.0, 2.0, 10))
    if k == 4:
        L = make_lines(s(1e6), 0.0, 5000.0, seed, 18.0, sort=sort)
        return Workload("c4: 1e6 lines, 0-5000 @ 0.01, cut 25, 16 paired (T, P)", [L],
                        Grid(0.0, 0.01, 500000), 25.0,
                        np.logspace(np.log10(300.0), np.log10(2500.0), 16),
                        np.logspace(-3.0, 1.0, 16), paired=True)
    raise ValueError(k)


def upstream_grad(nTP: int, nbins: int, seed: int) -> np.ndarray:
    """Upstream gradient g ~ N(0, 1) per bin and (T, P) point (seed + 100)."""
    return stream(seed + 100, "grad").standard_normal((nTP, nbins)).astype(np.float32)
