"""Thin ctypes binding of libhk (include/hk.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Tensors are PyTorch CUDA tensors; PyTorch provides the device
memory and the stream, nothing else.  If the library is missing, importing
this module raises -- there is no CPU fallback.
"""
import ctypes
import os
from dataclasses import dataclass
from typing import List, Optional, Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhk.so")

HK_OK, HK_EINVAL, HK_ENOMEM, HK_ECUDA, HK_ETIMEOUT, HK_ENOTSUP, HK_ERANGE, HK_ESIZE = range(8)
HK_NOALLOC_SCRATCH_BYTES = 16 << 20
HK_S_REF, HK_S_EINSTEIN_A = 0, 1
HK_FP32C, HK_FP64 = 0, 1
HK_CUT_FIXED, HK_CUT_NONE, HK_CUT_DOPPLER, HK_CUT_LORENTZ = 0, 1, 2, 3
HK_PER_GRAM = 1
HK_SIGMA_F64 = 2
HK_REMOVE_PLINTH = 4
HK_PROFILE_VOIGT, HK_PROFILE_LORENTZ, HK_PROFILE_DOPPLER, HK_PROFILE_BINNED_GAUSS = 0, 1, 2, 3

EXPORTS = ["hk_line_strength", "hk_widths", "hk_voigt_accumulate", "hk_cross_section",
           "hk_cross_section_batched", "hk_cross_section_backward", "hk_workspace_size",
           "hk_autotune", "hk_sync_status", "hk_release", "hk_strerror", "hk_last_cuda_error",
           "hk_constants", "hk_version", "hk_count_pairs", "hk_count_ring_pairs", "hk_profile",
           "hk_cross_section_noalloc", "hk_tuning", "hk_cross_section_host", "hk_set_tuning",
           "hk_noalloc_status", "hk_measure_peak"]


class hk_lines(ctypes.Structure):
    _fields_ = [("nu0", ctypes.c_void_p), ("S_ref", ctypes.c_void_p), ("A", ctypes.c_void_p),
                ("g_up", ctypes.c_void_p), ("E_low", ctypes.c_void_p),
                ("gamma_ref", ctypes.c_void_p), ("n_T", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("mass_amu", ctypes.c_double), ("s_mode", ctypes.c_int), ("sorted", ctypes.c_int),
                ("gamma_self", ctypes.c_void_p), ("delta", ctypes.c_void_p)]


class hk_grid(ctypes.Structure):
    _fields_ = [("nu_min", ctypes.c_double), ("dnu", ctypes.c_double), ("nbins", ctypes.c_int64)]


class hk_state(ctypes.Structure):
    _fields_ = [("T", ctypes.c_double), ("P", ctypes.c_double), ("Q_T", ctypes.c_double),
                ("dlnQ_dT", ctypes.c_double), ("P_self", ctypes.c_double)]


class hk_opts(ctypes.Structure):
    _fields_ = [("T_ref", ctypes.c_double), ("P_ref", ctypes.c_double),
                ("Q_Tref", ctypes.c_double), ("cut", ctypes.c_double), ("cut_mode", ctypes.c_int),
                ("precision", ctypes.c_int), ("flags", ctypes.c_uint), ("profile", ctypes.c_int)]


class HKError(RuntimeError):
    def __init__(self, fn, status):
        self.status = status
        extra = ""
        if status == HK_ECUDA:
            extra = f" (cudaError {lib().hk_last_cuda_error()})"
        super().__init__(f"{fn}: {lib().hk_strerror(status).decode()}{extra}")


_lib = None


def lib():
    """Loads libhk.so (built by build.py).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libhk.so not built ({LIB_PATH}); run paper_2101_02005_gb300/build.py")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    vp, sz = ctypes.c_void_p, ctypes.c_size_t
    L.hk_line_strength.argtypes = [P(hk_lines), P(hk_state), P(hk_opts), vp, vp]
    L.hk_widths.argtypes = [P(hk_lines), P(hk_state), P(hk_opts), vp, vp, vp]
    L.hk_voigt_accumulate.argtypes = [vp, vp, vp, vp, ctypes.c_int64, P(hk_grid), ctypes.c_double,
                                      vp, ctypes.c_int, vp]
    L.hk_cross_section.argtypes = [P(hk_lines), P(hk_grid), P(hk_state), P(hk_opts), vp, vp]
    L.hk_cross_section_batched.argtypes = [P(hk_lines), ctypes.c_int, P(hk_state), ctypes.c_int,
                                           P(hk_grid), P(hk_opts), vp, vp, sz, vp]
    L.hk_cross_section_backward.argtypes = [P(hk_lines), P(hk_grid), P(hk_state), ctypes.c_int,
                                            P(hk_opts), vp, vp, vp, vp, vp, vp, sz, vp]
    L.hk_workspace_size.argtypes = [ctypes.c_int, P(hk_lines), ctypes.c_int, ctypes.c_int,
                                    P(hk_grid), P(hk_opts), P(sz)]
    L.hk_autotune.argtypes = [P(hk_lines), P(hk_grid), P(hk_state), P(hk_opts), vp]
    L.hk_sync_status.argtypes = [vp]
    L.hk_release.argtypes = []
    L.hk_strerror.argtypes = [ctypes.c_int]
    L.hk_strerror.restype = ctypes.c_char_p
    L.hk_last_cuda_error.argtypes = []
    L.hk_constants.argtypes = [P(ctypes.c_double)]
    L.hk_version.argtypes = []
    L.hk_count_ring_pairs.argtypes = [P(hk_lines), P(hk_grid), P(hk_state), P(hk_opts),
                                      P(ctypes.c_int64), vp]
    L.hk_count_pairs.argtypes = [P(hk_lines), P(hk_grid), P(hk_state), P(hk_opts),
                                 P(ctypes.c_int64), vp]
    L.hk_profile.argtypes = [ctypes.c_int, P(ctypes.c_double), P(ctypes.c_int64)]
    L.hk_tuning.argtypes = [ctypes.c_int, P(ctypes.c_int), P(ctypes.c_int)]
    L.hk_set_tuning.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.hk_cross_section_noalloc.argtypes = [P(hk_lines), P(hk_grid), P(hk_state), P(hk_opts),
                                           vp, vp]
    L.hk_cross_section_host.argtypes = [P(hk_lines), P(hk_grid), P(hk_state), P(hk_opts), vp,
                                        ctypes.c_int64, vp]
    L.hk_noalloc_status.argtypes = [vp]
    L.hk_measure_peak.argtypes = [ctypes.c_int, ctypes.c_double, P(ctypes.c_double), vp]
    _lib = L
    return L


def _check(fn, status):
    if status != HK_OK:
        raise HKError(fn, status)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _check_out(fn, t: torch.Tensor, numel: int, dtype, device=None, host_ok=False):
    """Rejects an output tensor the library would write past or misread: wrong
    element type, too few elements, not contiguous, or on the wrong device
    (the library trusts the pointer it is given)."""
    if t.dtype != dtype:
        raise ValueError(f"{fn}: output dtype {t.dtype}, expected {dtype}")
    if t.numel() < numel:
        raise ValueError(f"{fn}: output has {t.numel()} elements, needs {numel}")
    if not t.is_contiguous():
        raise ValueError(f"{fn}: output must be contiguous")
    if t.is_cuda:
        if device is not None and t.device != device:
            raise ValueError(f"{fn}: output on {t.device}, lines on {device}")
    elif not host_ok:
        raise ValueError(f"{fn}: output must be a CUDA tensor")


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


# ---------------------------------------------------------------- data holders


@dataclass
class DeviceLines:
    """A line list resident on the GPU (structure of arrays) plus its hk_lines view."""
    nu0: torch.Tensor
    S_ref: Optional[torch.Tensor]
    E_low: torch.Tensor
    gamma_ref: torch.Tensor
    n_T: torch.Tensor
    mass_amu: float
    A: Optional[torch.Tensor] = None
    g_up: Optional[torch.Tensor] = None
    s_mode: int = HK_S_REF
    sorted: bool = True
    gamma_self: Optional[torch.Tensor] = None
    delta: Optional[torch.Tensor] = None

    @property
    def n(self) -> int:
        return int(self.nu0.numel())

    def struct(self) -> hk_lines:
        p = lambda t: t.data_ptr() if t is not None else None
        return hk_lines(self.nu0.data_ptr(), p(self.S_ref), p(self.A), p(self.g_up),
                        self.E_low.data_ptr(), self.gamma_ref.data_ptr(), self.n_T.data_ptr(),
                        self.n, float(self.mass_amu), int(self.s_mode), int(bool(self.sorted)),
                        p(self.gamma_self), p(self.delta))

    @staticmethod
    def from_host(L, device="cuda", pin=False) -> "DeviceLines":
        """From a synth.LineList (numpy fields)."""
        def t(a, dt):
            if a is None:
                return None
            x = torch.from_numpy(a).to(dt)
            if pin:
                x = x.pin_memory()
            return x.to(device, non_blocking=pin)
        return DeviceLines(t(L.nu0, torch.float64), t(L.S_ref, torch.float32),
                           t(L.E_low, torch.float32), t(L.gamma_ref, torch.float32),
                           t(L.n_T, torch.float32), L.mass_amu, A=t(L.A, torch.float32),
                           g_up=t(L.g_up, torch.float32), s_mode=L.s_mode, sorted=L.sorted,
                           gamma_self=t(getattr(L, "gamma_self", None), torch.float32),
                           delta=t(getattr(L, "delta", None), torch.float32))


class HostLines(DeviceLines):
    """A line list in host memory (page-locked by default), for
    hk_cross_section_host; the same fields as DeviceLines, on the CPU."""

    @staticmethod
    def from_host(L, device="cpu", pin=True) -> "HostLines":
        def t(a, dt):
            if a is None:
                return None
            x = torch.from_numpy(a).to(dt).contiguous()
            return x.pin_memory() if pin else x
        return HostLines(t(L.nu0, torch.float64), t(L.S_ref, torch.float32),
                         t(L.E_low, torch.float32), t(L.gamma_ref, torch.float32),
                         t(L.n_T, torch.float32), L.mass_amu, A=t(L.A, torch.float32),
                         g_up=t(L.g_up, torch.float32), s_mode=L.s_mode, sorted=L.sorted,
                         gamma_self=t(getattr(L, "gamma_self", None), torch.float32),
                         delta=t(getattr(L, "delta", None), torch.float32))


def make_grid(nu_min, dnu, nbins) -> hk_grid:
    return hk_grid(float(nu_min), float(dnu), int(nbins))


def make_state(T, P, Q_T, dlnQ_dT=0.0, P_self=0.0) -> hk_state:
    return hk_state(float(T), float(P), float(Q_T), float(dlnQ_dT), float(P_self))


def make_opts(Q_Tref, cut, precision=HK_FP32C, T_ref=296.0, P_ref=1.0, cut_mode=None,
              flags=0, profile=HK_PROFILE_VOIGT) -> hk_opts:
    if cut_mode is None:
        cut_mode = HK_CUT_FIXED if cut > 0 else HK_CUT_NONE
    return hk_opts(float(T_ref), float(P_ref), float(Q_Tref), float(cut), int(cut_mode),
                   int(precision), int(flags), int(profile))


def sigma_dtype(opts: hk_opts):
    """Element type of a sigma output for these options."""
    if opts.precision == HK_FP64 or (opts.flags & HK_SIGMA_F64):
        return torch.float64
    return torch.float32


# ---------------------------------------------------------------- entry points


def hk_line_strength(lines: DeviceLines, state: hk_state, opts: hk_opts, S_out=None, stream=None):
    if S_out is None:
        S_out = torch.empty(lines.n, dtype=torch.float64, device=lines.nu0.device)
    L = lines.struct()
    _check("hk_line_strength", lib().hk_line_strength(ctypes.byref(L), ctypes.byref(state),
                                                      ctypes.byref(opts), _ptr(S_out),
                                                      _stream(stream)))
    return S_out


def hk_widths(lines: DeviceLines, state: hk_state, opts: hk_opts, stream=None):
    aD = torch.empty(lines.n, dtype=torch.float32, device=lines.nu0.device)
    y = torch.empty_like(aD)
    L = lines.struct()
    _check("hk_widths", lib().hk_widths(ctypes.byref(L), ctypes.byref(state), ctypes.byref(opts),
                                        _ptr(aD), _ptr(y), _stream(stream)))
    return aD, y


def hk_voigt_accumulate(nu0, S, alphaD_inv, y, grid: hk_grid, cut: float, sigma_inout,
                        precision=HK_FP32C, stream=None):
    _check_out("hk_voigt_accumulate", sigma_inout, grid.nbins,
               torch.float64 if precision == HK_FP64 else torch.float32, nu0.device)
    _check("hk_voigt_accumulate",
           lib().hk_voigt_accumulate(_ptr(nu0), _ptr(S), _ptr(alphaD_inv), _ptr(y), nu0.numel(),
                                     ctypes.byref(grid), float(cut), _ptr(sigma_inout),
                                     int(precision), _stream(stream)))
    return sigma_inout


def hk_cross_section(lines: DeviceLines, grid: hk_grid, state: hk_state, opts: hk_opts,
                     sigma_out=None, stream=None):
    if sigma_out is None:
        sigma_out = torch.empty(grid.nbins, dtype=sigma_dtype(opts), device=lines.nu0.device)
    _check_out("hk_cross_section", sigma_out, grid.nbins, sigma_dtype(opts), lines.nu0.device)
    L = lines.struct()
    _check("hk_cross_section", lib().hk_cross_section(ctypes.byref(L), ctypes.byref(grid),
                                                      ctypes.byref(state), ctypes.byref(opts),
                                                      _ptr(sigma_out), _stream(stream)))
    return sigma_out


def hk_cross_section_host(lines: HostLines, grid: hk_grid, state: hk_state, opts: hk_opts,
                          sigma_out=None, chunk_lines=0, stream=None):
    """Cross section of a host-resident line list, streamed to the GPU in
    blocks of chunk_lines (0: the library default).  sigma_out: a host
    (page-locked by default) or device tensor; complete once the stream has
    synchronised."""
    if sigma_out is None:
        sigma_out = torch.empty(grid.nbins, dtype=sigma_dtype(opts), pin_memory=True)
    _check_out("hk_cross_section_host", sigma_out, grid.nbins, sigma_dtype(opts), host_ok=True)
    L = lines.struct()
    _check("hk_cross_section_host",
           lib().hk_cross_section_host(ctypes.byref(L), ctypes.byref(grid), ctypes.byref(state),
                                       ctypes.byref(opts), _ptr(sigma_out), int(chunk_lines),
                                       _stream(stream)))
    return sigma_out


def hk_cross_section_noalloc(lines: DeviceLines, grid: hk_grid, state: hk_state, opts: hk_opts,
                             sigma_out: torch.Tensor, stream=None):
    """hk_cross_section with its scratch in the library's fixed device array:
    no device allocation by the library (the caller provides sigma_out)."""
    _check_out("hk_cross_section_noalloc", sigma_out, grid.nbins, sigma_dtype(opts),
               lines.nu0.device)
    L = lines.struct()
    _check("hk_cross_section_noalloc",
           lib().hk_cross_section_noalloc(ctypes.byref(L), ctypes.byref(grid),
                                          ctypes.byref(state), ctypes.byref(opts),
                                          _ptr(sigma_out), _stream(stream)))
    return sigma_out


def hk_workspace_size(kind: int, species: Sequence[DeviceLines], nTP: int, grid: hk_grid,
                      opts: hk_opts) -> int:
    arr = (hk_lines * len(species))(*[s.struct() for s in species])
    out = ctypes.c_size_t(0)
    _check("hk_workspace_size", lib().hk_workspace_size(kind, arr, len(species), int(nTP),
                                                        ctypes.byref(grid), ctypes.byref(opts),
                                                        ctypes.byref(out)))
    return int(out.value)


def hk_cross_section_batched(species: Sequence[DeviceLines], states: Sequence[hk_state],
                             grid: hk_grid, opts: hk_opts, sigma_out=None, workspace=None,
                             stream=None):
    dev = species[0].nu0.device
    if sigma_out is None:
        sigma_out = torch.empty((len(species), len(states), grid.nbins), dtype=sigma_dtype(opts),
                                device=dev)
    _check_out("hk_cross_section_batched", sigma_out, len(species) * len(states) * grid.nbins,
               sigma_dtype(opts), dev)
    need = hk_workspace_size(0, species, len(states), grid, opts)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    arr = (hk_lines * len(species))(*[s.struct() for s in species])
    st = (hk_state * len(states))(*states)
    _check("hk_cross_section_batched",
           lib().hk_cross_section_batched(arr, len(species), st, len(states), ctypes.byref(grid),
                                          ctypes.byref(opts), _ptr(sigma_out), _ptr(workspace),
                                          workspace.numel(), _stream(stream)))
    return sigma_out


def hk_cross_section_backward(lines: DeviceLines, grid: hk_grid, states: Sequence[hk_state],
                              opts: hk_opts, grad_sigma: torch.Tensor, workspace=None,
                              stream=None):
    dev = lines.nu0.device
    nTP = len(states)
    dT = torch.empty(nTP, dtype=torch.float64, device=dev)
    dP = torch.empty_like(dT)
    dS = torch.empty(lines.n, dtype=torch.float64, device=dev)
    dG = torch.empty_like(dS)
    need = hk_workspace_size(1, [lines], nTP, grid, opts)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    L = lines.struct()
    st = (hk_state * nTP)(*states)
    _check("hk_cross_section_backward",
           lib().hk_cross_section_backward(ctypes.byref(L), ctypes.byref(grid), st, nTP,
                                           ctypes.byref(opts), _ptr(grad_sigma.contiguous()),
                                           _ptr(dT), _ptr(dP), _ptr(dS), _ptr(dG),
                                           _ptr(workspace), workspace.numel(), _stream(stream)))
    return dT, dP, dS, dG


def hk_autotune(lines: DeviceLines, grid: hk_grid, state: hk_state, opts: hk_opts, stream=None):
    L = lines.struct()
    _check("hk_autotune", lib().hk_autotune(ctypes.byref(L), ctypes.byref(grid),
                                            ctypes.byref(state), ctypes.byref(opts),
                                            _stream(stream)))


def hk_count_pairs(lines: DeviceLines, grid: hk_grid, state: hk_state, opts: hk_opts,
                   stream=None):
    """[total, band gh1, gh2, gh3, gh4, core] pair counts (instrumentation)."""
    out = (ctypes.c_int64 * 6)()
    L = lines.struct()
    _check("hk_count_pairs", lib().hk_count_pairs(ctypes.byref(L), ctypes.byref(grid),
                                                  ctypes.byref(state), ctypes.byref(opts), out,
                                                  _stream(stream)))
    return [int(v) for v in out]


def hk_count_ring_pairs(lines: DeviceLines, grid: hk_grid, state: hk_state, opts: hk_opts,
                        stream=None) -> int:
    """Pairs of the core band that the FP32C short-line batches take with the
    8-node ring rule (instrumentation; 0 for other problems)."""
    out = ctypes.c_int64(0)
    L = lines.struct()
    _check("hk_count_ring_pairs", lib().hk_count_ring_pairs(ctypes.byref(L), ctypes.byref(grid),
                                                            ctypes.byref(state),
                                                            ctypes.byref(opts),
                                                            ctypes.byref(out), _stream(stream)))
    return int(out.value)


def hk_profile(mode: int):
    """mode 1: start timing the Voigt-sum launches; mode 0: stop and return
    (total_ms, launches)."""
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int64(0)
    _check("hk_profile", lib().hk_profile(int(mode), ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, int(n.value)


PEAK_FFMA, PEAK_RCP, PEAK_EX2, PEAK_DFMA, PEAK_FFMA2 = 0, 1, 2, 3, 4


def hk_measure_peak(kind: int, target_ms: float = 1000.0, stream=None) -> float:
    """Measured operations per second of one pipe (instrumentation):
    PEAK_FFMA (FMAs), PEAK_RCP, PEAK_EX2 (MUFU ops), PEAK_DFMA (FP64 FMAs), PEAK_FFMA2 (FMAs
    issued as packed FP32x2 instructions)."""
    v = ctypes.c_double(0.0)
    _check("hk_measure_peak", lib().hk_measure_peak(int(kind), float(target_ms), ctypes.byref(v),
                                                    _stream(stream)))
    return float(v.value)


def hk_tuning(precision: int = HK_FP32C) -> int:
    """Lines per work item currently used for `precision`."""
    return hk_tuning_full(precision)[0]


def hk_tuning_full(precision: int = HK_FP32C):
    """(lines per work item, tile width in bins) currently used for `precision`."""
    v = ctypes.c_int(0)
    t = ctypes.c_int(0)
    _check("hk_tuning", lib().hk_tuning(int(precision), ctypes.byref(v), ctypes.byref(t)))
    return int(v.value), int(t.value)


def hk_set_tuning(precision: int, lmax: int, tile_bins: int = 0):
    """Sets lines per work item (and, unless 0, the tile width) of `precision`
    on the current device."""
    _check("hk_set_tuning", lib().hk_set_tuning(int(precision), int(lmax), int(tile_bins)))


def hk_sync_status(stream=None):
    _check("hk_sync_status", lib().hk_sync_status(_stream(stream)))


def hk_noalloc_status(stream=None):
    """Raises HKError(HK_ERANGE) if the latest hk_cross_section_noalloc call
    on this device overflowed its float output (clears the flag)."""
    _check("hk_noalloc_status", lib().hk_noalloc_status(_stream(stream)))


def hk_release():
    _check("hk_release", lib().hk_release())


def hk_constants():
    out = (ctypes.c_double * 6)()
    _check("hk_constants", lib().hk_constants(out))
    return dict(zip(["c", "k_B", "h", "amu", "c2", "pi"], list(out)))


def hk_version() -> int:
    return int(lib().hk_version())


# ---------------------------------------------------------------- autograd


class CrossSectionFn(torch.autograd.Function):
    """sigma[k] for (T[k], P[k]) points of one species, as a [points, nbins]
    tensor differentiable in T, P (per point) and S_ref, gamma_ref (per line).
    Forward: hk_cross_section_batched (FP32C); backward:
    hk_cross_section_backward (recomputes the profiles).  Call as
    CrossSectionFn.apply(T, P, S_ref, gamma_ref, lines, grid, opts, Q_fn, dlnQ_fn)."""

    @staticmethod
    def forward(ctx, T, P, S_ref, gamma_ref, lines: DeviceLines, grid: hk_grid, opts: hk_opts,
                Q_fn, dlnQ_fn):
        Tl = [float(t) for t in T.detach().cpu().tolist()]
        Pl = [float(p) for p in P.detach().cpu().tolist()]
        states = [make_state(t, p, Q_fn(t), dlnQ_fn(t)) for t, p in zip(Tl, Pl)]
        L = DeviceLines(lines.nu0, S_ref.detach().contiguous(), lines.E_low,
                        gamma_ref.detach().contiguous(), lines.n_T, lines.mass_amu, A=lines.A,
                        g_up=lines.g_up, s_mode=lines.s_mode, sorted=lines.sorted)
        sigma = hk_cross_section_batched([L], states, grid, opts)
        ctx.L, ctx.states, ctx.grid, ctx.opts = L, states, grid, opts
        ctx.tp = (T.dtype, T.device, P.dtype, P.device)
        return sigma.reshape(len(states), grid.nbins)

    @staticmethod
    def backward(ctx, g):
        dT, dP, dS, dG = hk_cross_section_backward(ctx.L, ctx.grid, ctx.states, ctx.opts,
                                                   g.to(torch.float32).contiguous())
        tdt, tdev, pdt, pdev = ctx.tp
        return (dT.to(device=tdev, dtype=tdt), dP.to(device=pdev, dtype=pdt),
                dS.to(ctx.L.S_ref.dtype), dG.to(ctx.L.gamma_ref.dtype),
                None, None, None, None, None)
