/*
 * hk.h -- C ABI of libhk, a GB300 (sm_103a) implementation of the opacity hot
 * path of HELIOS-K 2.0 (Grimm et al. 2021, arXiv:2101.02005).
 *
 * For each temperature/pressure point (T, P) the library turns a spectral
 * line list into per-line strengths S(T) (Sect. 2.2.2, Eq. S and its split
 * form Eq. S1 of Sect. 2.4.3), Doppler and Lorentz widths (Sect. 2.2,
 * Eqs. gammaD and gammaL, ExoMol form; code parameters of Sect. 2.4.2), and
 * sums area-normalised Voigt profiles
 *
 *     phi(nu) = Re w(x + i y) / (alpha_D sqrt(pi)),
 *     x = (nu - nu0) / alpha_D,  y = Gamma_L / alpha_D,
 *     alpha_D = (nu0 / c) sqrt(2 k_B T / m)          (Eq. alphaD inverted)
 *
 * over every wavenumber bin within the cutting length (Sect. 2.4.3 item 4,
 * Sect. 2.4.5) into the cross section sigma(nu_i), nu_i = nu_min + i dnu.
 * w is the Faddeeva function (Sect. 2.2.3).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Memory.   Every array argument is a DEVICE pointer owned by the caller
 *           unless stated otherwise.  The library never frees caller memory.
 *           Struct arguments (hk_lines, hk_grid, ...) are HOST pointers read
 *           during the call only.
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *           stream).  Calls are asynchronous with respect to the host: they
 *           enqueue kernels on `stream` and return; results are valid once
 *           the stream reaches that point.
 * Errors.   Every entry point returns 0 (HK_OK) or a positive HK_E* code.
 *           Argument errors are detected on the host before anything is
 *           enqueued and leave all outputs untouched.  HK_ECUDA reports a
 *           failed launch or CUDA runtime call; hk_last_cuda_error() gives
 *           the cudaError_t.  Conditions found on the device (a float output
 *           that overflowed: HK_ERANGE) set a per-device status word that
 *           hk_sync_status() reports and clears.  No entry point aborts,
 *           traps or throws.
 * Scratch.  Single-point calls draw scratch memory from a per-device pool
 *           that grows on demand (cudaMalloc) up to HK_POOL_LIMIT_MB
 *           (environment, default 16384 MiB) and is released by
 *           hk_release().  Calls that need more return HK_ENOMEM.  Batched
 *           and adjoint calls take caller-provided workspace sized by
 *           hk_workspace_size().  Concurrent calls on different streams that
 *           use the pool must be serialised by the caller.
 * Order.    Lines must be sorted by nu0 (ascending) when hk_lines.sorted is
 *           1; with sorted = 0 the library sorts a copy (radix sort) and
 *           returns per-line gradients in the caller's original order.
 * Units.    nu in cm^-1, T in K, P in bar, S in cm/molecule (cm/g with
 *           HK_PER_GRAM), sigma in cm^2/molecule (cm^2/g).
 */
#ifndef HK_H
#define HK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define HK_OK 0
#define HK_EINVAL 1   /* invalid argument (null pointer, n < 0, nbins <= 0, dnu <= 0,
                         T <= 0, P < 0, Q <= 0, mass <= 0, NaN, unknown enum) */
#define HK_ENOMEM 2   /* scratch pool or caller workspace too small */
#define HK_ECUDA 3    /* a CUDA launch or runtime call failed */
#define HK_ETIMEOUT 4 /* a bounded device-side wait gave up (see hk_sync_status); reserved:
                         no kernel of this version waits on another block or launch */
#define HK_ENOTSUP 5  /* combination of options not supported */
#define HK_ERANGE 6   /* a float sigma output overflowed (reported by hk_sync_status);
                         request double output with HK_SIGMA_F64 */
#define HK_ESIZE 7    /* the grid is larger than hk_cross_section_noalloc's fixed scratch */

/* ---- enums -------------------------------------------------------------- */
/* line-strength mode (Sect. 2.2.2) */
#define HK_S_REF 0        /* S_ref given at T_ref; scaled with Q, Boltzmann and
                             stimulated-emission ratios */
#define HK_S_EINSTEIN_A 1 /* S from Einstein A and g' by Eq. S */
/* arithmetic of the Voigt sum */
#define HK_FP32C 0 /* FP32 profiles, compensated FP32 tile sums, FP64 final sum;
                      sigma out as float */
#define HK_FP64 1  /* FP64 throughout; sigma out as double */
/* cut mode (Sect. 2.4.3 item 4) */
#define HK_CUT_FIXED 0   /* |nu_i - nu0| <= cut; cut <= 0 means the whole grid */
#define HK_CUT_NONE 1    /* every bin of the grid */
#define HK_CUT_DOPPLER 2 /* per line: |nu_i - nu0| <= cut * Gamma_D, Gamma_D = sqrt(ln 2)
                            alpha_D the Doppler half width (Eq. gammaD), evaluated in
                            FP64 as cut * (nu0 * K_D), K_D = sqrt(ln 2) sqrt(2 k_B T/m)/c */
#define HK_CUT_LORENTZ 3 /* per line: |nu_i - nu0| <= cut * Gamma_L, the Lorentz half
                            width in FP64 (a bin within one ulp of such a boundary may be
                            decided differently from a CPU evaluation: pow differs in its
                            last bit between math libraries) */
/* line profile (Sect. 2.1: HELIOS-K offers four) */
#define HK_PROFILE_VOIGT 0         /* Re w(x + iy) / (alpha_D sqrt(pi)) */
#define HK_PROFILE_LORENTZ 1       /* (Gamma_L / pi) / ((nu - nu0)^2 + Gamma_L^2) */
#define HK_PROFILE_DOPPLER 2       /* exp(-x^2) / (alpha_D sqrt(pi)) */
#define HK_PROFILE_BINNED_GAUSS 3  /* the Doppler profile averaged over each bin
                                      [nu_i - dnu/2, nu_i + dnu/2]: the "binned Gaussian
                                      integrated cross section" of ExoCross */
/* flags */
#define HK_PER_GRAM 1u  /* divide S by the molecular mass in grams (Eq. S units) */
#define HK_SIGMA_F64 2u /* HK_FP32C: write sigma as double instead of float.  The
                           FP32C arithmetic is unchanged; use it when S(T) can exceed
                           the float range (S_ref scaled to T >> T_ref for lines of
                           large E'' gives S(T) ~ 1e40 and more) */
#define HK_REMOVE_PLINTH 4u /* subtract from every bin inside a line's cut the line's own
                               value at its cutting length, S phi(nu0 + cut) (Sect. 2.1,
                               "Removing the Plinth"); no effect without a cut.  Not
                               supported by hk_cross_section_backward (HK_ENOTSUP) */

/* ---- data structures ---------------------------------------------------- */

/* One species' line list, structure of arrays, DEVICE pointers, read-only.
 * Field set of the binary line format of Sect. 2.5 (Tables binary1/2). */
typedef struct {
    const double *nu0;       /* [n] line centre, cm^-1 */
    const float *S_ref;      /* [n] strength at T_ref, cm/molecule (HK_S_REF) */
    const float *A;          /* [n] Einstein A, s^-1; NULL means 0.  Enters
                                Gamma_L as A/(4 pi c) and S in HK_S_EINSTEIN_A */
    const float *g_up;       /* [n] upper-state weight g' (HK_S_EINSTEIN_A only) */
    const float *E_low;      /* [n] lower-state energy E'', cm^-1 */
    const float *gamma_ref;  /* [n] Lorentz HWHM at T_ref, P_ref, cm^-1 bar^-1 */
    const float *n_T;        /* [n] temperature exponent n */
    int64_t n;               /* number of lines, >= 0 */
    double mass_amu;         /* molecular mass, atomic mass units */
    int s_mode;              /* HK_S_REF or HK_S_EINSTEIN_A */
    int sorted;              /* 1 if nu0 is ascending */
    const float *gamma_self; /* [n] or NULL.  Non-NULL: HITRAN widths (Sect. 2.2, Eq.
                                gammaL), gamma_ref is then gamma_air and
                                Gamma_L = A/(4 pi c) + (T_ref/T)^n [gamma_air (P - P_self)
                                + gamma_self P_self] / P_ref */
    const float *delta;      /* [n] or NULL: pressure shift (Table binary2), cm^-1 per
                                P_ref; the line sits at nu0 + delta P / P_ref (FP64), its
                                strength and Doppler width keep nu0.  Sorting is by nu0 */
} hk_lines;

/* Uniform wavenumber grid nu_i = nu_min + i * dnu, 0 <= i < nbins
 * (point-sampled; nu_max = nu_min + nbins * dnu is excluded). */
typedef struct {
    double nu_min;
    double dnu;
    int64_t nbins;
} hk_grid;

/* Thermodynamic point.  Q_T = Q(T) and dlnQ_dT = d ln Q / dT are supplied by
 * the caller (the partition function of Sect. 2.2.2, Eq. partition, is an
 * input, not computed here); dlnQ_dT is used by the adjoint only. */
typedef struct {
    double T;
    double P;
    double Q_T;
    double dlnQ_dT;
    double P_self;           /* self partial pressure (HITRAN widths only), 0 <= P_self */
} hk_state;

/* Options.  T_ref, P_ref, Q_Tref: reference state of S_ref and gamma_ref
 * (296 K, 1 bar in the benchmark configurations).  cut: cutting length in
 * cm^-1 (HK_CUT_FIXED; cut <= 0 means no cut), or the factor (> 0) of the
 * per-line half width (HK_CUT_DOPPLER, HK_CUT_LORENTZ; Sect. 2.4.3 item 4:
 * fixed length, Doppler or Lorentz half-width multiples).  precision:
 * HK_FP32C or HK_FP64.  flags: HK_PER_GRAM, HK_SIGMA_F64, HK_REMOVE_PLINTH.
 * profile: HK_PROFILE_* (the plinth is the chosen profile's value at the
 * cutting length).  The per-line cut modes, the plinth and the profiles
 * apply to every sigma entry point; hk_voigt_accumulate takes its own fixed
 * cut and the Voigt profile, and hk_cross_section_backward supports the Voigt
 * profile with HK_CUT_FIXED / HK_CUT_NONE, no plinth and lines without
 * gamma_self or delta (else HK_ENOTSUP). */
typedef struct {
    double T_ref;
    double P_ref;
    double Q_Tref;
    double cut;
    int cut_mode;
    int precision;
    unsigned flags;
    int profile;
} hk_opts;

/* ---- entry points ------------------------------------------------------- */

/* Per-line strength S(T) (Sect. 2.2.2 Eq. S; split form Eqs. S1/S1' of
 * Sect. 2.4.3, step 2).  HK_S_REF:
 *   S = S_ref (Q(T_ref)/Q(T)) exp(-c2 E'' (1/T - 1/T_ref))
 *       (1 - exp(-c2 nu0/T)) / (1 - exp(-c2 nu0/T_ref)),   c2 = h c / k_B.
 * HK_S_EINSTEIN_A: S = A g' / (8 pi c nu0^2 Q(T)) exp(-c2 E''/T)(1 - exp(-c2 nu0/T)).
 * S_out: DEVICE double[n], overwritten, in the caller's line order. */
int hk_line_strength(const hk_lines *lines, const hk_state *state, const hk_opts *opts,
                     double *S_out, void *stream);

/* Per-line code parameters of Sect. 2.4.2: alphaD_inv = (c/nu0) sqrt(m/(2 k_B T))
 * (Eq. alphaD) and y = Gamma_L * alphaD_inv with the ExoMol Lorentz width
 * Gamma_L = A/(4 pi c) + gamma_ref (T_ref/T)^n (P/P_ref) (Sect. 2.2).
 * alphaD_inv_out, y_out: DEVICE float[n], overwritten, caller's order. */
int hk_widths(const hk_lines *lines, const hk_state *state, const hk_opts *opts,
              float *alphaD_inv_out, float *y_out, void *stream);

/* Voigt sum with precomputed line parameters (Sect. 2.4.4, kernel "K"):
 * sigma[i] += sum_l S[l] * Re w(x_il + i y[l]) * alphaD_inv[l] / sqrt(pi)
 * over bins with |nu_i - nu0[l]| <= cut (cut <= 0: every bin).
 * nu0 must be ascending.  nu0, S: DEVICE double[n]; alphaD_inv, y: DEVICE
 * float[n].  sigma_inout: DEVICE float[nbins] (HK_FP32C) or double[nbins]
 * (HK_FP64); the sum is ADDED to its contents. */
int hk_voigt_accumulate(const double *nu0, const double *S, const float *alphaD_inv,
                        const float *y, int64_t n, const hk_grid *grid, double cut,
                        void *sigma_inout, int precision, void *stream);

/* Whole path for one (T, P): strengths, widths and the Voigt sum, fused in
 * one pass over the lines (steps of Sect. 2.4.6: L, I, K, A).
 * sigma_out: DEVICE float[nbins] (HK_FP32C) or double[nbins] (HK_FP64, or
 * HK_FP32C with HK_SIGMA_F64), overwritten.  Lines with nu0 <= 0 have no
 * Doppler width (Eq. gammaD) and contribute nothing. */
int hk_cross_section(const hk_lines *lines, const hk_grid *grid, const hk_state *state,
                     const hk_opts *opts, void *sigma_out, void *stream);

/* hk_cross_section for a line list in HOST memory, streamed to the GPU in
 * blocks whose copies overlap the sums of the previous block (Sect. 2.3;
 * Sect. 2.4.1, asynchronous interleaved copies of line-list blocks;
 * Sect. 2.4.6 and its workflow figure, copies "C" hidden behind the
 * kernels).  Blocks grow from chunk_lines/8 to chunk_lines lines (0: 2^26,
 * two device buffers of 1.6 GB for five fields; a list shorter than that
 * takes buffers of its own size); each is copied on an
 * internal copy stream into one of two device buffers, then summed exactly
 * as hk_cross_section sums a device-resident list (its own strength, FP32
 * scale and tile schedule) into an FP64 partial sigma.  Even blocks run on
 * `stream`, odd ones on an internal second stream (so one block's work fills
 * the SMs the previous block's launch leaves idle at its end); `stream` then
 * adds the two partial sums, converts to the output type and copies the
 * result to sigma_out.  The sum over blocks is a sum over lines, so the
 * result equals hk_cross_section's up to the FP32 rounding of the per-block
 * tile sums.
 * lines: the hk_lines fields are HOST pointers (page-locked memory gives
 * full copy speed and overlap; pageable memory works, slower); the list may
 * be unsorted (each block is then sorted on the GPU).  sigma_out: HOST or
 * DEVICE float[nbins] (HK_FP32C) or double[nbins] (HK_FP64, or
 * HK_SIGMA_F64), overwritten.  Everything is enqueued on `stream`: the
 * host buffers must stay valid, and sigma_out is complete, once `stream`
 * has synchronised.  Calls on one device share the library's scratch pool
 * and copy stream and must not overlap. */
int hk_cross_section_host(const hk_lines *lines, const hk_grid *grid, const hk_state *state,
                          const hk_opts *opts, void *sigma_out, int64_t chunk_lines,
                          void *stream);

/* hk_cross_section for callers that must not allocate device memory.  The
 * paper has no counterpart; this is a service of the library.
 *
 * Some callers cannot let a library call cudaMalloc: an application that
 * owns every byte of the GPU through its own allocator and forbids other
 * allocations, a process with a hard device-memory budget, or a loop that
 * cannot afford the device-wide synchronisation cudaMalloc/cudaFree imply.
 * This entry point computes exactly what hk_cross_section computes (same
 * kernels, same arithmetic, same output layout) but takes its scratch
 * memory -- the FP64 accumulator, the per-tile line ranges and the work
 * counter -- from one fixed array that the library declares in device
 * memory: HK_NOALLOC_SCRATCH_BYTES (16 MiB).  Every GPU that loads libhk
 * holds that array until the process exits; this call never calls cudaMalloc,
 * cudaFree or any allocating routine.
 *
 * Limits: the lines must be sorted (hk_lines.sorted = 1; sorting needs
 * scratch proportional to n, so unsorted lists return HK_ENOTSUP); the grid
 * must fit the array: about 2.09e6 bins for HK_FP32C and 2.6e8 for HK_FP64,
 * exactly when hk_cross_section's workspace plus 256 bytes is at most
 * HK_NOALLOC_SCRATCH_BYTES; larger grids return HK_ESIZE before anything is
 * enqueued.  A float output that overflows sets a status flag inside the
 * array (not the word hk_sync_status reads): hk_noalloc_status reports it;
 * request HK_SIGMA_F64 when S(T) can exceed the float range.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls on a device share the one array,
 * which keeps the previous call's contents (the call clears what must start
 * at zero), so calls whose work overlaps on the GPU -- on different streams
 * without ordering -- race and must be serialised by the caller.
 * sigma_out: DEVICE float[nbins] (HK_FP32C) or double[nbins] (HK_FP64, or
 * HK_SIGMA_F64), overwritten. */
#define HK_NOALLOC_SCRATCH_BYTES (16u << 20)
int hk_cross_section_noalloc(const hk_lines *lines, const hk_grid *grid, const hk_state *state,
                             const hk_opts *opts, void *sigma_out, void *stream);

/* Status of the most recent hk_cross_section_noalloc call on the current
 * device (no paper counterpart): synchronises `stream` (the stream that call
 * ran on), then returns HK_ERANGE if its float sigma output overflowed, else
 * 0 (HK_ECUDA on a CUDA error), and clears the flag.  Like the call itself it
 * allocates no device memory; before any hk_cross_section_noalloc call on the
 * device it returns 0. */
int hk_noalloc_status(void *stream);

/* Opacity table in one persistent launch: every species x every (T, P)
 * point (pressure batching of Sect. 2.4.6 / Sect. 3.5, generalised to a T-P
 * grid and several species).  species: HOST array of nspecies hk_lines
 * (each with DEVICE field pointers).  TP: HOST array of nTP states.
 * sigma_out: DEVICE float[nspecies][nTP][nbins] (HK_FP32C; double with
 * HK_SIGMA_F64), overwritten.  workspace: DEVICE, ws_bytes >=
 * hk_workspace_size(...). */
int hk_cross_section_batched(const hk_lines *species, int nspecies, const hk_state *TP, int nTP,
                             const hk_grid *grid, const hk_opts *opts, void *sigma_out,
                             void *workspace, size_t ws_bytes, void *stream);

/* Adjoint of L = sum_k sum_i grad_sigma[k][i] sigma_k[i] over nTP points of
 * one species in HK_S_REF mode: the chain rule through S(T) (Sect. 2.2.2),
 * alpha_D(T) (Eq. alphaD), Gamma_L(T, P) (ExoMol form of Sect. 2.2) and the
 * Faddeeva derivative w'(z) = -2 z w + 2i/sqrt(pi) (d Re w/dx = Re w',
 * d Re w/dy = -Im w').  Profiles are recomputed in FP32, never stored;
 * per-line sums are FP32, every reduction across lines or points is FP64.
 * grad_sigma: DEVICE float[nTP][nbins] (the upstream gradient dL/dsigma).
 * Outputs (DEVICE, overwritten): dL_dT, dL_dP: double[nTP];
 * dL_dSref, dL_dgamma_ref: double[n], summed over the nTP points, in the
 * caller's line order (S(T)/S_ref can exceed the float range at T >> T_ref,
 * hence double).  workspace: DEVICE, ws_bytes >= hk_workspace_size(1, ...). */
int hk_cross_section_backward(const hk_lines *lines, const hk_grid *grid, const hk_state *TP,
                              int nTP, const hk_opts *opts, const float *grad_sigma,
                              double *dL_dT, double *dL_dP, double *dL_dSref,
                              double *dL_dgamma_ref, void *workspace, size_t ws_bytes,
                              void *stream);

/* Workspace bytes for hk_cross_section_batched (kind 0) or
 * hk_cross_section_backward (kind 1) with these arguments. */
int hk_workspace_size(int kind, const hk_lines *species, int nspecies, int nTP,
                      const hk_grid *grid, const hk_opts *opts, size_t *bytes);

/* The self-tuning of Sect. 2.4.4 (the paper re-tunes its thread counts
 * during a run), done once: times the Voigt sum of this problem for each
 * candidate setting and caches the fastest for the current device and
 * opts->precision; later calls, batched ones included, use it.  Candidates:
 * lines per work item 1024, 2048, 4096, 16384 and 65536 (small items balance
 * uneven line density, large ones amortise per-item costs) and, for
 * HK_FP32C, a tile width of 1024 or 2048 bins (3 or 2 blocks of 8 warps per
 * SM; wide lines visit half as many 2048-bin tiles).  Runs the problem twice
 * per candidate (a warm-up and a timed call) and synchronises `stream`.
 * Allocates one nbins-sized buffer while it runs. */
int hk_autotune(const hk_lines *lines, const hk_grid *grid, const hk_state *state,
                const hk_opts *opts, void *stream);

/* The setting in use for a precision on the current device: lines per work
 * item (defaults 2048 for HK_FP32C and 16384 for HK_FP64 until hk_autotune
 * has run) and the tile width in bins (HK_FP32C default 1024; HK_FP64 512).
 * lmax, tile_bins: HOST ints (tile_bins may be NULL). */
int hk_tuning(int precision, int *lmax, int *tile_bins);

/* Sets the setting for a precision on the current device, e.g. to reuse what
 * hk_autotune found in an earlier process (no paper counterpart).  lmax: 32
 * .. 2^24; tile_bins: 0 keeps the current width, else 1024 or 2048 for
 * HK_FP32C, 512 for HK_FP64; other values give HK_EINVAL. */
int hk_set_tuning(int precision, int lmax, int tile_bins);

/* Instrumentation (no counterpart in the paper).  Counts the (line, bin)
 * pairs the cut admits for this problem: counts[0] = total (the algorithmic
 * Voigt-evaluation count, from the same cut bounds as the FP32 sum, which
 * equal those of the FP64 predicate |(i - i0) - r| <= W),
 * counts[1..5] = pairs whose r2 = x^2 + y^2 falls in the Faddeeva bands
 * r2 >= 1.5e6, [2500, 1.5e6), [200, 2500), [64, 200), < 64 (band edges
 * decided in FP64, so a few pairs at an edge may differ from the kernel's
 * FP32 choice).  counts: HOST int64[6].  Synchronises `stream`. */
int hk_count_pairs(const hk_lines *lines, const hk_grid *grid, const hk_state *state,
                   const hk_opts *opts, int64_t *counts, void *stream);

/* Instrumentation (no counterpart in the paper).  Of the pairs counted in
 * counts[5] by hk_count_pairs (r2 < 64), those that the FP32C short-line
 * batches evaluate with the 8-node Gauss-Hermite ring rule instead of the
 * trapezoid: R8(y) <= r2 < 64, R8(y) = max(26, ln(1.13e9 / y)) capped at 64
 * (decided in FP64).  Nonzero only for problems that take the short-line
 * path (HK_FP32C, the Voigt profile, a fixed cut of fewer than 1024 bins);
 * lines of a batch that does not share its structure take the trapezoid
 * there, so this is an upper bound.  *ring: HOST int64.  Synchronises
 * `stream`. */
int hk_count_ring_pairs(const hk_lines *lines, const hk_grid *grid, const hk_state *state,
                        const hk_opts *opts, int64_t *ring, void *stream);

/* Instrumentation (no counterpart in the paper).  mode 1: start recording
 * CUDA events around every launch of the Voigt-sum kernel on the stream it
 * runs on (previous records are dropped).  mode 0: stop, wait for the
 * recorded events, and return the summed kernel time in *ms and the number
 * of launches in *launches (either pointer may be NULL). */
int hk_profile(int mode, double *ms, int64_t *launches);

/* Instrumentation (no counterpart in the paper): the measured throughput of
 * one pipe of the current device, for the rooflines of the kernels.  kind 0:
 * FP32 fused multiply-adds per second; 1: MUFU reciprocals (rcp.approx.ftz)
 * per second; 2: MUFU base-2 exponentials (ex2.approx.ftz) per second; 3: FP64
 * fused multiply-adds per second; 4: FP32 fused multiply-adds per second
 * issued as packed FP32x2 instructions (two per lane and instruction).
 * Every SM runs 64 warps of independent
 * chains of the operation; a calibration launch sizes launches of ~100 ms,
 * repeated for about target_ms (0 < target_ms <= 60000).  *ops_per_s: HOST
 * double.  Synchronises `stream`; uses the scratch pool (2.5 MB). */
int hk_measure_peak(int kind, double target_ms, double *ops_per_s, void *stream);

/* Synchronises `stream`, then reports and clears the device status word of
 * the current device: HK_ERANGE if a float sigma output overflowed since the
 * last call, HK_ETIMEOUT if a bounded device wait gave up; HK_ECUDA on a CUDA
 * error; else 0. */
int hk_sync_status(void *stream);

/* Frees the scratch pool of the current device. */
int hk_release(void);

/* Human-readable text of a status code (static storage). */
const char *hk_strerror(int status);

/* cudaError_t of the most recent HK_ECUDA on this thread (0 if none). */
int hk_last_cuda_error(void);

/* The physical constants the device code uses: c, k_B, h, amu, c2, pi.
 * out6: HOST double[6].  Needs no GPU. */
int hk_constants(double *out6);

/* Library version (major*10000 + minor*100 + patch). */
int hk_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HK_H */
