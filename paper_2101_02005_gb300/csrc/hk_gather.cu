// hk_gather.cu -- the Voigt sum sigma_i = sum_l S_l phi_l(nu_i) on sm_103a.
//
// Design (GB300-first; the paper's line-parallel scatter with rotated
// shared-memory writes, Sect. 2.4.4, is prior art and not used):
//
// * Work items.  The grid is cut into tiles of NWARPS*32*BPT bins.  A tile's
//   candidate lines are a contiguous range of the nu0-sorted list (bisection
//   on nu0 with the cut), split into items of at most `lmax` lines.  Items of
//   every (problem, tile) are numbered by an exclusive scan; one persistent
//   launch pulls items from an atomic counter, so uneven line density
//   (log-normal windows) and many problems (species x T x P) balance across
//   the 152 SMs.
// * Bin-parallel gather.  Each lane owns BPT bins of its warp's slice of the
//   tile (lane-strided, so neighbouring lanes hold neighbouring bins and see
//   the same Faddeeva band).  Each warp stages its own candidate lines (those
//   within the cut of its bins, found by bisection on nu0), 32 at a time with
//   one lane per line, and reads them back as warp-wide broadcasts: no warp
//   waits for another inside an item.
// * Accumulation.  FP32C: FP32 partial sums per lane, folded every FLUSH
//   lines into a (hi, lo) two-sum pair; at the end of the item one FP64
//   atomicAdd per bin into a per-problem FP64 accumulator (the final
//   cross-tile sum is FP64).  FP64: double accumulators and atomics.
// * Exact cut.  Membership of a bin is decided by integer compare against the
//   line's [lo, hi] bin range, itself decided in FP64 by the predicate
//   |k - r| <= W (see line_geometry) -- the same decision as the oracle's.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <mutex>
#include <vector>

#include "hk_internal.cuh"
#include "hk_launch.h"

namespace hk {

constexpr int NWARPS = 8;
constexpr int NTHREADS = NWARPS * 32;
constexpr int FLUSH = 32;        // FP32 lines per two-sum fold

template <typename R> struct LineT {
    R b, r, y, s, h;   // h: the plinth s Re w(x_cut + iy), or 0
    int i0, lo, hi, pad;
};

// ---- scale prepass ---------------------------------------------------------------
// FP32C sums S * alphaD_inv / sqrt(pi) * Re w scaled by 2^-scale so that the
// largest value any line puts into any bin is about 1: far from overflow even
// after summing 1e9 lines, and with the 1e-10 dynamic range the parity bar
// looks at far from the float denormals.  A line's largest sampled value is
// at its nearest bin, x_n = |r_n| b (r_n in [-1/2, 1/2]); a narrow line whose
// centre falls between bins never reaches its peak, so the peak is not used.
// Re w(x, y) <= min(1, exp(-x^2) + y / (sqrt(pi) x^2)) bounds it within a
// small factor, which is all the exponent needs.
// The other profiles: Lorentz (y/sqrt(pi)) / (X + y^2) exactly, Doppler
// exp(-X) exactly, binned Gaussian at most min(1, sqrt(pi)/b).
__device__ __forceinline__ int sampled_peak_exp2(float x_n, float y, int profile, float b)
{
    float X = x_n * x_n;
    float B;
    if (profile == kProfLorentz) {
        B = (float)kInvSqrtPi * y / (X + y * y);
    } else if (profile == kProfDoppler) {
        B = expf(-X);
    } else if (profile == kProfBinned) {
        B = fminf(1.0f, (float)(1.0 / kInvSqrtPi) / b);
    } else {
        B = expf(-X) + (float)kInvSqrtPi * y / X;  // X = 0 gives +inf -> 1
        B = fminf(B, 1.0f);
    }
    return B > 0.0f && B < INFINITY ? ilogbf(B) : INT_MIN / 2;
}

// One line's largest sampled value as a power-of-two exponent (INT_MIN if it
// adds nothing).
// Only an exponent is needed, so the position, the coarse grid-range test and
// the nearest-bin offset are float (FP64 runs at a small fraction of the FP32
// rate and would dominate this pass): a line at the edge of the range may be
// counted or skipped, which moves the scale, never the sum.
__device__ __forceinline__ int line_peak_exp(const Prob &pr, const GridD &g, int64_t l,
                                             float nu_lo, float nu_hi, float nu_min,
                                             float inv_dnu)
{
    const float nu0 = (float)(pr.delta ? line_pos(pr, l) : pr.nu0[l]);
    if (!(nu0 > 0.0f) || (g.W > 0.0 && (nu0 < nu_lo || nu0 > nu_hi))) return INT_MIN;
    float u = (nu0 - nu_min) * inv_dnu;
    float rn = fabsf(u - rintf(u));
    if (pr.pre) {
        double v = pr.S_pre[l] * (double)pr.aDinv_pre[l] * kInvSqrtPi;
        float b = (float)g.dnu * pr.aDinv_pre[l];
        return v > 0.0 ? ilogb(v) + sampled_peak_exp2(rn * b, pr.y_pre[l], kProfVoigt, b)
                       : INT_MIN;
    }
    float P, aDinv, y;
    int e2;
    line_strength_f32(pr, l, &P, &e2, &aDinv, &y);
    float b = (float)g.dnu * aDinv;
    return P > 0.0f ? ilogbf(P) + e2 + sampled_peak_exp2(rn * b, y, g.profile, b) : INT_MIN;
}

// Four lines per thread and iteration, so that each thread has the loads of
// four lines in flight (the pass is a stream over the line list).
__global__ void k_scale_prepass(const Prob *__restrict__ probs, int nprob, GridD g)
{
    int p = blockIdx.y;
    if (p >= nprob) return;
    const Prob &pr = probs[p];
    const float nu_lo = (float)(g.nu_min - g.cut - 2.0 * g.dnu);
    const float nu_hi = (float)(g.nu_min + (double)g.nbins * g.dnu + g.cut + 2.0 * g.dnu);
    const float nu_min = (float)g.nu_min, inv_dnu = (float)g.inv_dnu;
    int emax = INT_MIN;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < pr.n; l += 4 * stride) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t lk = l + k * stride;
            if (lk < pr.n)
                emax = max(emax, line_peak_exp(pr, g, lk, nu_lo, nu_hi, nu_min, inv_dnu));
        }
    }
    for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    if ((threadIdx.x & 31) == 0 && emax != INT_MIN) atomicMax(pr.scale_exp, emax);
}

// ---- largest reach of a line: per-line cut plus pressure shift ----------------
// Non-negative doubles order like their bit patterns, so an integer atomicMax
// on the bits is a max on the values.
__global__ void k_cut_max(const Prob *__restrict__ probs, int nprob, GridD g)
{
    int p = blockIdx.y;
    if (p >= nprob) return;
    const Prob &pr = probs[p];
    unsigned long long best = 0ull;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < pr.n;
         l += (int64_t)gridDim.x * blockDim.x) {
        const double nu0 = pr.nu0[l], pos = line_pos(pr, l);
        if (!(pos > 0.0)) continue;
        // the float Lorentz width, inflated past its distance to the FP64 one
        const bool fl = g.cut_mode == kCutLorentz && !(pr.gamma_self && pr.press_air < 0.0);
        CutW cw = fl ? lorentz_cut_f32(pr, g, l) : line_cut(pr, g, l, nu0);
        if (fl) cw.W = cw.W * (1.0 + 1e-5) + 1e-3;
        if (cw.nocut) continue;
        // the reach of the line from its unshifted centre: cut plus |shift|
        const double cut = __dmul_rn(cw.W, g.dnu) * (1.0 + 1e-12) + fabs(pos - nu0) * (1.0 + 1e-12) +
                           1e-300;
        if (cut > 0.0 && cut < 1e300) best = max(best, (unsigned long long)__double_as_longlong(cut));
    }
    for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0 && best) atomicMax((unsigned long long *)pr.cutmax, best);
}

// ---- tile line ranges and item counts ---------------------------------------
__device__ __forceinline__ int64_t lower_bound_nu(const double *nu, int64_t n, double v)
{
    int64_t a = 0, b = n;
    while (a < b) {
        int64_t m = (a + b) >> 1;
        if (nu[m] < v) a = m + 1; else b = m;
    }
    return a;
}
__device__ __forceinline__ int64_t upper_bound_nu(const double *nu, int64_t n, double v)
{
    int64_t a = 0, b = n;
    while (a < b) {
        int64_t m = (a + b) >> 1;
        if (nu[m] <= v) a = m + 1; else b = m;
    }
    return a;
}

__global__ void k_tile_ranges(const Prob *__restrict__ probs, int nprob, GridD g, int tile_bins,
                              int64_t ntiles, int lmax, int64_t *tile_lb, int64_t *tile_le,
                              int64_t *counts)
{
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= nprob * ntiles) return;
    int p = (int)(idx / ntiles);
    int64_t t = idx - (int64_t)p * ntiles;
    const Prob &pr = probs[p];
    int64_t lb = 0, le = pr.n;
    if (g.halo > 0) {
        // the lines whose nearest bin lies in the tile's central tile_bins - 2H
        // bins (a line a hair past a boundary still fits the halo: H >= W + 2)
        const double step = (double)(tile_bins - 2 * g.halo);
        const double lo_nu = t == 0 ? g.nu_min - g.cut - 2.0 * g.dnu
                                    : g.nu_min + ((double)t * step - 0.5) * g.dnu;
        lb = lower_bound_nu(pr.nu0, pr.n, lo_nu);
        if (t == ntiles - 1)
            le = upper_bound_nu(pr.nu0, pr.n, g.nu_min + (double)g.nbins * g.dnu + g.cut + 2.0 * g.dnu);
        else
            le = lower_bound_nu(pr.nu0, pr.n, g.nu_min + ((double)(t + 1) * step - 0.5) * g.dnu);
    } else if (has_cut(g)) {
        const double cut = (g.W > 0.0 && !pr.delta) ? g.cut : *pr.cutmax;
        double lo_nu = g.nu_min + (double)(t * tile_bins) * g.dnu - cut - 2.0 * g.dnu;
        double hi_nu = g.nu_min + (double)(t * tile_bins + tile_bins - 1) * g.dnu + cut + 2.0 * g.dnu;
        lb = lower_bound_nu(pr.nu0, pr.n, lo_nu);
        le = upper_bound_nu(pr.nu0, pr.n, hi_nu);
    }
    tile_lb[idx] = lb;
    tile_le[idx] = le;
    counts[idx] = le > lb ? (le - lb + lmax - 1) / lmax : 0;
}

// Exclusive scan of counts[0..m) into off[0..m] (off[m] = total); one block.
__global__ void k_scan(const int64_t *counts, int64_t m, int64_t *off)
{
    __shared__ int64_t part[1024];
    int tid = threadIdx.x;
    int64_t seg = (m + blockDim.x - 1) / blockDim.x;
    int64_t a = tid * seg, b = min(m, a + seg);
    int64_t s = 0;
    for (int64_t i = a; i < b; ++i) s += counts[i];
    part[tid] = s;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        int64_t v = tid >= o ? part[tid - o] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    int64_t run = tid ? part[tid - 1] : 0;
    for (int64_t i = a; i < b; ++i) {
        off[i] = run;
        run += counts[i];
    }
    if (tid == blockDim.x - 1) off[m] = part[tid];
}

// ---- the gather ---------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void stage_line(const Prob &pr, const GridD &g, int64_t l, int scale,
                                           LineT<R> *out, double *nu_out)
{
    double nu0 = pr.nu0[l];
    int i0, lo, hi;
    double r;
    const CutW cw = line_cut(pr, g, l, nu0);
    bool any = line_geometry_w(line_pos(pr, l), g, cw.nocut, cw.W, &i0, &r, &lo, &hi);
    LineT<R> q;
    int c;
    double rn;
    nearest_bin(i0, r, &c, &rn);
    q.i0 = c;
    q.lo = lo;
    q.hi = hi;
    q.r = (R)rn;
    q.pad = 0;
    if (!any) {
        q.b = R(1);
        q.y = R(1);
        q.s = R(0);
    } else if (sizeof(R) == 4) {
        float aDinv, y, P;
        int e2;
        if (pr.pre) {
            aDinv = pr.aDinv_pre[l];
            y = pr.y_pre[l];
            double v = pr.S_pre[l] * (double)aDinv * kInvSqrtPi;
            P = (float)ldexp(v, -scale);
            e2 = 0;
            q.s = (R)P;
        } else {
            line_strength_f32(pr, l, &P, &e2, &aDinv, &y);
            q.s = (R)ldexpf(P, e2 - scale);
        }
        q.b = (R)((float)g.dnu * aDinv);
        q.y = (R)y;
    } else {
        double S, aDinv, y;
        if (pr.pre) {
            S = pr.S_pre[l];
            aDinv = (double)pr.aDinv_pre[l];
            y = (double)pr.y_pre[l];
        } else {
            line_strength_f64(pr, l, &S, &aDinv, &y);
        }
        q.s = (R)(S * aDinv * kInvSqrtPi);
        q.b = (R)(g.dnu * aDinv);
        q.y = (R)y;
    }
    // the plinth: this line's value at its cutting length, x_cut = W b
    q.h = (g.plinth && any && !cw.nocut) ? q.s * profile_rel<R>(g.profile, (R)cw.W * q.b, q.y, q.b)
                                         : R(0);
    *out = q;
    *nu_out = nu0;
}

// Contribution s * Re w(x + iy) of one (line, bin) pair; sy = s * y / sqrt(pi).
template <typename R> __device__ __forceinline__ R pair_value(R x, R y, R Y, R s, R sy)
{
    R X = x * x;
    R r2 = X + Y;
    if (r2 >= BandLimits<R>::gh3) {
        if (r2 >= BandLimits<R>::gh2) return sy * gh1_F<R>(r2);
        return sy * gh2_F<R>(X, Y, r2);
    }
    if (r2 >= BandLimits<R>::gh4) return sy * gh3_F<R>(X, Y, r2);
    if (r2 >= BandLimits<R>::core) return sy * gh4_F<R>(X, Y, r2);
    return s * core_re<R>(x, y);
}

template <typename R, int BPT>
__global__ void __launch_bounds__(NTHREADS, 2)
    k_gather(const Prob *__restrict__ probs, GridD g, int64_t ntiles, int64_t m,
             const int64_t *__restrict__ item_off,
             const int64_t *__restrict__ tile_lb, const int64_t *__restrict__ tile_le, int lmax,
             unsigned long long *counter)
{
    constexpr int TILE = NWARPS * 32 * BPT;
    __shared__ LineT<R> sl[NWARPS * 32];   // 32 staged lines per warp
    __shared__ long long s_item, s_pt, s_lb, s_le;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (;;) {
        if (warp == 0) {
            long long pt_, lb_, le_;
            const long long item =
                fetch_item(counter, item_off, m, tile_lb, tile_le, lmax, lane, &pt_, &lb_, &le_);
            if (lane == 0) {
                s_item = item;
                s_pt = pt_;
                s_lb = lb_;
                s_le = le_;
            }
        }
        __syncthreads();
        if (s_item < 0) break;
        const int64_t pt = s_pt;
        const int p = (int)(pt / ntiles);
        const int64_t t = pt - (int64_t)p * ntiles;
        const int64_t l_begin = s_lb, l_end = s_le;
        const Prob &pr = probs[p];
        const int scale = (sizeof(R) == 4) ? *pr.scale_exp : 0;

        const int wb0 = (int)(t * TILE) + warp * 32 * BPT;  // first bin of this warp
        const double wcut = (g.W > 0.0 && !pr.delta) ? g.cut : (has_cut(g) ? *pr.cutmax : 0.0);
        const double wnu_lo = g.nu_min + (double)wb0 * g.dnu - wcut - 2.0 * g.dnu;
        const double wnu_hi = g.nu_min + (double)(wb0 + 32 * BPT - 1) * g.dnu + wcut + 2.0 * g.dnu;

        R acc[BPT], shi[BPT], slo[BPT];
#pragma unroll
        for (int j = 0; j < BPT; ++j) acc[j] = shi[j] = slo[j] = R(0);
        int nsince = 0;

        // this warp's candidate lines among the item's (bisection on nu0); each
        // warp stages its own lines, 32 at a time, so no warp waits for another
        int64_t wa = l_begin, wb = l_end;
        if (has_cut(g)) {
            int64_t lo = l_begin, hi = l_end;
            while (lo < hi) {
                const int64_t m = (lo + hi) >> 1;
                if (pr.nu0[m] < wnu_lo) lo = m + 1; else hi = m;
            }
            wa = lo;
            hi = l_end;
            while (lo < hi) {
                const int64_t m = (lo + hi) >> 1;
                if (pr.nu0[m] <= wnu_hi) lo = m + 1; else hi = m;
            }
            wb = lo;
        }
        LineT<R> *const wsl = sl + warp * 32;
        for (int64_t cs = wa; cs < wb; cs += 32) {
            const int nl = (int)min((int64_t)32, wb - cs);
            __syncwarp();
            double nu_unused;
            if (lane < nl) stage_line<R>(pr, g, cs + lane, scale, &wsl[lane], &nu_unused);
            __syncwarp();
            for (int l = 0; l < nl; ++l) {
                const LineT<R> q = wsl[l];
                if (q.hi < wb0 || q.lo > wb0 + 32 * BPT - 1) continue;  // warp-uniform
                // x = (k - r) b for the integer bin offset k = bin - i0: formed as
                // fma(k, b, -r b) with k exact, one rounding, so a bin next to the
                // centre keeps full relative precision whatever the lane's first bin.
                const R kf0 = (R)(wb0 + lane - q.i0);
                const R rb = q.r * q.b;
                const R y = q.y, Y = y * y;
                const R sy = q.s * y * R(kInvSqrtPi);
                const unsigned span = (unsigned)(q.hi - q.lo);
                const int kk = wb0 + lane - q.lo;
#pragma unroll
                for (int j = 0; j < BPT; ++j) {
                    const bool inr = (unsigned)(kk + 32 * j) <= span;
                    const R x = fma(kf0 + R(32 * j), q.b, -rb);
                    const R v = (g.profile == kProfVoigt ? pair_value<R>(x, y, Y, q.s, sy)
                                                         : q.s * profile_rel<R>(g.profile, x, y, q.b)) -
                                q.h;
                    acc[j] += inr ? v : R(0);
                }
                if (sizeof(R) == 4 && ++nsince == FLUSH) {
                    nsince = 0;
#pragma unroll
                    for (int j = 0; j < BPT; ++j) {
                        float sh, e;
                        two_sum((float)shi[j], (float)acc[j], &sh, &e);
                        shi[j] = (R)sh;
                        slo[j] += (R)e;
                        acc[j] = R(0);
                    }
                }
            }
        }
        // fold and publish
#pragma unroll
        for (int j = 0; j < BPT; ++j) {
            const int64_t bin = (int64_t)wb0 + lane + 32 * j;
            double tot;
            if (sizeof(R) == 4) {
                float sh, e;
                two_sum((float)shi[j], (float)acc[j], &sh, &e);
                tot = (double)sh + ((double)slo[j] + (double)e);
            } else {
                tot = (double)acc[j];
            }
            if (bin < g.nbins && tot != 0.0) atomicAdd(pr.acc + bin, tot);
        }
        __syncthreads();
    }
}

// ---- finalize: sigma from the scaled FP64 accumulator --------------------------
// A scale slot still holding its fill value (no line with S > 0) means an
// all-zero accumulator.
constexpr int kNoScale = (int)0x80808080;

template <typename O>
__global__ void k_finalize(const Prob *__restrict__ probs, int nprob, int64_t nbins, O *out,
                           int accumulate)
{
    int p = blockIdx.y;
    const double *acc = probs[p].acc;
    int sc = *probs[p].scale_exp;
    if (sc == kNoScale) sc = 0;
    O *o = out + (int64_t)p * nbins;
    bool over = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nbins;
         i += (int64_t)gridDim.x * blockDim.x) {
        double v = ldexp(acc[i], sc);
        if (accumulate) v += (double)o[i];
        O ov = (O)v;
        over |= isinf((double)ov) && !isinf(v);
        o[i] = ov;
    }
    if (over) atomicOr(probs[p].status, kStatusRange);
}

// ---- pair / band counts (instrumentation) --------------------------------------
__global__ void k_count_pairs(Prob p, GridD g, unsigned long long *counts)
{
    unsigned long long c[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < p.n;
         l += (int64_t)gridDim.x * blockDim.x) {
        // the FP32 kernels' geometry (its pair total must equal the oracle's)
        int cb, lo, hi;
        float rnf;
        CutW cw;
        if (!line_geometry_cut(p, g, l, &cw, &cb, &rnf, &lo, &hi)) continue;
        const double r = (double)rnf;
        double S, aDinv, y;
        line_strength_f64(p, l, &S, &aDinv, &y);
        double b = g.dnu * aDinv;
        double klo = (double)(lo - cb), khi = (double)(hi - cb);
        c[0] += (unsigned long long)(hi - lo + 1);
        // pairs with r2 < R2: |k - rn| < sqrt(R2 - y^2) / b, k = i - cb
        const double R2[4] = {1.5e6, 2500.0, 200.0, 64.0};
        unsigned long long inside[4];
        for (int t = 0; t < 4; ++t) {
            double D2 = R2[t] - y * y;
            if (D2 <= 0.0) { inside[t] = 0; continue; }
            double D = sqrt(D2) / b;
            double a = fmax(klo, floor(r - D) + 1.0), e = fmin(khi, ceil(r + D) - 1.0);
            inside[t] = e >= a ? (unsigned long long)(e - a + 1.0) : 0ull;
        }
        unsigned long long tot = (unsigned long long)(hi - lo + 1);
        c[1] += tot - inside[0];
        c[2] += inside[0] - inside[1];
        c[3] += inside[1] - inside[2];
        c[4] += inside[2] - inside[3];
        c[5] += inside[3];
        // pairs with R8 <= r2 < 64, R8 = max(26, ln(1.13e9) - ln y) (at most 64):
        // the ring the FP32C short-line batches take with the 8-node rule
        const double R8 = fmin(64.0, fmax(26.0, 20.845483 - log(y)));
        const double D2 = R8 - y * y;
        unsigned long long in8 = 0;
        if (D2 > 0.0) {
            const double D = sqrt(D2) / b;
            const double a = fmax(klo, floor(r - D) + 1.0), e = fmin(khi, ceil(r + D) - 1.0);
            in8 = e >= a ? (unsigned long long)(e - a + 1.0) : 0ull;
        }
        c[6] += inside[3] > in8 ? inside[3] - in8 : 0ull;
    }
    for (int t = 0; t < 7; ++t) {
        unsigned long long v = c[t];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(counts + t, v);
    }
}

int count_pairs_run(const Prob &p, const GridD &g, unsigned long long *counts_d, cudaStream_t st,
                    int num_sms)
{
    cudaError_t e = cudaMemsetAsync(counts_d, 0, 7 * sizeof(unsigned long long), st);
    if (e) return fail_cuda(e);
    k_count_pairs<<<num_sms * 4, 256, 0, st>>>(p, g, counts_d);
    if ((e = cudaGetLastError())) return fail_cuda(e);
    return HK_OK;
}

// ---- launch profiling (instrumentation) -----------------------------------------
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::vector<cudaEvent_t> g_prof_ev;  // begin, end, begin, end, ...

void gather_profile_record(cudaStream_t st, bool begin)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on) return;
    if (!begin && g_prof_ev.size() % 2 == 0) return;
    cudaEvent_t ev;
    if (cudaEventCreate(&ev) != cudaSuccess) {
        (void)cudaGetLastError();
        return;
    }
    cudaEventRecord(ev, st);
    g_prof_ev.push_back(ev);
}

int gather_profile(int mode, double *ms, int64_t *launches)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    double tot = 0.0;
    int64_t n = 0;
    int rc = HK_OK;
    for (size_t i = 0; i + 1 < g_prof_ev.size(); i += 2) {
        cudaError_t e = cudaEventSynchronize(g_prof_ev[i + 1]);
        float t = 0.0f;
        if (!e) e = cudaEventElapsedTime(&t, g_prof_ev[i], g_prof_ev[i + 1]);
        if (e) rc = fail_cuda(e);
        tot += t;
        ++n;
    }
    for (cudaEvent_t ev : g_prof_ev) cudaEventDestroy(ev);
    g_prof_ev.clear();
    g_prof_on = (mode == 1);
    if (ms) *ms = mode == 1 ? 0.0 : tot;
    if (launches) *launches = mode == 1 ? 0 : n;
    return rc;
}

// ---- descriptor upload through kernel parameters ------------------------------
// Problem descriptors reach the device as kernel arguments (64 per launch,
// ~13 KB of parameters) instead of a copy from pageable host memory, so every
// call is a plain sequence of kernel launches and memsets: it can be captured
// into a CUDA graph and the host array may be freed as soon as the call returns.
constexpr int kProbsPerUpload = 64;
struct ProbChunk {
    Prob p[kProbsPerUpload];
    int n;
};
__global__ void k_store_probs(Prob *dst, const ProbChunk chunk)
{
    for (int i = threadIdx.x; i < chunk.n; i += blockDim.x) dst[i] = chunk.p[i];
}

constexpr int kDoublesPerUpload = 512;
struct DoubleChunk {
    double v[kDoublesPerUpload];
    int n;
};
__global__ void k_store_doubles(double *dst, const DoubleChunk chunk)
{
    for (int i = threadIdx.x; i < chunk.n; i += blockDim.x) dst[i] = chunk.v[i];
}

int upload_probs(Prob *dst, const Prob *src, int n, cudaStream_t st)
{
    for (int off = 0; off < n; off += kProbsPerUpload) {
        ProbChunk c;
        c.n = n - off < kProbsPerUpload ? n - off : kProbsPerUpload;
        for (int i = 0; i < c.n; ++i) c.p[i] = src[off + i];
        k_store_probs<<<1, kProbsPerUpload, 0, st>>>(dst + off, c);
        cudaError_t e = cudaGetLastError();
        if (e) return fail_cuda(e);
    }
    return HK_OK;
}

int upload_doubles(double *dst, const double *src, int n, cudaStream_t st)
{
    for (int off = 0; off < n; off += kDoublesPerUpload) {
        DoubleChunk c;
        c.n = n - off < kDoublesPerUpload ? n - off : kDoublesPerUpload;
        for (int i = 0; i < c.n; ++i) c.v[i] = src[off + i];
        k_store_doubles<<<1, 256, 0, st>>>(dst + off, c);
        cudaError_t e = cudaGetLastError();
        if (e) return fail_cuda(e);
    }
    return HK_OK;
}

// ---- host side ----------------------------------------------------------------

int gather_tile_bins(int precision, int bpt)
{
    return precision == 1 ? NWARPS * 32 * 2 : bpt;
}

// Tiles of a launch: ceil(nbins / tb), or with a halo H ceil(nbins / (tb - 2 H)).
static int64_t tile_count(int64_t nbins, int64_t tb, int halo)
{
    const int64_t step = tb - 2 * (int64_t)halo;
    return (nbins + step - 1) / step;
}

size_t gather_workspace(int nprob, const GridD &g, int precision, int bpt)
{
    const int64_t nbins = g.nbins;
    int64_t tb = gather_tile_bins(precision, bpt);
    // the halo tiling (used unless a pressure shift rules it out) needs more tiles
    int64_t ntiles = tile_count(nbins, tb, precision == 0 ? halo_bins(g, (int)tb) : 0);
    int64_t m = (int64_t)nprob * ntiles;
    size_t bytes = 0;
    auto add = [&](size_t b) { bytes += (b + 255) & ~(size_t)255; };
    add(sizeof(Prob) * nprob);
    add(sizeof(int) * nprob);
    add(sizeof(int64_t) * m);       // tile_lb
    add(sizeof(int64_t) * m);       // tile_le
    add(sizeof(int64_t) * m);       // counts
    add(sizeof(int64_t) * (m + 1)); // item_off
    add(sizeof(unsigned long long) * 2);
    add(sizeof(double) * nprob);    // largest per-line cut
    if (precision == 0) add(sizeof(double) * (size_t)nprob * nbins);
    return bytes;
}

int gather_run(Prob *probs_h, int nprob, const GridD &g, int precision, int bpt, int lmax,
               void *out, int out_f64, int accumulate, char *ws, size_t ws_bytes,
               unsigned *status_d, cudaStream_t st, int num_sms)
{
    int64_t tb = gather_tile_bins(precision, bpt);
    // FP32C short lines: tiles with a halo (every line summed in the one tile
    // that holds its centre), unless a pressure shift moves the centres
    GridD gh = g;
    gh.halo = 0;
    if (precision == 0) {
        bool shifted = false;
        for (int p = 0; p < nprob; ++p) shifted |= probs_h[p].delta != nullptr;
        if (!shifted) gh.halo = halo_bins(g, (int)tb);
    }
    const int64_t ntiles = tile_count(g.nbins, tb, gh.halo);
    int64_t m = (int64_t)nprob * ntiles;
    char *cur = ws;
    auto take = [&](size_t b) {
        char *r = cur;
        cur += (b + 255) & ~(size_t)255;
        return r;
    };
    Prob *probs_d = (Prob *)take(sizeof(Prob) * nprob);
    int *scales = (int *)take(sizeof(int) * nprob);
    int64_t *tile_lb = (int64_t *)take(sizeof(int64_t) * m);
    int64_t *tile_le = (int64_t *)take(sizeof(int64_t) * m);
    int64_t *counts = (int64_t *)take(sizeof(int64_t) * m);
    int64_t *item_off = (int64_t *)take(sizeof(int64_t) * (m + 1));
    unsigned long long *counter = (unsigned long long *)take(sizeof(unsigned long long) * 2);
    double *cutmax = (double *)take(sizeof(double) * nprob);
    // counter[0]: next work item of the persistent gather
    double *acc = nullptr;
    if (precision == 0) acc = (double *)take(sizeof(double) * (size_t)nprob * g.nbins);
    if ((size_t)(cur - ws) > ws_bytes) return HK_ENOMEM;

    for (int p = 0; p < nprob; ++p) {
        probs_h[p].status = status_d;
        probs_h[p].scale_exp = scales + p;
        probs_h[p].cutmax = cutmax + p;
        if (precision == 0) probs_h[p].acc = acc + (size_t)p * g.nbins;
        else probs_h[p].acc = (double *)out + (size_t)p * g.nbins;
    }
    cudaError_t e;
    int urc = upload_probs(probs_d, probs_h, nprob, st);
    if (urc) return urc;
    if ((e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long) * 2, st))) return fail_cuda(e);
    if (precision == 0) {
        if ((e = cudaMemsetAsync(acc, 0, sizeof(double) * (size_t)nprob * g.nbins, st)))
            return fail_cuda(e);
        // INT_MIN in every scale slot: 0x80 bytes give 0x80808080 < any real exponent
        if ((e = cudaMemsetAsync(scales, 0x80, sizeof(int) * nprob, st))) return fail_cuda(e);
        // enough warps in flight to keep the line reads at HBM speed
        dim3 grid(num_sms * 16, nprob);
        k_scale_prepass<<<grid, 256, 0, st>>>(probs_d, nprob, g);
        if ((e = cudaGetLastError())) return fail_cuda(e);
    } else if (!accumulate) {
        if ((e = cudaMemsetAsync(out, 0, sizeof(double) * (size_t)nprob * g.nbins, st)))
            return fail_cuda(e);
    }
    bool shifted = false;
    for (int p = 0; p < nprob; ++p) shifted |= probs_h[p].delta != nullptr;
    if (g.cut_mode == kCutDoppler || g.cut_mode == kCutLorentz || (shifted && has_cut(g))) {
        if ((e = cudaMemsetAsync(cutmax, 0, sizeof(double) * nprob, st))) return fail_cuda(e);
        dim3 grid(num_sms * 4, nprob);
        k_cut_max<<<grid, 256, 0, st>>>(probs_d, nprob, g);
        if ((e = cudaGetLastError())) return fail_cuda(e);
    }
    {
        int64_t blocks = (m + 255) / 256;
        k_tile_ranges<<<(unsigned)blocks, 256, 0, st>>>(probs_d, nprob, gh, (int)tb, ntiles, lmax,
                                                        tile_lb, tile_le, counts);
        if ((e = cudaGetLastError())) return fail_cuda(e);
        k_scan<<<1, 1024, 0, st>>>(counts, m, item_off);
        if ((e = cudaGetLastError())) return fail_cuda(e);
    }
    {
        dim3 grid(num_sms * 2);
        gather_profile_record(st, true);
        if (precision == 0) {
            int rc = gather_f32_launch(probs_d, gh, ntiles, m, item_off, tile_lb, tile_le, lmax,
                                       counter, st, num_sms, (int)tb);
            if (rc) return rc;
        } else {
            k_gather<double, 2><<<grid, NTHREADS, 0, st>>>(probs_d, g, ntiles, m, item_off, tile_lb, tile_le, lmax, counter);
        }
        if ((e = cudaGetLastError())) return fail_cuda(e);
        gather_profile_record(st, false);
    }
    if (precision == 0) {
        dim3 grid(num_sms * 4, nprob);
        if (out_f64)
            k_finalize<double><<<grid, 256, 0, st>>>(probs_d, nprob, g.nbins, (double *)out, accumulate);
        else
            k_finalize<float><<<grid, 256, 0, st>>>(probs_d, nprob, g.nbins, (float *)out, accumulate);
        if ((e = cudaGetLastError())) return fail_cuda(e);
    }
    return HK_OK;
}

}  // namespace hk
