// hk_internal.cuh -- device-side building blocks of libhk (sm_103a).
//
// * physical constants (the device copy; a test checks them against the
//   values printed in Sect. 2.2 / 2.2.2 of arXiv:2101.02005);
// * the banded Faddeeva evaluator Re w(x + iy) used by every kernel;
// * the per-line prologue: bin geometry (integer centre bin, remainder, cut
//   range) and the scaled strength S * alpha_D^-1 / sqrt(pi).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace hk {

// ---- constants ------------------------------------------------------------
constexpr double kC = 2.99792458e10;      // cm/s            (Sect. 2.2.2, Eq. S)
constexpr double kKB = 1.3806489e-16;     // erg/K           (Sect. 2.2, Eq. gammaD)
constexpr double kH = 6.62606957e-27;     // erg s, CODATA 2010 (the paper prints no h)
constexpr double kAMU = 1.660538921e-24;  // g, CODATA 2010
constexpr double kPI = 3.14159265358979323846;
constexpr double kC2 = kH * kC / kKB;     // second radiation constant, cm K
constexpr double kInvSqrtPi = 0.5641895835477563;
constexpr double kInvPi = 0.3183098861837907;
constexpr double kInvLn2 = 1.4426950408889634;

// Cut modes and line profiles (the values of HK_CUT_* and HK_PROFILE_* in hk.h).
constexpr int kCutFixed = 0, kCutNone = 1, kCutDoppler = 2, kCutLorentz = 3;
constexpr int kProfVoigt = 0, kProfLorentz = 1, kProfDoppler = 2, kProfBinned = 3;

// ---- Faddeeva function: banded evaluation of Re w(x + iy), y >= 0 ----------
//
// The a-u plane split of Sect. 2.2.3 (Table regions) is prior art; the bands
// here are chosen so that every band meets ~1e-6 relative error on Re w in
// FP32, including y -> 0 where Re w = exp(-x^2) + O(y):
//
//   r2 = x^2 + y^2      method                                  rel. error
//   r2 >= 1.5e6         1-node Gauss-Hermite  y / (sqrt(pi) r2)   1.0e-6
//   2500 <= r2 < 1.5e6  2-node Gauss-Hermite                      4e-7
//   200  <= r2 < 2500   3-node Gauss-Hermite                      7e-7
//   64   <= r2 < 200    4-node Gauss-Hermite                      1e-6
//   r2 < 64             trapezoid on (i/pi) int e^{-t^2}/(z-t) dt with
//                       step 1/2, |t| <= 5.75 (FP64; t in [-4, 4.75] in FP32), plus the pole correction
//                       2 e^{-z^2}/(1 -/+ e^{-2 pi i z/h}) and a half-step
//                       shift of the nodes when x is near one
//                       (Chiarella & Reichel 1968; Matta & Reichel 1971)
//
// An n-node Gauss-Hermite rule applied to w = (i/pi) int e^{-t^2}/(z - t) dt
// gives, for symmetric node pairs +-t_j with normalised weights W_j
// (sum of all W = 1) and tau_j = t_j^2,
//   Re w = (y / sqrt(pi)) [ sum_pairs 2 W_j (r2 + tau_j) / |z^2 - tau_j|^2 + W_0 / r2 ],
//   |z^2 - tau|^2 = (x^2 - y^2 - tau)^2 + 4 x^2 y^2,
// a sum of positive terms: relative accuracy survives y -> 0.
// The GH functions below return the bracket F, so Re w = y F / sqrt(pi).

enum Band : int { kBandGH1 = 0, kBandGH2 = 1, kBandGH3 = 2, kBandGH4 = 3, kBandCore = 4 };

template <typename R> struct BandLimits {
    static constexpr R core = R(64), gh4 = R(200), gh3 = R(2500), gh2 = R(1.5e6);
};

template <typename R> __device__ __forceinline__ R gh1_F(R r2) { return R(1) / r2; }

// 2 nodes: t = +-1/sqrt(2), W = 1/2 each -> 2W = 1.
template <typename R> __device__ __forceinline__ R gh2_F(R X, R Y, R r2)
{
    R a = X - (Y + R(0.5));
    R d = a * a + X * (R(4) * Y);
    return (r2 + R(0.5)) / d;
}

// 3 nodes: t = 0 (W0 = 2/3) and +-sqrt(3/2) (W = 1/6 each).
template <typename R> __device__ __forceinline__ R gh3_F(R X, R Y, R r2)
{
    R a = X - (Y + R(1.5));
    R d = a * a + X * (R(4) * Y);
    // (2/3)/r2 + (1/3)(r2 + 3/2)/d over a common denominator
    return (R(2.0 / 3.0) * d + R(1.0 / 3.0) * (r2 + R(1.5)) * r2) / (r2 * d);
}

// 4 nodes: tau = (3 -+ sqrt 6)/2, W = (3 +- sqrt 6)/12.
template <typename R> __device__ __forceinline__ R gh4_F(R X, R Y, R r2)
{
    const R ta = R(0.27525512860841106), tb = R(2.724744871391589);
    const R wa = R(2 * 0.4541241452319315), wb = R(2 * 0.04587585476806851);
    R a1 = X - (Y + ta), a2 = X - (Y + tb);
    R fy = X * (R(4) * Y);
    R d1 = a1 * a1 + fy, d2 = a2 * a2 + fy;
    return (wa * (r2 + ta) * d2 + wb * (r2 + tb) * d1) / (d1 * d2);
}

// 1/a from the hardware reciprocal alone (PTX rcp.approx.ftz.f32: at most
// 1 ulp, subnormal arguments and results flushed to zero, so no fix-up path).
// Every float sum here is scaled so that its peak is near 1: a term that
// flushes lies below 2^-126 of the peak.
__device__ __forceinline__ float rcp_ftz(float a)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}

template <typename R> struct Math;
template <> struct Math<float> {
    static __device__ __forceinline__ float exp_(float a) { return expf(a); }
    static __device__ __forceinline__ float expm1_(float a) { return expm1f(a); }
    static __device__ __forceinline__ void sincos_(float a, float *s, float *c) { sincosf(a, s, c); }
    static __device__ __forceinline__ void sincospi_(float a, float *s, float *c) { sincospif(a, s, c); }
    static __device__ __forceinline__ float floor_(float a) { return floorf(a); }
    static __device__ __forceinline__ float div_(float a, float b) { return a * rcp_ftz(b); }
};
template <> struct Math<double> {
    static __device__ __forceinline__ double exp_(double a) { return exp(a); }
    static __device__ __forceinline__ double expm1_(double a) { return expm1(a); }
    static __device__ __forceinline__ void sincos_(double a, double *s, double *c) { sincos(a, s, c); }
    static __device__ __forceinline__ void sincospi_(double a, double *s, double *c) { sincospi(a, s, c); }
    static __device__ __forceinline__ double floor_(double a) { return floor(a); }
    static __device__ __forceinline__ double div_(double a, double b) { return a / b; }
};

// Trapezoid nodes t = n/2 (W0) and (n + 1/2)/2 (W1), n = -11 .. 11; weights e^{-t^2}.
#define HK_TRAP_W0                                                                           \
    {7.28772409581969219e-14, 1.38879438649640209e-11, 1.60522805518561165e-09,              \
     1.12535174719259116e-07, 4.78511739212900875e-06, 1.23409804086679561e-04,              \
     1.93045413622770930e-03, 1.83156388887341787e-02, 1.05399224561864333e-01,              \
     3.67879441171442334e-01, 7.78800783071404878e-01, 1.00000000000000000e+00,              \
     7.78800783071404878e-01, 3.67879441171442334e-01, 1.05399224561864333e-01,              \
     1.83156388887341787e-02, 1.93045413622770930e-03, 1.23409804086679561e-04,              \
     4.78511739212900875e-06, 1.12535174719259116e-07, 1.60522805518561165e-09,              \
     1.38879438649640209e-11, 7.28772409581969219e-14}
#define HK_TRAP_W1                                                                           \
    {1.07092323825080766e-12, 1.58939100945163677e-10, 1.43072419185676882e-08,              \
     7.81148940830449097e-07, 2.58681002226541202e-05, 5.19574682154838445e-04,              \
     6.32971542748574697e-03, 4.67706223839589805e-02, 2.09611387151097811e-01,              \
     5.69782824730923010e-01, 9.39413062813475808e-01, 9.39413062813475808e-01,              \
     5.69782824730923010e-01, 2.09611387151097811e-01, 4.67706223839589805e-02,              \
     6.32971542748574697e-03, 5.19574682154838445e-04, 2.58681002226541202e-05,              \
     7.81148940830449097e-07, 1.43072419185676882e-08, 1.58939100945163677e-10,              \
     1.07092323825080766e-12, 4.37661850287085020e-15}

// sin(pi a), cos(pi a) for the float core: exact reduction a = n + f with
// |f| <= 1/2 (a - rint(a) is exact), then the hardware sine and cosine of
// pi f (absolute error ~4e-7 on [-pi/2, pi/2]) and the sign of n's parity.
__device__ __forceinline__ void sincospi_core(float a, float *s, float *c)
{
    const float n = rintf(a);
    const float f = a - n;
    float sf, cf;
    __sincosf((float)kPI * f, &sf, &cf);
    const bool odd = ((int)n) & 1;
    *s = odd ? -sf : sf;
    *c = odd ? -cf : cf;
}

// sin, cos of a >= 0 for the float core: a = 2 pi k + r with r in [-pi, pi]
// (2 pi split in two floats so the reduction keeps ~1e-7 absolute), then the
// hardware sine and cosine.
__device__ __forceinline__ void sincos_core(float a, float *s, float *c)
{
    const float k = rintf(a * (float)(0.5 * kInvPi));
    const float r = fmaf(-k, 6.28318548202514648f, fmaf(-k, -1.7484556e-7f, a));
    __sincosf(r, s, c);
}

// Re w(x + iy) for r2 < 64 (any x sign; uses |x|).
template <typename R> __device__ __forceinline__ R core_re(R x, R y)
{
    constexpr double w0[23] = HK_TRAP_W0;
    constexpr double w1[23] = HK_TRAP_W1;
    R ax = x < R(0) ? -x : x;
    R Y = y * y;
    R u = ax * R(2);                      // x / h, h = 1/2
    R fr = u - Math<R>::floor_(u);
    bool sh = !(fr > R(0.25) && fr < R(0.75));  // x within h/4 of a node: shift lattice
    R off = sh ? R(0.5) : R(0);
    R s = R(0);
    // nodes t = (n + off) / 2: x - t = (x - off / 2) - n / 2
    const R axs = ax - off * R(0.5);
    if constexpr (sizeof(R) == 4) {
        // float: nodes n = -8 .. 9, i.e. t in [-4, 4.5] (shifted: [-3.75, 4.75]);
        // with |x| >= 0 the dropped terms are below 1e-8 of Re w for every
        // r2 < 64 (|x - t| >= 1/8 by the lattice shift; 6e-9 against scipy's
        // wofz in exact arithmetic)
#pragma unroll
        for (int n = -8; n <= 9; ++n) {
            R wt = sh ? R(w1[n + 11]) : R(w0[n + 11]);
            R d = axs - R(0.5 * n);
            s += Math<R>::div_(wt, d * d + Y);
        }
    } else {
#pragma unroll
        for (int n = -11; n <= 11; ++n) {
            R wt = sh ? R(w1[n + 11]) : R(w0[n + 11]);
            R d = axs - R(0.5 * n);
            s += Math<R>::div_(wt, d * d + Y);
        }
    }
    R re = R(0.5 * kInvPi) * y * s;       // (h / pi) y sum e^{-t^2} / ((x-t)^2 + y^2)
    if (y < R(2)) {
        // Re[ 2 e^{-z^2} / (1 -/+ e^{-2 pi i z / h}) ], h = 1/2: eta = 4 pi y, theta = 4 pi x
        // e^eta - 1; in float E itself is what matters (den >= 2 E), so the
        // hardware exponential less 1 serves
        R em = sizeof(R) == 4 ? (R)(__expf((float)(R(4 * kPI) * y)) - 1.0f)
                              : Math<R>::expm1_(R(4 * kPI) * y);
        R E = R(1) + em;
        R sn, cs;
        R s2, c2;
        if (sizeof(R) == 4) {
            float sf, cf, s2f, c2f;
            sincospi_core((float)(R(4) * ax), &sf, &cf);
            sincos_core((float)(R(2) * ax * y), &s2f, &c2f);
            sn = (R)sf;
            cs = (R)cf;
            s2 = (R)s2f;
            c2 = (R)c2f;
        } else {
            Math<R>::sincospi_(R(4) * ax, &sn, &cs);
            Math<R>::sincos_(R(2) * ax * y, &s2, &c2);
        }
        if (sh) {                          // theta + pi for the shifted lattice
            sn = -sn;
            cs = -cs;
        }
        R num = c2 * (R(1) - E * cs) - s2 * E * sn;
        R den = em * em + R(2) * E * (R(1) - cs);
        if (sizeof(R) == 4) {
            // cs <= 0 on either lattice, so den >= 2 E >= 2: a bare reciprocal;
            // the hardware exponential's relative error, |arg| * 2^-24, stays
            // below ~1e-6 wherever this term matters (it is below e^-10 of Re w
            // when |arg| > 16)
            re += R(2) * (R)__expf((float)(Y - ax * ax)) * num * (R)rcp_ftz((float)den);
        } else {
            re += R(2) * Math<R>::exp_(Y - ax * ax) * num / den;
        }
    }
    return re;
}

// Re w for any band; `X` = x^2, `Y` = y^2.
template <typename R> __device__ __forceinline__ R voigt_re(R x, R y)
{
    R X = x * x, Y = y * y, r2 = X + Y;
    const R k = R(kInvSqrtPi);
    if (r2 >= BandLimits<R>::gh3) {
        if (r2 >= BandLimits<R>::gh2)
            return k * y * gh1_F<R>(r2);
        return k * y * gh2_F<R>(X, Y, r2);
    }
    if (r2 >= BandLimits<R>::gh4)
        return k * y * gh3_F<R>(X, Y, r2);
    if (r2 >= BandLimits<R>::core)
        return k * y * gh4_F<R>(X, Y, r2);
    return core_re<R>(x, y);
}

// A line's value at offset x (in alpha_D; y = Gamma_L / alpha_D, b = dnu /
// alpha_D) relative to s = S alpha_D^-1 / sqrt(pi), for each profile of
// Sect. 2.1: Voigt Re w(x + iy); Lorentz (y / sqrt(pi)) / (x^2 + y^2);
// Doppler exp(-x^2); binned Gaussian (the Doppler profile averaged over the
// bin) sqrt(pi)/(2b) [erf(|x| + b/2) - erf(|x| - b/2)], as a difference of
// erfc of positive arguments away from the centre so that no two values near
// 1 are subtracted.
template <typename R> __device__ __forceinline__ R profile_rel(int profile, R x, R y, R b)
{
    switch (profile) {
    case kProfLorentz:
        return R(kInvSqrtPi) * y / (x * x + y * y);
    case kProfDoppler:
        return exp(-x * x);
    case kProfBinned: {
        const R ax = x < R(0) ? -x : x, hb = R(0.5) * b;
        const R a = ax - hb, c = ax + hb;
        const R v = a >= R(0) ? erfc(a) - erfc(c) : erf(c) + erf(-a);
        return R(0.5 / kInvSqrtPi) / b * v;
    }
    default:
        return voigt_re<R>(x, y);
    }
}

// ---- problem descriptors ----------------------------------------------------

// One sigma array to compute: one species at one (T, P), scalars prepared on
// the host in FP64.
struct Prob {
    // line fields (device)
    const double *nu0;
    const float *S_ref, *A, *g_up, *E_low, *gamma, *n_T;
    const double *S_pre;        // precomputed mode: S, alphaD_inv, y
    const float *aDinv_pre, *y_pre;
    int64_t n;
    int s_mode;                 // 0 S_ref scaling, 1 Einstein A
    int pre;                    // precomputed-parameter mode
    // strength
    double K2;                  // log2 Boltzmann slope: S-mode -c2(1/T - 1/T_ref)/ln2, A-mode -c2/(T ln2)
    double qratio;              // S-mode Q(T_ref)/Q(T); A-mode 1/(8 pi c Q(T))
    double c2T, c2Tref;         // c2/T, c2/T_ref
    double mass_scale;          // 1/m[g] with HK_PER_GRAM, else 1
    // widths
    double aD_coef;             // alphaD_inv = aD_coef / nu0, aD_coef = c sqrt(m / (2 k_B T))
    double log2_tratio;         // log2(T_ref / T)
    double press;               // P / P_ref
    double inv_Pref;            // 1 / P_ref
    double nat_coef;            // 1 / (4 pi c)
    double tratio;              // T_ref / T
    const float *gamma_self;    // HITRAN self widths (gamma is then gamma_air), or null
    const float *delta;         // pressure shifts (cm^-1 per P_ref), or null
    double press_air, press_self;   // (P - P_self) / P_ref, P_self / P_ref
    float press_air_f, press_self_f;
    double K_D;                 // sqrt(ln 2) sqrt(2 k_B T / m) / c: Gamma_D = nu0 K_D
    const double *cutmax;       // device: largest cutting length of the lines (per-line modes)
    // device: each line's bin geometry (c, rn as float bits, lo, hi), computed
    // once for problems that share it (a fixed cut or none, no pressure shift),
    // or null (the FP32C kernel then computes it per record)
    const int4 *geo;
    // the same scalars rounded to float (set with them on the host), for the
    // FP32 strength; K2 as a float pair K2_hi + K2_lo (about 48 bits)
    float qratio_f, c2T_f, c2Tref_f, mass_scale_f, aD_coef_f, log2_tratio_f, press_f,
        nat_coef_f, K2_hi, K2_lo;
    // outputs
    double *acc;                // [nbins] FP64 accumulator (or the FP64 output itself)
    int *scale_exp;             // device int: sigma in acc is scaled by 2^-scale (FP32C)
    unsigned *status;           // device status word (HK_STATUS_* bits)
};

// Bits of the per-device status word.
constexpr unsigned kStatusRange = 1u;    // a float output overflowed
constexpr unsigned kStatusTimeout = 2u;  // a bounded device wait gave up

struct GridD {
    double nu_min, dnu, inv_dnu;
    double W;                   // fixed cut / dnu (as cut * inv_dnu); <= 0: no fixed cut
    double cut;                 // fixed cut, cm^-1 (0 without one)
    int64_t nbins;
    int Wi;                     // floor(W) for 0 < W < 2^30, else -1 (no fast cut path)
    float Wf;                   // W - Wi rounded to float
    int cut_mode;               // kCut*: per-line modes take cut_factor times a half width
    double cut_factor;
    int plinth;                 // subtract each line's value at its cutting length
    int profile;                // kProf*
    int halo;                   // FP32C short lines: tile halo in bins (0: tiles without halo)
};

// Tiles with a halo (FP32C, the short-line batch instances: Voigt profile,
// fixed cut of 2W + 1 < 1024 bins, with or without the plinth): a tile of `tile_bins` bins owns
// the lines whose nearest bin lies in its central tile_bins - 2H bins, and
// its window reaches H bins further on each side, H a multiple of 32 with
// H >= W + 2 -- every line is summed in one tile, unclipped.  Returns H, or 0
// when the cut is too wide to leave at least 256 central bins.
__device__ __host__ __forceinline__ int halo_bins(const GridD &g, int tile_bins)
{
    if (g.cut_mode != kCutFixed || !(g.W > 0.0) || g.profile != kProfVoigt ||
        2.0 * g.W + 1.0 >= 1024.0)
        return 0;
    const int need = (int)g.W + 3;   // ceil(W) + 2, W not an integer or W + 1 + 2
    const int H = 32 * ((need + 31) / 32);
    return tile_bins - 2 * H >= 256 ? H : 0;
}

// Whether the lines have a cut at all (fixed or per line).
__device__ __host__ __forceinline__ bool has_cut(const GridD &g)
{
    return g.cut_mode == kCutDoppler || g.cut_mode == kCutLorentz || g.W > 0.0;
}

// Per-line kernel parameters, as staged in shared memory.
struct LineP {
    float b;     // dnu * alphaD^-1 (x step per bin)
    float r;     // centre offset from bin i0 in bins, in [-1/2, 1/2] (see nearest_bin)
    float y;     // Gamma_L * alphaD^-1
    float s;     // S * alphaD^-1 / sqrt(pi) * 2^-scale  (FP32C)
    int i0;      // nearest bin to the centre
    int lo, hi;  // inclusive bin range inside the cut and the grid; empty if lo > hi
    int pad;
};

// Cut predicate of the FP64 reading: |k - r| <= W (no FMA contraction).
__device__ __forceinline__ bool in_cut(long long k, double r, double W)
{
    return fabs(__dsub_rn((double)k, r)) <= W;
}

// One line's cutting length in bins.  nocut: the whole grid.  Per-line
// modes: W = (factor * Gamma) * inv_dnu with Gamma = nu0 * K_D (Doppler) or
// the FP64 Lorentz half width A/(4 pi c) + gamma (T_ref/T)^n P/P_ref, in the
// operation order of the oracle's definition.  Wi, Wf: the FP32 split of W
// (Wi = -1 when W >= 2^30: no fast path).
struct CutW {
    bool nocut;
    double W;
    int Wi;
    float Wf;
};

// Where line l sits on the grid: nu0, or nu0 + delta P / P_ref (FP64) with a
// pressure shift.
__device__ __forceinline__ double line_pos(const Prob &p, int64_t l)
{
    const double nu0 = p.nu0[l];
    return p.delta ? __dadd_rn(nu0, __dmul_rn((double)p.delta[l], p.press)) : nu0;
}

__device__ __forceinline__ CutW line_cut(const Prob &p, const GridD &g, int64_t l, double nu0)
{
    CutW c;
    if (g.cut_mode == kCutDoppler || g.cut_mode == kCutLorentz) {
        double G;
        if (g.cut_mode == kCutDoppler) {
            G = __dmul_rn(nu0, p.K_D);
        } else {
            const double nat = p.A ? __ddiv_rn((double)p.A[l], 4.0 * kPI * kC) : 0.0;
            const double tn = pow(p.tratio, (double)p.n_T[l]);
            G = p.gamma_self
                    ? __dadd_rn(nat, __dmul_rn(tn, __dadd_rn(__dmul_rn((double)p.gamma[l], p.press_air),
                                                             __dmul_rn((double)p.gamma_self[l],
                                                                       p.press_self))))
                    : __dadd_rn(nat, __dmul_rn(__dmul_rn((double)p.gamma[l], tn), p.press));
        }
        c.nocut = false;
        c.W = __dmul_rn(__dmul_rn(g.cut_factor, G), g.inv_dnu);
        if (c.W >= 0.0 && c.W < 1073741824.0) {
            c.Wi = (int)floor(c.W);
            c.Wf = (float)__dsub_rn(c.W, (double)c.Wi);
        } else {
            c.Wi = -1;
            c.Wf = 0.0f;
        }
    } else {
        c.nocut = !(g.W > 0.0);
        c.W = g.W;
        c.Wi = g.Wi;
        c.Wf = g.Wf;
    }
    return c;
}

// Bin geometry of one line with cutting length W bins (nocut: the whole
// grid).  Returns false if no bin of the grid is inside.
__device__ __forceinline__ bool line_geometry_w(double nu0, const GridD &g, bool nocut, double W,
                                                int *i0_out, double *r_out, int *lo_out,
                                                int *hi_out)
{
    double u = __dmul_rn(__dsub_rn(nu0, g.nu_min), g.inv_dnu);
    double f = floor(u);
    double r = __dsub_rn(u, f);
    long long i0 = (long long)f;
    long long lo, hi;
    if (nocut) {
        lo = 0;
        hi = g.nbins - 1;
    } else {
        long long kh = (long long)floor(__dadd_rn(r, W));
        long long kl = (long long)ceil(__dsub_rn(r, W));
        // walk to the exact predicate boundary (at most a step or two)
        for (int it = 0; it < 4 && in_cut(kh + 1, r, W); ++it) ++kh;
        for (int it = 0; it < 4 && !in_cut(kh, r, W) && kh >= kl; ++it) --kh;
        for (int it = 0; it < 4 && in_cut(kl - 1, r, W); ++it) --kl;
        for (int it = 0; it < 4 && !in_cut(kl, r, W) && kl <= kh; ++it) ++kl;
        lo = i0 + kl;
        hi = i0 + kh;
        if (lo < 0) lo = 0;
        if (hi > g.nbins - 1) hi = g.nbins - 1;
    }
    *r_out = r;
    if (!(nu0 > 0.0)) hi = lo - 1;  // no Doppler width for nu0 <= 0 (Eq. gammaD): ignored
    if (hi < lo || f < -2147483647.0 || f > 2147483647.0) {
        // empty: a range no bin index can fall into, so every range test fails
        *i0_out = 0;
        *lo_out = 0x3fffffff;
        *hi_out = -0x3fffffff;
        return hi >= lo;  // an in-range line with an int32-overflowing centre cannot occur
    }
    *i0_out = (int)i0;
    *lo_out = (int)lo;
    *hi_out = (int)hi;
    return true;
}

// The grid's fixed cut (or none).
__device__ __forceinline__ bool line_geometry(double nu0, const GridD &g, int *i0_out,
                                              double *r_out, int *lo_out, int *hi_out)
{
    return line_geometry_w(nu0, g, !(g.W > 0.0), g.W, i0_out, r_out, lo_out, hi_out);
}

// Bin geometry for the FP32 kernels, with as little FP64 arithmetic as the
// exact cut decision allows (FP64 throughput is a small fraction of FP32).
// u, i0 = floor(u) and r = u - i0 are the FP64 values of line_geometry.  The
// bounds kh = max k with |k - r| <= W and kl = min such k (k = i - i0) are
// floor(r + W) and ceil(r - W) of the exact reals unless r +- W lies within
// about ulp(W) of an integer (the rounding of k - r in the predicate), so with
// W = Wi + Wf they come from FP32 sums rf +- Wf (error below 3e-7) whenever
// those lie more than 1e-5 from an integer; otherwise (and for W >= 2^30)
// from line_geometry's exact FP64 walk.  Also returns the nearest bin c and
// the offset rn in [-1/2, 1/2] (see nearest_bin) as a float.
// margin: distance from a tie (in bins) below which the FP32 sums cannot
// decide; walk: take the exact FP64 walk then (else return -1, undecided).
// Returns 1 if some bin of the grid is inside, 0 if none.
__device__ __forceinline__ int line_geometry_f32_m(double nu0, const GridD &g, const CutW &cw,
                                                   float margin, bool walk, int *c_out,
                                                   float *rn_out, int *lo_out, int *hi_out)
{
    const double u = __dmul_rn(__dsub_rn(nu0, g.nu_min), g.inv_dnu);
    const double f = floor(u);
    const double r = __dsub_rn(u, f);
    const float rf = (float)r;
    long long lo, hi;
    const long long i0 = (long long)f;
    bool exact = true;
    if (cw.nocut) {
        lo = 0;
        hi = g.nbins - 1;
        exact = false;
    } else if (cw.Wi >= 0) {
        const float sh = rf + cw.Wf, sl = rf - cw.Wf;
        const float th = sh - rintf(sh), tl = sl - rintf(sl);
        if (fabsf(th) > margin && fabsf(tl) > margin) {
            hi = i0 + cw.Wi + (long long)floorf(sh);
            lo = i0 - cw.Wi + (long long)ceilf(sl);
            exact = false;
        }
    }
    if (exact && !walk) return -1;
    if (exact) {
        int i0e, loe, hie;
        double re;
        const bool any = line_geometry_w(nu0, g, cw.nocut, cw.W, &i0e, &re, &loe, &hie);
        lo = any ? loe : 1;
        hi = any ? hie : 0;
    } else {
        if (lo < 0) lo = 0;
        if (hi > g.nbins - 1) hi = g.nbins - 1;
        if (!(nu0 > 0.0) || i0 < -2147483647LL || i0 > 2147483647LL) hi = lo - 1;
    }
    if (hi < lo) {
        *c_out = 0;
        *rn_out = 0.0f;
        *lo_out = 0x3fffffff;
        *hi_out = -0x3fffffff;
        return 0;
    }
    const bool up = rf >= 0.5f;   // either choice is a valid nearest-bin split
    *c_out = (int)i0 + (up ? 1 : 0);
    *rn_out = (float)(up ? r - 1.0 : r);
    *lo_out = (int)lo;
    *hi_out = (int)hi;
    return 1;
}

__device__ __forceinline__ bool line_geometry_f32(double nu0, const GridD &g, const CutW &cw,
                                                  int *c_out, float *rn_out, int *lo_out,
                                                  int *hi_out)
{
    return line_geometry_f32_m(nu0, g, cw, 1e-5f, true, c_out, rn_out, lo_out, hi_out) == 1;
}

// The Lorentz-multiple cut from the float Lorentz width (as the FP32 strength
// forms it): within ~4e-6 relative of the FP64 width of line_cut.
__device__ __forceinline__ CutW lorentz_cut_f32(const Prob &p, const GridD &g, int64_t l)
{
    const float nat = p.A ? p.A[l] * p.nat_coef_f : 0.0f;
    const float trn = exp2f(p.n_T[l] * p.log2_tratio_f);
    const float GL = p.gamma_self
                         ? nat + trn * fmaf(p.gamma[l], p.press_air_f, p.gamma_self[l] * p.press_self_f)
                         : nat + p.gamma[l] * trn * p.press_f;
    const float W = (float)g.cut_factor * GL * (float)g.inv_dnu;
    CutW c;
    c.nocut = false;
    c.W = (double)W;
    if (W >= 0.0f && W < 8388608.0f) {
        c.Wi = (int)floorf(W);
        c.Wf = W - (float)c.Wi;
    } else {
        c.Wi = -1;
        c.Wf = 0.0f;
    }
    return c;
}

// FP32-kernel geometry with the line's own cut.  Lorentz-multiple cuts try
// the float width first, with a tie margin covering its distance to the FP64
// width (the FP64 pow is slow on this GPU), and take the FP64 width only for
// a line the float width cannot decide; every other mode is exact at once.
// cw_out: the width used (its W serves the plinth).
__device__ __forceinline__ bool line_geometry_cut(const Prob &p, const GridD &g, int64_t l,
                                                  CutW *cw_out, int *c_out, float *rn_out,
                                                  int *lo_out, int *hi_out)
{
    const double pos = line_pos(p, l);
    // (with P_self > P the HITRAN width is a difference: no float shortcut)
    if (g.cut_mode == kCutLorentz && !(p.gamma_self && p.press_air < 0.0)) {
        const CutW a = lorentz_cut_f32(p, g, l);
        const float margin = 1e-5f + 4e-6f * (float)a.W;
        const int res = line_geometry_f32_m(pos, g, a, margin, false, c_out, rn_out, lo_out, hi_out);
        if (res >= 0) {
            *cw_out = a;
            return res == 1;
        }
    }
    const CutW cw = line_cut(p, g, l, p.nu0[l]);
    *cw_out = cw;
    return line_geometry_f32(pos, g, cw, c_out, rn_out, lo_out, hi_out);
}

// Offset of bin i from the line centre in bins, as (i - c) - rn with the
// NEAREST bin c and rn in [-1/2, 1/2]: for |i - c| >= 1 the float subtraction
// is well conditioned and for i = c the offset is -rn itself, so a bin that
// lies a tiny fraction of a bin from the centre keeps full relative
// precision.  (i0, r) are the floor-based values of line_geometry.
__device__ __forceinline__ void nearest_bin(int i0, double r, int *c, double *rn)
{
    if (r >= 0.5) {
        *c = i0 + 1;
        *rn = r - 1.0;
    } else {
        *c = i0;
        *rn = r;
    }
}

// Strength of line l in FP32 as a mantissa part P and a power of two: S *
// alphaD_inv / sqrt(pi) * mass_scale = P * 2^e2.  Also returns alphaD_inv and y.
__device__ __forceinline__ void line_strength_f32(const Prob &p, int64_t l, float *P_out,
                                                  int *e2_out, float *aDinv_out, float *y_out)
{
    const float nu0f = (float)p.nu0[l];
    float aDinv = p.aD_coef_f / nu0f;
    float nat = p.A ? p.A[l] * p.nat_coef_f : 0.0f;
    const float trn = exp2f(p.n_T[l] * p.log2_tratio_f);
    float GL = p.gamma_self
                   ? nat + trn * fmaf(p.gamma[l], p.press_air_f, p.gamma_self[l] * p.press_self_f)
                   : nat + p.gamma[l] * trn * p.press_f;
    // log2 of the Boltzmann factor, E'' K2, as a float pair Lh + Ll: E'' is a
    // float, so E'' K2_hi has the exact error term fma(E'', K2_hi, -Lh)
    const float E = p.E_low[l];
    const float Lh = E * p.K2_hi;
    const float Ll = fmaf(E, p.K2_lo, fmaf(E, p.K2_hi, -Lh));
    const float nL = rintf(Lh);
    float bz = exp2f((Lh - nL) + Ll);   // Lh - nL is exact
    float P;
    if (p.s_mode == 0) {
        float stim = expm1f(-p.c2T_f * nu0f) / expm1f(-p.c2Tref_f * nu0f);
        P = p.S_ref[l] * p.qratio_f * bz * stim;
    } else {
        float stim = -expm1f(-p.c2T_f * nu0f);
        P = p.A[l] * p.g_up[l] * p.qratio_f / (nu0f * nu0f) * bz * stim;
    }
    P = P * (aDinv * (float)kInvSqrtPi) * p.mass_scale_f;
    *P_out = P;
    *e2_out = (int)nL;
    *aDinv_out = aDinv;
    *y_out = GL * aDinv;
}

// FP64 strength S (no alphaD factor), alphaD_inv and y in double.
__device__ __forceinline__ void line_strength_f64(const Prob &p, int64_t l, double *S_out,
                                                  double *aDinv_out, double *y_out)
{
    double nu0 = p.nu0[l];
    double aDinv = p.aD_coef / nu0;
    double nat = p.A ? (double)p.A[l] * p.nat_coef : 0.0;
    const double trn = exp2((double)p.n_T[l] * p.log2_tratio);
    double GL = p.gamma_self ? nat + trn * ((double)p.gamma[l] * p.press_air +
                                            (double)p.gamma_self[l] * p.press_self)
                             : nat + (double)p.gamma[l] * trn * p.press;
    double bz = exp2((double)p.E_low[l] * p.K2);
    double S;
    if (p.s_mode == 0) {
        double stim = expm1(-p.c2T * nu0) / expm1(-p.c2Tref * nu0);
        S = (double)p.S_ref[l] * p.qratio * bz * stim;
    } else {
        double stim = -expm1(-p.c2T * nu0);
        S = (double)p.A[l] * (double)p.g_up[l] * p.qratio / (nu0 * nu0) * bz * stim;
    }
    *S_out = S * p.mass_scale;
    *aDinv_out = aDinv;
    *y_out = GL * aDinv;
}

// The work item of a persistent gather: called by a whole warp.  Lane 0 takes
// the next item number from `counter`; the warp finds its (problem, tile)
// entry -- the largest a with item_off[a] <= item in the non-decreasing
// exclusive scan item_off[0..m] -- by a 32-way search (32 probes and a ballot
// per step, so ~log32(m) dependent loads instead of log2(m)).  Returns the
// item number (-1 once all are taken) and sets *pt, *lb, *le for it.
__device__ __forceinline__ long long fetch_item(unsigned long long *counter,
                                                const int64_t *__restrict__ item_off, int64_t m,
                                                const int64_t *__restrict__ tile_lb,
                                                const int64_t *__restrict__ tile_le, int lmax,
                                                int lane, long long *pt, long long *lb,
                                                long long *le)
{
    long long item = 0;
    if (lane == 0) item = (long long)atomicAdd(counter, 1ull);
    item = __shfl_sync(0xffffffffu, item, 0);
    const long long total = item_off[m];
    if (item >= total) return -1;
    long long a = 0, b = m;   // item_off[a] <= item < item_off[b]
    while (b - a > 1) {
        const long long step = (b - a + 31) >> 5;
        const long long idx = a + (long long)lane * step;
        const bool le_ = idx < b && item_off[idx] <= item;
        const unsigned msk = __ballot_sync(0xffffffffu, le_);   // a prefix of the lanes
        const int k = 31 - __clz(msk);                           // lane 0 always holds
        a += (long long)k * step;
        b = min(b, a + step);
    }
    const long long l0 = tile_lb[a] + (item - item_off[a]) * lmax;
    *pt = a;
    *lb = l0;
    *le = min((long long)tile_le[a], l0 + lmax);
    return item;
}

// Two-sum: s + e = a + b exactly (Knuth).
__device__ __forceinline__ void two_sum(float a, float b, float *s, float *e)
{
    float t = a + b;
    float bp = t - a;
    float ap = t - bp;
    *e = (a - ap) + (b - bp);
    *s = t;
}

}  // namespace hk
