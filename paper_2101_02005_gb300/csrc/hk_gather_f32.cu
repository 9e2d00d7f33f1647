// hk_gather_f32.cu -- the FP32-compensated Voigt sum (HK_FP32C) on sm_103a.
//
// Line-major warps over a shared-memory tile of the grid:
//
// * Work items are (problem, tile of TILE bins, chunk of <= lmax lines), as
//   in the FP64 gather; a persistent grid pulls them from an atomic counter.
// * Inside an item every warp takes 32 lines at a time: lane i computes the
//   parameters of line i once (the centre-to-bin offset in FP64, the cut
//   bounds from FP32 sums away from ties, strength and widths in FP32, band
//   boundaries, the plinth) into a per-warp record table; then the warp
//   sweeps each line's bins inside the tile, 32 consecutive bins per step
//   (lane = bin).  Only a line's first and last groups can be partial: the
//   masked instance tests every group (short lines), the peeled one only
//   those two (wide lines), and takes a tile that lies wholly inside one
//   one-node segment of a line in a single unmasked pass.
// * The Faddeeva band of a 32-bin group is the band of its bin nearest the
//   line centre.  The bands form nested intervals of group indices around
//   the centre, computed once per line, so each group runs one formula with
//   no divergence.  Bins of the central groups that fall in the core band
//   (r2 < 64) are evaluated 32 at a time as (bin, line) slots: per line from
//   a per-warp queue, per batch of co-located short lines from the batch's
//   core and ring ranges (the trapezoid rule inside the ring radius, the
//   8-node Gauss-Hermite rule between it and r2 = 64).  The Lorentzian
//   profile is the one-node band on every group; the Doppler and
//   binned-Gaussian profiles run one formula per line in their own instances.
// * Short lines go in batches of NLS co-located lines that share one sweep per
//   group.  When all 32 lines of a round share their centre bin and groups,
//   their two- or four-node values over the interior groups are one series in
//   1/x about line 0 (coefficients taken lane-parallel and summed by
//   shuffles): one reciprocal and a Horner sum per bin for the whole round.
//   Wide Voigt lines take the same kind of series over the far groups of a
//   tile where every line of the round is inside its cut and its two-node
//   band, and batches of NLB lines on the rest.
// * Each warp adds into its own FP32 copy of the tile in shared memory
//   (consecutive bins, no bank conflicts, no atomics); every FLUSH_ROUNDS
//   rounds the copies are summed into a (hi, lo) two-sum pair per bin, and at
//   the end of the item hi + lo goes to the FP64 accumulator of the problem
//   with one atomicAdd per bin.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <map>
#include <mutex>

#include "hk_internal.cuh"
#include "hk_launch.h"

namespace hk {

namespace f32g {

constexpr int NW = 8;             // warps per block
constexpr int NT = NW * 32;
constexpr int TILE_MAX = 2048;    // widest tile (bins); the tile width is a launch parameter
constexpr int QCAP = 64;          // core-queue entries per warp
constexpr int FLUSH_ROUNDS = 4;   // rounds (32 lines per warp each) between two-sum folds

// Per-line record, computed once per (line, item) by one lane.  Groups are
// aligned to absolute bin indices: group g holds bins [32 g, 32 g + 31], so a
// tile (a multiple of 32 bins) is a contiguous range of groups and a line's
// band segments are tile-independent group ranges.  Bands: gh1 (r2 >= 1.5e6),
// gh2 (r2 >= 2500), gh4 (r2 >= 64), core (r2 < 64); a group takes the band
// of its bin nearest the line centre.
// The fields are grouped in 16-byte quads in the order a batch of lines reads
// them (one 128-bit shared load per quad): two-node parameters, four-node
// parameters, structure, ranges.
struct __align__(16) Rec {
    float b, rnb, Y, sy;        // x step per bin, rn b, y^2, s y / sqrt(pi)
    float Ca, Cb, sa, sb;       // 2 tau Y + tau^2 for both 4-node pairs, 2 W sy      (4 nodes)
    int c, gA, gB, lo;          // nearest bin to the centre; the line's groups; first bin in the cut
    int hi, L4, R4, cl;         // last bin; groups of band gh4 or inner; first core bin
    int ch, Lc, Rc, L2;         // last core bin (core: r2 < R8(y)); bins with r2 < 64;
    int R2;                     //   groups of band gh2 or inner
    float rn, s, y;             // centre offset from bin c, scaled strength, Gamma_L / alpha_D
    float h, k2a, k2b, pad;     // the plinth s Re w(x_cut + iy) (or 0); Y - 1/2, 2 Y (2 nodes;
                                //   binned Gaussian: sqrt(pi)/(2b) s, b/2)
};
static_assert(sizeof(Rec) == 112, "Rec is seven 16-byte quads");

// Shared memory: this fixed part, then the tile-sized arrays
// float acc[NW][tile] (each warp's FP32 copy of the tile), hi[tile], lo[tile].
struct Smem {
    Rec rec[NW][32];
    unsigned queue[NW][QCAP];
    float cval[NW][32];         // core values of one evaluation, by lane
};
static_assert(sizeof(Smem) % 16 == 0, "the tile arrays follow 16-byte aligned");

// Bands of the non-Voigt profiles (the Lorentzian is the one-node band itself)
constexpr int kBandGauss = 10, kBandBinned = 11;

constexpr float kTa = 0.27525512860841106f, kTb = 2.724744871391589f;   // 4-node tau
constexpr float kWa = 2.0f * 0.4541241452319315f, kWb = 2.0f * 0.04587585476806851f;

// Groups meeting the bins c + k, |k - rn| < D with D = sqrt(R - Y) / b (widened
// by a relative 1e-4 and 1e-3 bins so an edge group takes the more accurate
// band), nested in [Lp, Rp]; an empty band sits at Rp + 1.  ib = 1/b.
__device__ __forceinline__ void band_groups(float R, float Y, float ib, float rn, int c, int Lp,
                                            int Rp, int *L, int *R_)
{
    const float d2 = R - Y;
    if (!(d2 > 0.0f) || Lp > Rp) {
        *L = Rp + 1;
        *R_ = Rp;
        return;
    }
    // sqrt(d2) / b from the hardware reciprocal square root and reciprocal
    // (a few ulp; the widening covers them)
    const float D = fminf(d2 * rsqrtf(d2) * ib * 1.0001f + 1e-3f, 1.0e9f);
    const int kL = (int)floorf(rn - D) + 1, kR = (int)ceilf(rn + D) - 1;
    int lo = (c + kL) >> 5, hi = (c + kR) >> 5;   // arithmetic shifts: floor division
    lo = max(lo, Lp);
    hi = min(hi, Rp);
    if (kL > kR || lo > hi) {
        *L = Rp + 1;
        *R_ = Rp;
    } else {
        *L = lo;
        *R_ = hi;
    }
}

// Inner radius (in r2) of the ring where the 8-node Gauss-Hermite rule
// serves the short-line batches in place of the trapezoid: 26, or more where
// y is so small that exp(-x^2), which a Gauss-Hermite sum cannot represent,
// would exceed ~1e-7 of Re w ~ y / (sqrt(pi) x^2) (x^2 < 64 in the bound).
// Checked against scipy's wofz in exact arithmetic: at most 1.3e-7 relative
// error over 26 <= r2 < 64, y from 1e-9 to 8.
__device__ __forceinline__ float ring_r2(float y)
{
    return fminf(64.0f, fmaxf(26.0f, 20.845483f - __logf(y)));   // ln(1.13e9) - ln y
}

// 8-node Gauss-Hermite value sy F8 of one pair (r2 = x^2 + y^2 at least the
// line's ring radius): the four node pairs +-t_j (tau_j = t_j^2, normalised
// weights 2 W_j) give F8 = sum_j 2 W_j (r2 + tau_j) / D_j,
// D_j = r2^2 - 2 tau_j X + 2 tau_j Y + tau_j^2, summed over one common
// denominator: one reciprocal.  D_j >= (r2 - tau_j)^2 >= 300, and for
// r2 <= 4096 D_j <= 1.7e7, so the products stay inside the float range.  A
// line of the batch far outside its own ring there (a huge y, or a much
// narrower line) has r2 > 4096 and takes the two-node rule, valid and within
// ~1.5e-7 for r2 >= 2500 (the sweeps' own rule there).
__device__ __forceinline__ float gh8_val(float x, float Y, float sy)
{
    constexpr float t1 = 0.14530352150331709f, t2 = 1.3390972881263614f,
                    t3 = 3.9269635013582872f, t4 = 8.5886356890120343f;
    constexpr float w1 = 0.74602451535815470f, w2 = 0.23447981532351803f,
                    w3 = 0.019270440241576534f, w4 = 0.00022522907675073554f;
    const float X = x * x, r2 = X + Y;
    if (r2 > 4096.0f) {
        const float Xp = fmaf(x, x, Y - 0.5f);   // X' = x^2 + Y - 1/2
        return fmaf(Xp, sy, sy) * rcp_ftz(fmaf(Xp, Xp, 2.0f * Y));
    }
    const float D1 = fmaf(r2, r2, fmaf(-2.0f * t1, X, fmaf(2.0f * t1, Y, t1 * t1)));
    const float D2 = fmaf(r2, r2, fmaf(-2.0f * t2, X, fmaf(2.0f * t2, Y, t2 * t2)));
    const float D3 = fmaf(r2, r2, fmaf(-2.0f * t3, X, fmaf(2.0f * t3, Y, t3 * t3)));
    const float D4 = fmaf(r2, r2, fmaf(-2.0f * t4, X, fmaf(2.0f * t4, Y, t4 * t4)));
    const float n1 = fmaf(w1, r2, w1 * t1), n2 = fmaf(w2, r2, w2 * t2);
    const float n3 = fmaf(w3, r2, w3 * t3), n4 = fmaf(w4, r2, w4 * t4);
    const float D12 = D1 * D2, D34 = D3 * D4;
    const float num = fmaf(fmaf(n1, D2, n2 * D1), D34, fmaf(n3, D4, n4 * D3) * D12);
    return sy * num * rcp_ftz(D12 * D34);
}

__device__ __forceinline__ void make_rec(const Prob &pr, const GridD &g, int64_t l, int scale,
                                         Rec *out)
{
    Rec q;
    int c, lo, hi;
    float rn;
    CutW cw;
    bool any;
    if (pr.geo) {   // computed once for all problems of the line list (fixed cut or none)
        const int4 G = pr.geo[l];
        c = G.x;
        rn = __int_as_float(G.y);
        lo = G.z;
        hi = G.w;
        any = lo <= hi;
        cw.nocut = !(g.W > 0.0);
        cw.W = g.W;
        cw.Wi = g.Wi;
        cw.Wf = g.Wf;
    } else {
        any = line_geometry_cut(pr, g, l, &cw, &c, &rn, &lo, &hi);
    }
    q.c = c;
    q.lo = lo;
    q.hi = hi;
    q.rn = rn;
    float aDinv, y, sv;
    if (!any) {
        aDinv = 1.0f;
        y = 1.0f;
        sv = 0.0f;
    } else if (pr.pre) {
        aDinv = pr.aDinv_pre[l];
        y = pr.y_pre[l];
        sv = (float)ldexp(pr.S_pre[l] * (double)aDinv * kInvSqrtPi, -scale);
    } else {
        float P;
        int e2;
        line_strength_f32(pr, l, &P, &e2, &aDinv, &y);
        sv = ldexpf(P, e2 - scale);
    }
    const float b = (float)g.dnu * aDinv, Y = y * y, sy = sv * y * (float)kInvSqrtPi;
    q.b = b;
    q.Y = Y;
    q.s = sv;
    q.y = y;
    q.rnb = q.rn * b;
    q.sy = sy;
    q.k2a = Y - 0.5f;
    q.k2b = 2.0f * Y;
    q.Ca = fmaf(2.0f * kTa, Y, kTa * kTa);
    q.Cb = fmaf(2.0f * kTb, Y, kTb * kTb);
    q.sa = sy * kWa;
    q.sb = sy * kWb;
    // the plinth: this line's value at its cutting length, x_cut = W b
    q.h = (g.plinth && any && !cw.nocut)
              ? sv * profile_rel<float>(g.profile, (float)cw.W * b, y, b)
              : 0.0f;
    if (g.profile == kProfBinned) {          // sqrt(pi)/(2b) s and b/2 in the 2-node slots
        q.k2a = sv * (float)(0.5 / kInvSqrtPi) / b;
        q.k2b = 0.5f * b;
    }
    if (any) {
        q.gA = lo >> 5;
        q.gB = hi >> 5;
    } else {
        q.gA = 1;
        q.gB = 0;
    }
    const float ib = rcp_ftz(b);
    band_groups(1.5e6f, Y, ib, q.rn, c, q.gA, q.gB, &q.L2, &q.R2);
    band_groups(2500.0f, Y, ib, q.rn, c, q.L2, q.R2, &q.L4, &q.R4);
    // bins c + k with |k - rn| < sqrt(R - Y) / b, inside [lo, hi] (inside the
    // four-node groups: those take a wider margin); empty: first > last.
    // R = 64: the trapezoid's band [Lc, Rc]; R = R8 (y): the inner core
    // [cl, ch], the ring between them being the 8-node rule's (short lines).
    q.cl = q.Lc = 1;
    q.ch = q.Rc = 0;
    if (any && Y < 64.0f) {
        auto bins = [&](float R, int *first, int *last) {
            // (the band edge to a few ulp: the rules on either side of it are
            // both valid there)
            const float d2 = R - Y;
            const float Dc = fminf(d2 * rsqrtf(d2) * ib, 1.0e9f);
            const int kl = (int)floorf(q.rn - Dc) + 1, kh = (int)ceilf(q.rn + Dc) - 1;
            const int a = max(c + kl, lo), e = min(c + kh, hi);
            if (a <= e) {
                *first = a;
                *last = e;
            }
        };
        bins(64.0f, &q.Lc, &q.Rc);
        const float R8 = ring_r2(y);
        if (Y < R8) bins(R8, &q.cl, &q.ch);
    }
    q.pad = 0.0f;
    if (g.profile == kProfLorentz) {          // (y/sqrt(pi)) s / r2 on every bin: all one-node
        q.L2 = q.L4 = q.Lc = q.gB + 1;
        q.R2 = q.R4 = q.Rc = q.gB;
        q.cl = 1;
        q.ch = 0;
    }
    *out = q;
}

// Value of one pair in band BAND at offset kf (float bin offset from c).
template <int BAND> __device__ __forceinline__ float pair_raw(const Rec &q, float kf)
{
    const float x = fmaf(kf, q.b, -q.rnb);
    const float X = x * x;
    const float r2 = X + q.Y;
    // one hardware reciprocal and a multiply, within 2 ulp while the divisor
    // is below 2^126 (gh1 beyond that gives 0, far below any sum)
    if (BAND == kBandGauss) {
        return q.s * exp2f(-X * 1.4426950408889634f);
    } else if (BAND == kBandBinned) {
        const float ax = fabsf(x), a = ax - q.k2b, c = ax + q.k2b;
        return q.k2a * (a >= 0.0f ? erfcf(a) - erfcf(c) : erff(c) + erff(-a));
    } else if (BAND == kBandGH1) {
        return q.sy * rcp_ftz(r2);
    } else if (BAND == kBandGH2) {          // |z^2 - 1/2|^2 = r2^2 - X + Y + 1/4
        const float Xp = fmaf(x, x, q.k2a);      // X' = x^2 + Y - 1/2
        return fmaf(Xp, q.sy, q.sy) * rcp_ftz(fmaf(Xp, Xp, q.k2b));
    } else {                                // 4 nodes: |z^2 - tau|^2 = r2^2 - 2 tau (X - Y) + tau^2
        const float da = fmaf(r2, r2, fmaf(-2.0f * kTa, X, q.Ca));
        const float db = fmaf(r2, r2, fmaf(-2.0f * kTb, X, q.Cb));
        return fmaf(q.sa * (r2 + kTa), db, q.sb * (r2 + kTb) * da) * rcp_ftz(da * db);
    }
}

// Launch variants V: bit 1 peels the edge groups (wide lines), bit 2 removes
// the plinth (every in-range pair less the line's value at its cut), bits 4
// and 8 select the Doppler and binned-Gaussian profiles (one formula for all
// bins of a line; Voigt and Lorentzian run the banded sweeps).
constexpr int kVPeel = 1, kVPlinth = 2, kVDoppler = 4, kVBinned = 8;

template <int BAND, int V> __device__ __forceinline__ float pair_f(const Rec &q, float kf)
{
    const float v = pair_raw<BAND>(q, kf);
    return (V & kVPlinth) ? v - q.h : v;
}

// One masked group: lanes add only where bin 32 g + lane lies in the line's
// range [lo, hi].
template <int BAND, int V>
__device__ __forceinline__ void edge_group(const Rec &q, int g, int tg0, float *base, int kfc,
                                           int lane)
{
    if ((unsigned)(32 * g + lane - q.lo) <= (unsigned)(q.hi - q.lo))
        base[32 * (g - tg0)] += pair_f<BAND, V>(q, (float)(32 * g + kfc));
}

// One band over groups [g0, g1] (inclusive), clipped to [lo_g, hi_g].  `base`
// is the warp's tile copy at group tg0 plus this lane; kfc = lane - c.  Only
// the line's first and last groups (gA, gB) can be partial.  Without kVPeel
// a lane adds only if its bin lies in the line's range (one compare per
// group, best for lines a few groups wide); with kVPeel gA and gB are peeled
// off and masked, the groups between them run unmasked (best for wide lines,
// where the per-band test costs less than the per-group one).
template <int BAND, int V>
__device__ __forceinline__ void sweep(const Rec &q, int g0, int g1, int lo_g, int hi_g, int tg0,
                                      float *base, int kfc, int lane)
{
    g0 = max(g0, lo_g);
    g1 = min(g1, hi_g);
    if (g0 > g1) return;
    float kf;
    float *p, *pe;
    if (V & kVPeel) {
        if (g0 == q.gA) {
            edge_group<BAND, V>(q, g0, tg0, base, kfc, lane);
            if (++g0 > g1) return;
        }
        if (g1 == q.gB) {
            edge_group<BAND, V>(q, g1, tg0, base, kfc, lane);
            if (--g1 < g0) return;
        }
        kf = (float)(32 * g0 + kfc);
        p = base + 32 * (g0 - tg0);
        pe = base + 32 * (g1 - tg0);
        for (; p < pe; p += 64, kf += 64.0f) {   // two groups per step
            const float v0 = pair_f<BAND, V>(q, kf);
            const float v1 = pair_f<BAND, V>(q, kf + 32.0f);
            p[0] += v0;
            p[32] += v1;
        }
        if (p == pe) p[0] += pair_f<BAND, V>(q, kf);
    } else {
        const unsigned span = (unsigned)(q.hi - q.lo);
        unsigned rel = (unsigned)(32 * g0 + lane - q.lo);   // bin - lo
        kf = (float)(32 * g0 + kfc);
        p = base + 32 * (g0 - tg0);
        pe = base + 32 * (g1 - tg0);
        for (; p < pe; p += 64, kf += 64.0f, rel += 64u) {   // two groups per step
            const float v0 = pair_f<BAND, V>(q, kf);
            const float v1 = pair_f<BAND, V>(q, kf + 32.0f);
            if (rel <= span) p[0] += v0;
            if (rel + 32u <= span) p[32] += v1;
        }
        if (p == pe && rel <= span) p[0] += pair_f<BAND, V>(q, kf);
    }
}

// The binned Gaussian over groups [g0, g1] with shared bin edges: bin k's
// value is sbin (F(e_k+1) - F(e_k)), e_k = x_k - b/2 its lower edge, F = erf,
// taken through E(e) = erfc(|e|) (both edges >= 0: E_lo - E_hi; both <= 0:
// E_hi - E_lo; straddling the centre: 2 - E_lo - E_hi).  Each lane evaluates
// E at its bin's lower edge only; the upper edge is the next lane's lower edge
// (lane 31: the next group's lane 0), so a group is finished one step later
// and one extra edge closes the pass.  Edge groups gA, gB go through the
// masked per-bin form.
template <int V>
__device__ __forceinline__ void sweep_binned(const Rec &q, int g0, int g1, int lo_g, int hi_g,
                                             int tg0, float *base, int kfc, int lane)
{
    g0 = max(g0, lo_g);
    g1 = min(g1, hi_g);
    if (g0 > g1) return;
    if (g0 == q.gA) {
        edge_group<kBandBinned, V>(q, g0, tg0, base, kfc, lane);
        if (++g0 > g1) return;
    }
    if (g1 == q.gB) {
        edge_group<kBandBinned, V>(q, g1, tg0, base, kfc, lane);
        if (--g1 < g0) return;
    }
    // lower edge of this lane's bin in group g: x - b/2
    auto lower = [&](int g) { return fmaf((float)(32 * g + kfc), q.b, -q.rnb) - q.k2b; };
    float e = lower(g0);
    float E = erfcf(fabsf(e));
    for (int g = g0; g <= g1; ++g) {
        const float en = lower(g + 1);                 // the next group's lower edges
        const float En = erfcf(fabsf(en));
        float eh = __shfl_down_sync(0xffffffffu, e, 1);
        float Eh = __shfl_down_sync(0xffffffffu, E, 1);
        const float e0 = __shfl_sync(0xffffffffu, en, 0), E0 = __shfl_sync(0xffffffffu, En, 0);
        if (lane == 31) {
            eh = e0;
            Eh = E0;
        }
        const float d = (e >= 0.0f) ? E - Eh : (eh <= 0.0f ? Eh - E : 2.0f - E - Eh);
        float v = q.k2a * d;
        if (V & kVPlinth) v -= q.h;
        base[32 * (g - tg0)] += v;
        e = en;
        E = En;
    }
}

// Evaluates up to 32 queued core pairs, one per lane (lanes >= n idle), and
// adds them into the warp's tile copy.  Entries may share a bin (the lines of
// a batch share their centre): lanes of one bin, found by a match, add up
// through the warp's scratch row and one of them updates the bin, so the
// update needs no atomics.  Called by the whole warp.
__device__ __forceinline__ void core_entry(Smem &S, int warp, int t0, unsigned e, int lane, int n,
                                           float *accw)
{
    const bool valid = lane < n;
    float v = 0.0f;
    int tidx = -1 - lane;                        // distinct keys for idle lanes
    if (valid) {
        const Rec &qq = S.rec[warp][e >> 16];
        tidx = (int)(e & 0xffffu);
        const float kk = (float)(t0 + tidx - qq.c);
        const float xx = fmaf(kk, qq.b, -qq.rnb);
        v = qq.s * core_re<float>(xx, qq.y) - qq.h;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, tidx);
    S.cval[warp][lane] = v;
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) {
        float sum = v;
        for (unsigned m = peers & (peers - 1u); m; m &= m - 1u) sum += S.cval[warp][__ffs(m) - 1];
        accw[tidx] += sum;
    }
    __syncwarp();
}

// Groups holding core bins: lanes with r2 >= 64 take the 4-node rule (valid
// for every r2 >= 64) in place; core lanes (r2 < 64) are queued as (record
// slot, tile index) and the queue is evaluated 32 entries at a time with the
// trapezoid rule.
template <int V>
__device__ __forceinline__ void sweep_core(const Rec &q, int slot, int g0, int g1, int lo_g,
                                           int hi_g, int tg0, float *base, int kfc, int lane,
                                           unsigned *queue, int &qn, Smem &S, int warp, int t0)
{
    g0 = max(g0, lo_g);
    g1 = min(g1, hi_g);
    const unsigned span = (unsigned)(q.hi - q.lo);
    for (int g = g0; g <= g1; ++g) {
        const bool act = (unsigned)(32 * g + lane - q.lo) <= span;
        const float kf = (float)(32 * g + kfc);
        const float x = fmaf(kf, q.b, -q.rnb);
        const float r2 = fmaf(x, x, q.Y);
        const bool core = act && r2 < 64.0f;
        if (act && !core) base[32 * (g - tg0)] += pair_f<kBandGH4, V>(q, kf);
        const unsigned m = __ballot_sync(0xffffffffu, core);
        if (m) {
            const int pos = qn + __popc(m & ((1u << lane) - 1u));
            if (core) queue[pos] = ((unsigned)slot << 16) | (unsigned)(32 * g + lane - t0);
            qn += __popc(m);
            __syncwarp();
            if (qn >= 32) {
                core_entry(S, warp, t0, queue[lane], lane, 32, base - lane);
                __syncwarp();
                if (lane < qn - 32) queue[lane] = queue[lane + 32];
                qn -= 32;
                __syncwarp();
            }
        }
    }
}

__device__ __forceinline__ void drain_rest(unsigned *queue, int &qn, Smem &S, int warp, int lane,
                                           int t0, float *accw)
{
    if (qn > 0) {
        core_entry(S, warp, t0, queue[lane], lane, qn, accw);
        qn = 0;
    }
    __syncwarp();
}

// One line's bins in groups [r0, r1] of the tile (groups [tg0, tg1]; base is
// the warp's copy of the tile at its first group).
template <int V>
__device__ __forceinline__ void do_line(const Rec &q, int slot, int tg0, int tg1, float *base,
                                        int lane, unsigned *queue, int &qn, Smem &S, int warp,
                                        int t0, int r0, int r1)
{
    const int ga = max(q.gA, r0), gb = min(q.gB, r1);
    if (ga > gb) return;  // warp-uniform
    const int kfc = lane - q.c;
    if (V & kVDoppler) {
        sweep<kBandGauss, V>(q, q.gA, q.gB, ga, gb, tg0, base, kfc, lane);
        return;
    }
    if (V & kVBinned) {
        sweep_binned<V>(q, q.gA, q.gB, ga, gb, tg0, base, kfc, lane);
        return;
    }
    // a range inside one one-node segment of a wide line, clear of its edge
    // groups: one unmasked pass and none of the other bands' prologues
    if ((V & kVPeel) && r1 < q.gB && ((r0 > q.gA && r1 < q.L2) || r0 > q.R2)) {
        float kf = (float)(32 * r0 + kfc);
        float *p = base + 32 * (r0 - tg0);
        float *const pe = base + 32 * (r1 - tg0);
        for (; p < pe; p += 64, kf += 64.0f) {
            const float v0 = pair_f<kBandGH1, V>(q, kf);
            const float v1 = pair_f<kBandGH1, V>(q, kf + 32.0f);
            p[0] += v0;
            p[32] += v1;
        }
        if (p == pe) p[0] += pair_f<kBandGH1, V>(q, kf);
        return;
    }
    // short lines (no kVPeel): the one-node region takes the two-node rule, one
    // pass fewer on each side for a few more flops per far-wing pair
    if (V & kVPeel) {
        sweep<kBandGH1, V>(q, q.gA, q.L2 - 1, ga, gb, tg0, base, kfc, lane);
        sweep<kBandGH2, V>(q, q.L2, q.L4 - 1, ga, gb, tg0, base, kfc, lane);
    } else {
        sweep<kBandGH2, V>(q, q.gA, q.L4 - 1, ga, gb, tg0, base, kfc, lane);
    }
    if (q.L4 <= q.R4)   // the four-node groups and the core groups in one pass
        sweep_core<V>(q, slot, q.L4, q.R4, ga, gb, tg0, base, kfc, lane, queue, qn, S, warp, t0);
    if (V & kVPeel) {
        sweep<kBandGH2, V>(q, q.R4 + 1, q.R2, ga, gb, tg0, base, kfc, lane);
        sweep<kBandGH1, V>(q, q.R2 + 1, q.gB, ga, gb, tg0, base, kfc, lane);
    } else {
        sweep<kBandGH2, V>(q, q.R4 + 1, q.gB, ga, gb, tg0, base, kfc, lane);
    }
}

// ---- batches of co-located lines (short lines, Voigt, no plinth) --------------
//
// In a dense sorted list, consecutive lines share their nearest bin and so
// their group structure: the same first and last groups (gA, gB)
// and band boundaries inside the same few central groups.  For NLB such lines
// the warp takes each group once and sums the lines' values in a register,
// updating the tile copy once per group instead of once per line.  The
// groups strictly between gA and the batch's first four-node group (and
// between its last one and gB) run the two-node rule with no mask and no
// band test; gA and gB run it with each line's lane mask; the central groups
// [min L4, max R4] run the four-node rule per line, core bins (r2 < 64)
// going to the core queue.  x is formed exactly as on the per-line path (the
// two-node rule is the same rational function, regrouped in X = x^2).  A
// batch whose lines differ in gA, gB or the nearest bin c, or whose central
// groups reach gA or gB, takes the per-line path.
constexpr int NLB = 4;   // lines per batch: wide lines
constexpr int NLS = 4;   // lines per batch: short lines

// Two-node value of a pair, as fma(num, 1/d, acc).  The rule's
// |z^2 - 1/2|^2 = X^2 + (2Y - 1) X + (Y + 1/2)^2 (X = x^2) is, with
// X' = x^2 + Y - 1/2, X'^2 + 2Y, and its numerator sy (X + Y + 1/2) is
// sy (X' + 1): three FMAs and the reciprocal after x (Ym = Y - 1/2, Y2 = 2Y).
// In the band, x^2 + Y >= 2500, so neither sum cancels.
__device__ __forceinline__ float gh2_acc(float kf, float b, float nrb, float Ym, float Y2, float sy,
                                         float acc)
{
    const float x = fmaf(kf, b, nrb);
    const float Xp = fmaf(x, x, Ym);
    return fmaf(fmaf(Xp, sy, sy), rcp_ftz(fmaf(Xp, Xp, Y2)), acc);
}

// Four-node value of a pair (valid for every r2 >= 64); *r2 = x^2 + y^2.
__device__ __forceinline__ float gh4_val(float kf, float b, float nrb, float Y, float Ca,
                                         float Cb, float sa, float sb, float *r2_out)
{
    const float x = fmaf(kf, b, nrb);
    const float X = x * x;
    const float r2 = X + Y;
    const float da = fmaf(r2, r2, fmaf(-2.0f * kTa, X, Ca));
    const float db = fmaf(r2, r2, fmaf(-2.0f * kTb, X, Cb));
    *r2_out = r2;
    return fmaf(sa * (r2 + kTa), db, sb * (r2 + kTb) * da) * rcp_ftz(da * db);
}

// Two lines' two-node values with one reciprocal, n0/d0 + n1/d1 =
// (n0 d1 + n1 d0) / (d0 d1): the same issue count as two reciprocals and half
// the MUFU work.  The caller bounds r2 (d <= (r2 + 1)^2) so that the products
// stay in the float range.
__device__ __forceinline__ float gh2_pair_acc(float kf0, float b0, float nrb0, float Ym0, float Y20,
                                              float sy0, float kf1, float b1, float nrb1, float Ym1,
                                              float Y21, float sy1, float acc)
{
    const float x0 = fmaf(kf0, b0, nrb0), x1 = fmaf(kf1, b1, nrb1);
    const float X0 = fmaf(x0, x0, Ym0), X1 = fmaf(x1, x1, Ym1);
    const float d0 = fmaf(X0, X0, Y20), d1 = fmaf(X1, X1, Y21);
    const float n0 = fmaf(X0, sy0, sy0), n1 = fmaf(X1, sy1, sy1);
    return fmaf(fmaf(n0, d1, n1 * d0), rcp_ftz(d0 * d1), acc);
}

// Largest r2 = x^2 + y^2 of lines (b, Y) at integer offsets |k| <= kmax from
// their nearest bin (|rn| <= 1/2), as a bound for the shared reciprocals:
// below kShareR2 both the denominators' product and the numerators' products
// stay far inside the float range.
constexpr float kShareR2 = 2.5e8f;
constexpr int kMaskSpan = 4;      // widest masked spans of a wide batch (groups, both ends)
__device__ __forceinline__ float r2_bound(float kmax, float b, float Y)
{
    const float xm = (kmax + 0.5f) * b;
    return fmaf(xm, xm, Y);
}

// A wide line's batch flags for the tile [tg0, tg1], taken per line (one lane
// per line, in the record stage) instead of per batch: bits 0-1 the rule that
// serves the whole tile clear of the line's edge groups (1 one node, where the
// tile lies in the one-node band; 2 two nodes, where it lies in the one- and
// two-node bands and meets no four-node or core group; 0 neither); bit 2 set when every r2 of the tile stays below the
// shared-reciprocal bound of that band; bit 3 set when x may be formed from the
// tile's origin (one node, every |x| of the tile <= 4110: the origin's
// rounding, at most half an ulp of 4110, moves r2 = x^2 + y^2 >= 1.5e6 by at
// most 2 |x| 2.4e-4 / r2 <= 3e-7 relative); bit 4 set when the two-node rule
// may serve the line over the tile (r2 < 1e17), bit 5 when two-node values may
// share reciprocals over the tile, bit 6 when the line's four-node and core
// groups meet the tile.
__device__ __forceinline__ int wide_flags(const Rec &q, int tg0, int tg1, bool voigt)
{
    const float km = (float)max(abs(32 * tg0 - q.c), abs(32 * tg1 + 31 - q.c));
    const float r2m = r2_bound(km, q.b, q.Y);
    // the two-node rule may serve a Voigt line anywhere in the tile outside its
    // four-node and core groups while X'^2 ~ r2^2 stays in the float range (it
    // is the more accurate rule in the one-node band); the Lorentzian is the
    // one-node rule itself
    const bool gh2ok = voigt && r2m < 1e17f;
    const bool meets4 = q.L4 <= q.R4 && q.L4 <= tg1 && q.R4 >= tg0;
    int cls = 0;
    if (tg0 > q.gA && tg1 < q.gB) {
        if (tg1 < q.L2 || tg0 > q.R2) cls = 1;
        else if (!meets4 && gh2ok) cls = 2;
    }
    const bool share = cls != 0 && r2m < (cls == 1 ? 1e17f : kShareR2);
    const bool origin = cls == 1 && share && (km + 0.5f) * q.b < 1225.0f * 2e-7f * 16777216.0f;
    return cls | (share ? 4 : 0) | (origin ? 8 : 0) | (gh2ok ? 16 : 0) |
           (gh2ok && r2m < kShareR2 ? 32 : 0) | (meets4 ? 64 : 0);
}

// The i-th 16-byte quad of a record, as one 128-bit shared load.
__device__ __forceinline__ float4 quadf(const Rec &q, int i)
{
    return reinterpret_cast<const float4 *>(&q)[i];
}
__device__ __forceinline__ int4 quadi(const Rec &q, int i)
{
    return reinterpret_cast<const int4 *>(&q)[i];
}

// The structure of each batch of NLS consecutive lines (lanes NLS k ..
// NLS k + NLS - 1 of the record stage), taken lane-parallel by shuffles and
// kept in the batch's first two records, in fields the short-line path does
// not otherwise read.  First record: Lc, Rc = the smallest L4 and the largest
// R4 of the lines with a four-node band; L2, R2 = U, the union of the lines'
// inner core ranges [cl, ch] (empty: INT_MAX, INT_MIN); pad = flags, bit 0
// when the lines share c, gA and gB (gA <= gB), bit 1 when they share their
// cut range [lo, hi].  Second record: Lc, Rc = U8, the union of the lines'
// r2 < 64 ranges (U lies inside U8).
__device__ __forceinline__ void batch_summary(Rec &q, int lane)
{
    constexpr unsigned FULL = 0xffffffffu, kAll = (1u << NLS) - 1u;
    const int first = lane & ~(NLS - 1);
    // every lane takes every shuffle (no short-circuit evaluation around them)
    const int c0 = __shfl_sync(FULL, q.c, first), gA0 = __shfl_sync(FULL, q.gA, first),
              gB0 = __shfl_sync(FULL, q.gB, first), lo0 = __shfl_sync(FULL, q.lo, first),
              hi0 = __shfl_sync(FULL, q.hi, first);
    const bool same = (c0 == q.c) & (gA0 == q.gA) & (gB0 == q.gB) & (q.gA <= q.gB);
    const bool scut = (lo0 == q.lo) & (hi0 == q.hi);
    const unsigned ms = __ballot_sync(FULL, same), mc = __ballot_sync(FULL, scut);
    const bool has4 = q.L4 <= q.R4, hasc = q.cl <= q.ch, has8 = q.Lc <= q.Rc;
    int a = has4 ? q.L4 : INT_MAX, e = has4 ? q.R4 : INT_MIN;
    int u = hasc ? q.cl : INT_MAX, v = hasc ? q.ch : INT_MIN;
    int u8 = has8 ? q.Lc : INT_MAX, v8 = has8 ? q.Rc : INT_MIN;
#pragma unroll
    for (int o = 1; o < NLS; o <<= 1) {
        a = min(a, __shfl_xor_sync(FULL, a, o));
        e = max(e, __shfl_xor_sync(FULL, e, o));
        u = min(u, __shfl_xor_sync(FULL, u, o));
        v = max(v, __shfl_xor_sync(FULL, v, o));
        u8 = min(u8, __shfl_xor_sync(FULL, u8, o));
        v8 = max(v8, __shfl_xor_sync(FULL, v8, o));
    }
    if (lane == first + 1) {
        q.Lc = u8;
        q.Rc = v8;
    }
    if (lane == first) {
        q.Lc = a;
        q.Rc = e;
        q.L2 = u;
        q.R2 = v;
        q.pad = __int_as_float((((ms >> first) & kAll) == kAll ? 1 : 0) |
                               (((mc >> first) & kAll) == kAll ? 2 : 0));
    }
}

// ---- a round's lines as one series in 1/x ------------------------------------
//
// When the 32 lines of a warp's round share their nearest bin c and their
// groups gA, gB (dense sorted lists), their sum over the groups between the
// edge groups can be taken for all 32 lines at once.  A Gauss-Hermite value of
// a line is a sum of Lorentzians: (y/sqrt(pi)) sum_k W_k / ((x_j - t_k)^2 + y^2)
// over its nodes t_k.  With x = (k - rn_0) b_0 the offset of bin c + k from
// line 0 and x_j = beta_j x + d_j (beta_j = b_j / b_0, d_j = (rn_0 - rn_j) b_j),
// each Lorentzian is 1 / (beta_j^2 ((x - a)^2 + c^2)) = Im(1 / (x - z)) / (beta_j^2 c),
// z = a + i c, a = (t_k - d_j) / beta_j, c = y_j / beta_j, and
// 1 / (x - z) = sum_m z^m / x^(m+1) for |x| > |z|.  So the round's sum is
// sum_m B_m / x^(m+1), B_m = sum over lines and nodes of
// s_j W_k / (sqrt(pi) beta_j) Im(z^m): the coefficients are taken lane-parallel
// (lane j, line j) and summed over the warp, then every bin costs one
// reciprocal and a Horner sum for the whole round.  Two forms:
// * four nodes, 12 terms, over every bin of [gA + 1, gB - 1] outside U8 (the
//   union of the lines' r2 < 64 bins): where every line has y <= 1.2 and
//   |d_j| <= 0.2, |x| >= ~7.7 there and the terms after z^12 stay below
//   1e-8 of the sum (8e-9 against the direct four-node sums in FP64 over
//   seeded rounds); the batches keep only their edge groups, and their core
//   and ring passes take the round's unions U and U8.
// * two nodes (t = 1/sqrt 2, W = 1/2), 7 terms, over the two-node interiors
//   [gA + 1, min L4 - 1] and [max R4 + 1, gB - 1] of the round: where every
//   |z| <= 3 (|x| >= ~47 in the two-node band, terms after z^7 below 3.5e-8;
//   5e-9 against the direct two-node sums in FP64); with 12 terms where every
//   |z| <= 7 (terms after z^12 below 13 (7/47)^12 = 1e-9).
constexpr int KMP2 = 7, KMP4 = 12;   // series terms
constexpr int kNoBin = 0x3fffffff;   // a bin index no grid reaches
constexpr float kTnode = 0.70710678118654752f;
constexpr float kT4a = 0.52464762327529031f, kT4b = 1.6506801238857845f;   // sqrt(tau_a, tau_b)

// The series' parameters, written by lane 0 into the warp's queue rows (free
// until the batches run: a round with a series has no per-line fallback).
struct RoundSeries {
    float B[KMP4 + 1];   // B[1..K]
    float b0, nrb0, H;
    int c0, gA, gB;
    int RA, RB;          // two nodes: the series covers [gA + 1, RA - 1] and [RB + 1, gB - 1]
    int ulo, uhi, u8lo, u8hi;   // four nodes: the round's U and U8
};
static_assert(sizeof(RoundSeries) <= QCAP * sizeof(unsigned), "the series fits the queue rows");

// Decides whether the round takes a series and takes its coefficients.  q:
// this lane's record (line `lane` of the round), before the batch summary.
// Called by the whole warp.
template <int V>
__device__ __forceinline__ int round_series(const Rec &q, int lane, RoundSeries &rs)
{
    constexpr unsigned FULL = 0xffffffffu;
    const int c0 = __shfl_sync(FULL, q.c, 0), gA = __shfl_sync(FULL, q.gA, 0),
              gB = __shfl_sync(FULL, q.gB, 0);
    const float b0 = __shfl_sync(FULL, q.b, 0), rn0 = __shfl_sync(FULL, q.rn, 0);
    const bool has4 = q.L4 <= q.R4;
    int mL4 = has4 ? q.L4 : INT_MAX, MR4 = has4 ? q.R4 : INT_MIN;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mL4 = min(mL4, __shfl_xor_sync(FULL, mL4, o));
        MR4 = max(MR4, __shfl_xor_sync(FULL, MR4, o));
    }
    const float beta = q.b / b0;
    const float ib = 1.0f / beta;
    const float d = (rn0 - q.rn) * q.b;
    const float cc = q.y * ib, c2 = cc * cc;
    const float ap = (kTnode - d) * ib, am = (-kTnode - d) * ib;
    const bool base = (c0 == q.c) & (gA == q.gA) & (gB == q.gB) & (gA <= gB) &
                      (mL4 > MR4 || (mL4 > gA && MR4 < gB));
    const bool ok4 = base & (q.y <= 1.2f) & (fabsf(d) <= 0.2f);
    const float zz = fmaxf(fmaf(ap, ap, c2), fmaf(am, am, c2));
    const bool ok2 = base & (zz <= 9.0f), ok3 = base & (zz <= 49.0f);
    // 4: four nodes; 2: two nodes, 7 terms; 3: two nodes, 12 terms
    const int mode = __all_sync(FULL, ok4) ? 4
                     : (__all_sync(FULL, ok2) ? 2 : (__all_sync(FULL, ok3) ? 3 : 0));
    if (mode == 0) return 0;   // warp-uniform
    const float ws = q.s * (float)kInvSqrtPi * ib;   // s / (sqrt(pi) beta), times W per node
    float B[KMP4 + 1];
#pragma unroll
    for (int k = 0; k <= KMP4; ++k) B[k] = 0.0f;
    auto pole = [&](float a, float wt, int K) {
        float zr = a, zi = cc;
#pragma unroll
        for (int k = 1; k <= KMP4; ++k) {
            if (k > K) break;
            B[k] = fmaf(wt, zi, B[k]);
            const float nr = fmaf(zr, a, -zi * cc), ni = fmaf(zr, cc, zi * a);
            zr = nr;
            zi = ni;
        }
    };
    if (mode == 4) {
        const float wa = ws * (float)kWa * 0.5f, wb = ws * (float)kWb * 0.5f;
        pole((kT4a - d) * ib, wa, KMP4);
        pole((-kT4a - d) * ib, wa, KMP4);
        pole((kT4b - d) * ib, wb, KMP4);
        pole((-kT4b - d) * ib, wb, KMP4);
    } else {
        pole(ap, 0.5f * ws, mode == 3 ? KMP4 : KMP2);
        pole(am, 0.5f * ws, mode == 3 ? KMP4 : KMP2);
    }
    float H = (V & kVPlinth) ? q.h : 0.0f;
    const int K = mode == 2 ? KMP2 : KMP4;
    // the round's U and U8 (four nodes): unions of the lines' [cl, ch] and [Lc, Rc]
    int ul = q.cl <= q.ch ? q.cl : INT_MAX, uh = q.cl <= q.ch ? q.ch : INT_MIN;
    int vl = q.Lc <= q.Rc ? q.Lc : INT_MAX, vh = q.Lc <= q.Rc ? q.Rc : INT_MIN;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 1; k <= KMP4; ++k)
            if (k <= K) B[k] += __shfl_xor_sync(FULL, B[k], o);
        if (V & kVPlinth) H += __shfl_xor_sync(FULL, H, o);
        if (mode == 4) {
            ul = min(ul, __shfl_xor_sync(FULL, ul, o));
            uh = max(uh, __shfl_xor_sync(FULL, uh, o));
            vl = min(vl, __shfl_xor_sync(FULL, vl, o));
            vh = max(vh, __shfl_xor_sync(FULL, vh, o));
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k <= KMP4; ++k) rs.B[k] = B[k];
        rs.b0 = b0;
        rs.nrb0 = -rn0 * b0;
        rs.H = H;
        rs.c0 = c0;
        rs.gA = gA;
        rs.gB = gB;
        rs.ulo = ul;
        rs.uhi = uh;
        rs.u8lo = vl;
        rs.u8hi = vh;
        if (mode == 4 || mL4 > MR4) {   // all of [gA + 1, gB - 1] on the left
            rs.RA = gB;
            rs.RB = gB - 1;
        } else {
            rs.RA = mL4;
            rs.RB = MR4;
        }
    }
    __syncwarp();
    return mode;
}

// The series (K terms) over groups [g0, g1] of the tile (p: the warp's tile
// copy at g0); bins in [mlo, mhi] are left out (mlo <= mhi; kNoBin, kNoBin
// for none: no bin reaches it).
template <int K>
__device__ __forceinline__ void round_sweep(const RoundSeries &rs, int g0, int g1, int tg0,
                                            int tg1, float *base, int lane, int mlo, int mhi)
{
    g0 = max(g0, tg0);
    g1 = min(g1, tg1);
    if (g0 > g1) return;
    const unsigned mspan = (unsigned)(mhi - mlo);
    float B[K + 1];
#pragma unroll
    for (int k = 1; k <= K; ++k) B[k] = rs.B[k];
    const float b0 = rs.b0, nrb0 = rs.nrb0, H = rs.H;
    float kf = (float)(32 * g0 + lane - rs.c0);
    int bin = 32 * g0 + lane;
    float *p = base + 32 * (g0 - tg0);
    float *const pe = base + 32 * (g1 - tg0);
    for (; p <= pe; p += 32, kf += 32.0f, bin += 32) {
        const float x = fmaf(kf, b0, nrb0);
        const float w = rcp_ftz(x);
        float h = B[K];
#pragma unroll
        for (int k = K - 1; k >= 1; --k) h = fmaf(h, w, B[k]);
        if ((unsigned)(bin - mlo) > mspan) p[0] += fmaf(h, w * w, -H);
    }
}

// Returns the lines (bit j for line j0 + j) whose core bins are left to the
// caller's core-range pass: those of a batch that took the batched sweep.
template <int V, int NB>
__device__ __forceinline__ unsigned do_batch(Smem &S, int warp, int j0, int tg0, int tg1,
                                             float *base, int lane, unsigned *queue, int &qn,
                                             int t0, int RA, int RB, bool edges_only)
{
    constexpr unsigned kAll = (1u << NB) - 1u;
    const Rec *R = &S.rec[warp][j0];
    // the batch's structure, from the summary in its first record
    const int4 s0 = quadi(R[0], 2);   // (c, gA, gB, lo)
    const int4 s4 = quadi(R[0], 4);   // (ch, smallest L4, largest R4, first bin of U)
    static_assert(NB >= 2, "the batch summary spans two records");
    const int c0 = s0.x, gA = s0.y, gB = s0.z, lo0 = s0.w, mL4 = s4.y, MR4 = s4.z;
    const int flags = __float_as_int(R[0].pad);
    const bool central = mL4 <= MR4;
    const bool uni = (flags & 1) && (!central || (mL4 > gA && MR4 < gB));
    // the lines' cut ranges: most batches share one (the same centre bin and
    // nearly the same remainder), and then an edge group needs one mask
    const bool same_cut = (flags & 2) != 0;
    if (!uni) {   // warp-uniform
        for (int j = 0; j < NB; ++j) {
            const Rec q = S.rec[warp][j0 + j];
            do_line<V>(q, j0 + j, tg0, tg1, base, lane, queue, qn, S, warp, t0, tg0, tg1);
        }
        return 0u;
    }
    if (max(gA, tg0) > min(gB, tg1)) return 0u;
    float b[NB], nrb[NB], Ym[NB], Y2[NB], sy[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        const float4 t = quadf(R[j], 0);   // (b, rn b, Y, sy)
        b[j] = t.x;
        nrb[j] = -t.y;              // x = (k - rn) b, the per-line path's arithmetic
        Ym[j] = t.z - 0.5f;
        Y2[j] = 2.0f * t.z;
        sy[j] = t.w;
    }
    const int kfc = lane - c0;
    // the plinths: every line of the batch is inside its cut in the interior
    // groups, so they subtract the batch's sum of plinths there
    float H = 0.0f;
    if (V & kVPlinth) {
#pragma unroll
        for (int j = 0; j < NB; ++j) H += R[j].h;
    }
    // the batch's two-node sum at one group, less the plinths
    auto two_node = [&](float kf) {
        float v = -H;
#pragma unroll
        for (int j = 0; j < NB; ++j) v = gh2_acc(kf, b[j], nrb[j], Ym[j], Y2[j], sy[j], v);
        return v;
    };
    // the two-node rule over [g0, g1] (clipped to the tile), unmasked
    auto interior = [&](int g0, int g1) {
        g0 = max(g0, tg0);
        g1 = min(g1, tg1);
        if (g0 > g1) return;
        float kf = (float)(32 * g0 + kfc);
        float *p = base + 32 * (g0 - tg0);
        float *const pe = base + 32 * (g1 - tg0);
        for (; p <= pe; p += 32, kf += 32.0f) p[0] += two_node(kf);
    };
    // an edge group: each line adds where its lane's bin is inside its range
    // (one mask for the batch when the lines share their range)
    auto edge = [&](int g) {
        if (g < tg0 || g > tg1) return;
        const float kf = (float)(32 * g + kfc);
        const int bin = 32 * g + lane;
        float v;
        if (same_cut) {   // warp-uniform
            v = (unsigned)(bin - lo0) <= (unsigned)(R[0].hi - lo0) ? two_node(kf) : 0.0f;
        } else {
            v = 0.0f;
#pragma unroll
            for (int j = 0; j < NB; ++j) {
                float t = gh2_acc(kf, b[j], nrb[j], Ym[j], Y2[j], sy[j], 0.0f);
                if (V & kVPlinth) t -= R[j].h;
                v += (bin >= R[j].lo && bin <= R[j].hi) ? t : 0.0f;
            }
        }
        base[32 * (g - tg0)] += v;
    };
    edge(gA);
    if (gB == gA) return kAll;
    edge(gB);
    if (edges_only) return kAll;   // warp-uniform: the round's four-node series took the rest
    // (the round's series covers [gA + 1, RA - 1] and [RB + 1, gB - 1]; with no
    // series RA = gA + 1 and RB = gB - 1, which cover nothing)
    if (!central) {
        interior(max(gA + 1, RA), min(gB - 1, RB));
        return kAll;
    }
    interior(max(gA + 1, RA), mL4 - 1);
    interior(MR4 + 1, min(gB - 1, RB));
    // the central groups: the four-node rule (valid for every r2 >= 64) for
    // every bin outside U8, summed over the batch; U8 is the union of the
    // lines' r2 < 64 ranges, and the caller's core and ring passes evaluate
    // every line at every bin of U8 (the trapezoid rule on U, the union of the
    // inner cores; the 8-node rule on the rest).
    // The two-node parameters are dead here, which keeps the registers in
    // bounds.
    const int c0g = max(mL4, tg0), c1g = min(MR4, tg1);
    if (c0g > c1g) return kAll;
    int ulo = R[1].Lc, uhi = R[1].Rc;   // U8 (empty: ulo > uhi)
    if (ulo > uhi) {   // no core bins: a U8 no bin can meet
        ulo = 0x3fffffff;
        uhi = ulo;
    }
    const unsigned uspan = (unsigned)(uhi - ulo);
    // (the four-node constants are read from shared memory in the loop: a
    // 128-bit load per line and group costs less than holding them)
    float Yc[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) Yc[j] = R[j].Y;
    float kf = (float)(32 * c0g + kfc);
    float *p = base + 32 * (c0g - tg0);
    int bin = 32 * c0g + lane;
    for (int g = c0g; g <= c1g; ++g, kf += 32.0f, p += 32, bin += 32) {
        float v = -H;
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            const float4 f = quadf(R[j], 1);   // (Ca, Cb, sa, sb)
            float r2;
            v += gh4_val(kf, b[j], nrb[j], Yc[j], f.x, f.y, f.z, f.w, &r2);
        }
        if ((unsigned)(bin - ulo) > uspan) p[0] += v;
    }
    return kAll;
}

// The core and ring bins of the batches whose lines took the batched sweep
// (`mask`: NB bits per batch), from the batch summary: U, the union of the
// lines' inner core ranges, and U8 \ U (two intervals), U8 the union of
// their r2 < 64 ranges; the batched sweep left all of U8 out for every line
// of the batch.  Here every line takes every bin of its set inside its cut:
// the trapezoid rule on U (valid for any r2: a bin of U outside a line's own
// inner core is one it would otherwise have taken with another rule), the
// 8-node Gauss-Hermite rule on U8 \ U (every line's r2 there is at least its
// own ring radius R8(y)).  The pairs of all such intervals are laid end to
// end as (interval, bin u, line) with the line innermost -- NB slots per bin,
// so the lanes of an aligned group of NB hold one bin's values, summed by
// shuffles and added by one lane -- and evaluated 32 slots at a time.  A slot
// whose bin lies outside its line's cut adds 0.  Groups of two intervals in
// one step may share a bin: the update is a shared-memory atomic add.  The
// warp's queue rows serve as scratch (the queue is empty here).
template <int NB, bool RING>
__device__ __forceinline__ void core_slots(Smem &S, int warp, int lane, unsigned mask, int t0,
                                           int t1, float *accw)
{
    constexpr int NBR = 32 / NB;                      // batches per round
    constexpr int NI = RING ? 2 * NBR : NBR;          // intervals per round
    constexpr int LG = NB == 8 ? 3 : 2;               // log2 NB
    constexpr unsigned kAll = (1u << NB) - 1u;
    int u0 = 0, nu = 0;
    const int kb = RING ? lane >> 1 : lane;           // this lane's batch
    if (lane < NI && ((mask >> (NB * kb)) & kAll) == kAll) {
        const Rec &q0 = S.rec[warp][NB * kb];         // U = [L2, R2]
        int lo = q0.L2, hi = q0.R2;
        if (RING) {
            const Rec &q1 = S.rec[warp][NB * kb + 1];   // U8 = [Lc, Rc]
            const bool right = lane & 1;
            if (lo > hi) {   // U empty: all of U8 in the left interval
                lo = right ? 1 : q1.Lc;
                hi = right ? 0 : q1.Rc;
            } else {
                const int l8 = right ? hi + 1 : q1.Lc, h8 = right ? q1.Rc : lo - 1;
                lo = l8;
                hi = h8;
            }
        }
        lo = max(lo, t0);
        hi = min(hi, t1);
        if (lo <= hi) {
            u0 = lo;
            nu = hi - lo + 1;
        }
    }
    int inc = NB * nu;
#pragma unroll
    for (int o = 1; o < NI; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    const int total = __shfl_sync(0xffffffffu, inc, NI - 1);
    if (total == 0) return;   // warp-uniform
    int *pre = reinterpret_cast<int *>(S.queue[warp]);   // first slot of interval k
    int *ub = pre + NI;                                  // first bin of interval k
    if (lane < NI) {
        pre[lane] = inc - NB * nu;
        ub[lane] = u0;
    }
    __syncwarp();
    for (int base = 0; base < total; base += 32) {
        const int sl = base + lane;
        // the last interval whose first slot is <= sl (empty intervals share
        // their successor's first slot)
        int k = 0;
#pragma unroll
        for (int st = NI / 2; st > 0; st >>= 1)
            if (k + st < NI && pre[k + st] <= sl) k += st;
        const int rel = sl - pre[k];
        const int u = ub[k] + (rel >> LG);
        const Rec &q = S.rec[warp][NB * (RING ? k >> 1 : k) + (rel & (NB - 1))];
        float v = 0.0f;
        if (sl < total && u >= quadi(q, 2).w && u <= quadi(q, 3).x) {
            const float4 p0 = quadf(q, 0);   // (b, rn b, Y, sy)
            const float kk = (float)(u - quadi(q, 2).x);
            const float x = fmaf(kk, p0.x, -p0.y);
            if (RING) {
                v = gh8_val(x, p0.z, p0.w) - q.h;
            } else {
                const float4 p5 = quadf(q, 5);   // (R2, rn, s, y)
                v = p5.z * core_re<float>(x, p5.w) - q.h;
            }
        }
#pragma unroll
        for (int o = 1; o < NB; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((lane & (NB - 1)) == 0 && sl < total && v != 0.0f) atomicAdd(&accw[u - t0], v);
    }
    __syncwarp();
}

// One batched run over groups [g0, g1] (p: the warp's tile copy at g0) where
// every line is inside its cut and served by rule `cls` (1: one node, 2: two
// nodes): the warp sums the NLB lines per group in a register (x from each
// line's exact integer bin offset, kept exact as a float), less the lines'
// plinths.  share: pairs of lines share one reciprocal (every r2 of the run
// below the rule's bound); origin: one node with x from the run's origin.
template <int V>
__device__ __forceinline__ void wide_sweep(const Rec *R, int cls, bool share, bool origin, int g0,
                                           int g1, float *p, int lane)
{
    float kf[NLB], b[NLB], nrb[NLB], P1[NLB], P2[NLB], sy[NLB];
    float H = 0.0f;
#pragma unroll
    for (int j = 0; j < NLB; ++j) {
        kf[j] = (float)(32 * g0 + lane - R[j].c);   // exact: |offset| < 2^24 bins
        b[j] = R[j].b;
        nrb[j] = -R[j].rnb;
        sy[j] = R[j].sy;
        const float Y = R[j].Y;
        P1[j] = cls == 1 ? Y : Y - 0.5f;   // one node: r2 = x^2 + Y; two nodes: Y - 1/2
        P2[j] = 2.0f * Y;
        if (V & kVPlinth) H += R[j].h;
    }
    float *const pe = p + 32 * (g1 - g0);
    // one node, with x from the run's origin: x = fma(g, 32 b, x0), g the
    // group count from the run's start (wide_flags bounds the cost of rounding x0)
    if (origin) {
        float x0[NLB], b32[NLB];
#pragma unroll
        for (int j = 0; j < NLB; ++j) {
            x0[j] = fmaf(kf[j], b[j], nrb[j]);
            b32[j] = 32.0f * b[j];
        }
        float gf = 0.0f;
        for (; p <= pe; p += 32, gf += 1.0f) {
            float v = -H;
#pragma unroll
            for (int j = 0; j < NLB; j += 2) {
                const float xa = fmaf(gf, b32[j], x0[j]), xb = fmaf(gf, b32[j + 1], x0[j + 1]);
                const float r0 = fmaf(xa, xa, P1[j]), r1 = fmaf(xb, xb, P1[j + 1]);
                v = fmaf(fmaf(sy[j], r1, sy[j + 1] * r0), rcp_ftz(r0 * r1), v);
            }
            p[0] += v;
        }
    } else if (cls == 1 && share) {
        for (; p <= pe; p += 32) {
            float v = -H;
#pragma unroll
            for (int j = 0; j < NLB; j += 2) {
                const float x0 = fmaf(kf[j], b[j], nrb[j]), x1 = fmaf(kf[j + 1], b[j + 1], nrb[j + 1]);
                const float r0 = fmaf(x0, x0, P1[j]), r1 = fmaf(x1, x1, P1[j + 1]);
                v = fmaf(fmaf(sy[j], r1, sy[j + 1] * r0), rcp_ftz(r0 * r1), v);
                kf[j] += 32.0f;
                kf[j + 1] += 32.0f;
            }
            p[0] += v;
        }
    } else if (cls == 1) {
        for (; p <= pe; p += 32) {
            float v = -H;
#pragma unroll
            for (int j = 0; j < NLB; ++j) {
                const float x = fmaf(kf[j], b[j], nrb[j]);
                v = fmaf(sy[j], rcp_ftz(fmaf(x, x, P1[j])), v);
                kf[j] += 32.0f;
            }
            p[0] += v;
        }
    } else if (share) {
        for (; p <= pe; p += 32) {
            float v = -H;
#pragma unroll
            for (int j = 0; j < NLB; j += 2) {
                v = gh2_pair_acc(kf[j], b[j], nrb[j], P1[j], P2[j], sy[j], kf[j + 1], b[j + 1],
                                 nrb[j + 1], P1[j + 1], P2[j + 1], sy[j + 1], v);
                kf[j] += 32.0f;
                kf[j + 1] += 32.0f;
            }
            p[0] += v;
        }
    } else {
        for (; p <= pe; p += 32) {
            float v = -H;
#pragma unroll
            for (int j = 0; j < NLB; ++j) {
                v = gh2_acc(kf[j], b[j], nrb[j], P1[j], P2[j], sy[j], v);
                kf[j] += 32.0f;
            }
            p[0] += v;
        }
    }
}


// The two-node rule over groups [g0, g1] (p: the warp's tile copy at g0) where
// lines of the batch start or end: each line adds where its lane's bin lies in
// its cut, less its plinth there.
template <int V>
__device__ __forceinline__ void wide_masked(const Rec *R, int g0, int g1, float *p, int lane)
{
    float kf[NLB], b[NLB], nrb[NLB], Ym[NLB], Y2[NLB], sy[NLB];
    int lo[NLB];
    unsigned span[NLB];
#pragma unroll
    for (int j = 0; j < NLB; ++j) {
        kf[j] = (float)(32 * g0 + lane - R[j].c);
        b[j] = R[j].b;
        nrb[j] = -R[j].rnb;
        sy[j] = R[j].sy;
        Ym[j] = R[j].Y - 0.5f;
        Y2[j] = 2.0f * R[j].Y;
        lo[j] = R[j].lo;
        span[j] = (unsigned)(R[j].hi - R[j].lo);
    }
    int bin = 32 * g0 + lane;
    float *const pe = p + 32 * (g1 - g0);
    for (; p <= pe; p += 32, bin += 32) {
        float v = 0.0f;
#pragma unroll
        for (int j = 0; j < NLB; ++j) {
            float t = gh2_acc(kf[j], b[j], nrb[j], Ym[j], Y2[j], sy[j], 0.0f);
            if (V & kVPlinth) t -= R[j].h;
            v += (unsigned)(bin - lo[j]) <= span[j] ? t : 0.0f;
            kf[j] += 32.0f;
        }
        p[0] += v;
    }
}

// ---- a wide round's far groups as one series in 1/x --------------------------
//
// Wide lines (the peeled Voigt instance): the 32 lines of a warp's round, all
// inside their cut and outside their four-node groups over a stretch of the
// tile -- left of every line's four-node groups, [max gA + 1, min L4 - 1], and
// right of them, [max R4 + 1, min gB - 1] -- take the two-node rule there,
// and their sum is the series of the short-line rounds (two Lorentzians per
// line, expanded about line 0's offset x; d_j now includes the lines' whole
// bin offsets).  It is used on the groups whose every bin has |x| >= 5 |z|max
// (the terms after z^12 stay below 13 0.2^12 = 5.3e-8 of the sum) with 12
// terms, and with the first 4 terms where |x| >= 100 |z|max (5 0.01^4 = 5e-8);
// never when |z|max > 1000 (the powers' float range) or when line 0 has no
// four-node band.  Returns the groups it covered, [cv[0], cv[1]] and
// [cv[2], cv[3]] (empty: first > last), left for the batches to skip.
constexpr int KW = 12, KWF = 4;

template <int K>
__device__ __forceinline__ void wide_series_sweep(const float *B, float b0, float nrb0, float H,
                                                  int c0, int g0, int g1, int tg0, float *base,
                                                  int lane)
{
    if (g0 > g1) return;
    float kf = (float)(32 * g0 + lane - c0);
    float *p = base + 32 * (g0 - tg0);
    float *const pe = base + 32 * (g1 - tg0);
    for (; p <= pe; p += 32, kf += 32.0f) {
        const float x = fmaf(kf, b0, nrb0);
        const float w = rcp_ftz(x);
        float h = B[K];
#pragma unroll
        for (int k = K - 1; k >= 1; --k) h = fmaf(h, w, B[k]);
        p[0] += fmaf(h, w * w, -H);
    }
}

template <int V>
__device__ __forceinline__ void wide_round(const Rec &q, bool valid, int lane, int tg0, int tg1,
                                           float *base, int *cv)
{
    constexpr unsigned FULL = 0xffffffffu;
    cv[0] = cv[2] = 1;
    cv[1] = cv[3] = 0;
    const bool has4 = q.L4 <= q.R4;
    const int c0 = __shfl_sync(FULL, q.c, 0);
    const float b0 = __shfl_sync(FULL, q.b, 0), rn0 = __shfl_sync(FULL, q.rn, 0);
    const bool has40 = __shfl_sync(FULL, has4 ? 1 : 0, 0) != 0;
    // this line's two nodes about line 0's offset
    const float beta = q.b / b0;
    const float ib = 1.0f / beta;
    const float d = ((float)(c0 - q.c) + (rn0 - q.rn)) * q.b;
    const float cc = q.y * ib;
    const float ap = (kTnode - d) * ib, am = (-kTnode - d) * ib;
    float zm = sqrtf(fmaxf(fmaf(ap, ap, cc * cc), fmaf(am, am, cc * cc)));
    // the safe stretches: inside every cut, outside every line's four-node groups
    int aL = q.gA + 1, bL = has4 ? q.L4 - 1 : q.gB - 1;
    int aR = has4 ? q.R4 + 1 : q.gA + 1, bR = q.gB - 1;
    int any4 = has4 ? 1 : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        zm = fmaxf(zm, __shfl_xor_sync(FULL, zm, o));
        aL = max(aL, __shfl_xor_sync(FULL, aL, o));
        bL = min(bL, __shfl_xor_sync(FULL, bL, o));
        aR = max(aR, __shfl_xor_sync(FULL, aR, o));
        bR = min(bR, __shfl_xor_sync(FULL, bR, o));
        any4 |= __shfl_xor_sync(FULL, any4, o);
    }
    const bool ok = valid && q.gA <= q.gB;
    if (!__all_sync(FULL, ok) || !has40 || !(zm <= 1000.0f)) return;   // warp-uniform
    // groups whose every bin is at least X from the reference centre c0 + rn0
    const float cen = (float)c0 + rn0;
    auto left_of = [&](float X) { return (int)floorf((cen - X / b0 - 31.0f) * (1.0f / 32.0f)); };
    auto right_of = [&](float X) { return (int)ceilf((cen + X / b0) * (1.0f / 32.0f)); };
    const int gl = left_of(5.0f * zm), gr = right_of(5.0f * zm);
    const int gl4 = left_of(100.0f * zm), gr4 = right_of(100.0f * zm);
    // left cover [l0, l1], right cover [r0, r1] (both clear of line 0's centre)
    const int l0 = max(aL, tg0), l1 = min(min(bL, gl), tg1);
    const int r0 = max(max(aR, gr), tg0), r1 = min(bR, tg1);
    const bool useL = l0 <= l1, useR = r0 <= r1 && any4;
    if (!useL && !useR) return;
    // coefficients: lane j, line j; summed over the warp
    const float wt = q.s * (float)(0.5 * kInvSqrtPi) * ib;
    float B[KW + 1];
#pragma unroll
    for (int k = 0; k <= KW; ++k) B[k] = 0.0f;
#pragma unroll
    for (int sgn = 0; sgn < 2; ++sgn) {
        const float a = sgn ? am : ap;
        float zr = a, zi = cc;
#pragma unroll
        for (int k = 1; k <= KW; ++k) {
            B[k] = fmaf(wt, zi, B[k]);
            const float nr = fmaf(zr, a, -zi * cc), ni = fmaf(zr, cc, zi * a);
            zr = nr;
            zi = ni;
        }
    }
    float H = (V & kVPlinth) ? q.h : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 1; k <= KW; ++k) B[k] += __shfl_xor_sync(FULL, B[k], o);
        if (V & kVPlinth) H += __shfl_xor_sync(FULL, H, o);
    }
    const float nrb0 = -rn0 * b0;
    if (useL) {   // far part (4 terms) then near part (12 terms)
        const int m = min(l1, gl4);
        wide_series_sweep<KWF>(B, b0, nrb0, H, c0, l0, m, tg0, base, lane);
        wide_series_sweep<KW>(B, b0, nrb0, H, c0, max(l0, m + 1), l1, tg0, base, lane);
        cv[0] = l0;
        cv[1] = l1;
    }
    if (useR) {
        const int m = max(r0, gr4);
        wide_series_sweep<KW>(B, b0, nrb0, H, c0, r0, m - 1 < r1 ? m - 1 : r1, tg0, base, lane);
        wide_series_sweep<KWF>(B, b0, nrb0, H, c0, m, r1, tg0, base, lane);
        cv[2] = r0;
        cv[3] = r1;
    }
}

// Batches of wide lines (the peeled instances: Voigt and Lorentzian, with or
// without the plinth).  The lines of a batch have their own centres; their
// per-tile flags (wide_flags) decide the tile's handling:
// - every line in one band over the whole tile, clear of its edge groups: one
//   batched run, one-node or two-node rule (a tile across a line's
//   one-/two-node boundary takes the two-node rule for every line);
// - else, when the two-node rule may serve every line over the tile and no
//   line's four-node or core groups meet it: the spans where lines start or
//   end ([min gA, max gA], [min gB, max gB]) run the masked two-node rule and
//   the groups between them one unmasked batched two-node run;
// - else the whole tile goes line by line.
template <int V>
__device__ __forceinline__ void do_batch_wide(Smem &S, int warp, int j0, int tg0, int tg1,
                                              float *base, int lane, unsigned *queue, int &qn,
                                              int t0, int rg0, int rg1)
{
    const Rec *R = &S.rec[warp][j0];
    int fand = 127, fany = 0, cls = -1;
    int A0 = INT_MAX, A1 = INT_MIN, B0 = INT_MAX, B1 = INT_MIN;
#pragma unroll
    for (int j = 0; j < NLB; ++j) {
        const int f = __float_as_int(R[j].pad);
        fand &= f;
        fany |= f;
        cls = j == 0 ? (f & 3) : (cls == (f & 3) ? cls : 0);
        A0 = min(A0, R[j].gA);
        A1 = max(A1, R[j].gA);
        B0 = min(B0, R[j].gB);
        B1 = max(B1, R[j].gB);
    }
    const bool edges = cls == 0;
    // masked spans of at most kMaskSpan groups in all: the masked rule takes
    // every line in every group of a span, whether the line has bins there or not
    const int span = max(min(A1, rg1) - max(A0, rg0) + 1, 0) + max(min(B1, rg1) - max(B0, rg0) + 1, 0);
    if (edges && !((fand & 16) && !(fany & 64) && A1 < B0 && span <= kMaskSpan)) {
        for (int j = 0; j < NLB; ++j) {
            const Rec q = S.rec[warp][j0 + j];
            do_line<V>(q, j0 + j, tg0, tg1, base, lane, queue, qn, S, warp, t0, rg0, rg1);
        }
        return;
    }
    const int g0 = edges ? max(A1 + 1, rg0) : rg0, g1 = edges ? min(B0 - 1, rg1) : rg1;
    if (g0 <= g1)
        wide_sweep<V>(R, edges ? 2 : cls, (fand & (edges ? 32 : 4)) != 0, !edges && (fand & 8),
                      g0, g1, base + 32 * (g0 - tg0), lane);
    if (edges) {   // the masked spans, from the records again
        int a0 = INT_MAX, a1 = INT_MIN, b0 = INT_MAX, b1 = INT_MIN;
#pragma unroll
        for (int j = 0; j < NLB; ++j) {
            a0 = min(a0, R[j].gA);
            a1 = max(a1, R[j].gA);
            b0 = min(b0, R[j].gB);
            b1 = max(b1, R[j].gB);
        }
        for (int k = 0; k < 2; ++k) {
            const int m0 = max(k ? b0 : a0, rg0), m1 = min(k ? b1 : a1, rg1);
            if (m0 <= m1) wide_masked<V>(R, m0, m1, base + 32 * (m0 - tg0), lane);
        }
    }
}

__device__ __forceinline__ void fold(float *accs, float *hi, float *lo, int tile, int tid)
{
    for (int i = tid; i < tile; i += NT) {
        float sum = 0.0f;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            sum += accs[w * tile + i];
            accs[w * tile + i] = 0.0f;
        }
        float h, e;
        two_sum(hi[i], sum, &h, &e);
        hi[i] = h;
        lo[i] += e;
    }
}

template <int V>
__global__ void __launch_bounds__(NT, 3)
    k_gather_f32(const Prob *__restrict__ probs, GridD g, int64_t ntiles, int64_t m,
                 const int64_t *__restrict__ item_off, const int64_t *__restrict__ tile_lb,
                 const int64_t *__restrict__ tile_le, int lmax, unsigned long long *counter,
                 int tile)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem &S = *reinterpret_cast<Smem *>(smem_raw);
    float *const accs = reinterpret_cast<float *>(smem_raw + sizeof(Smem));   // [NW][tile]
    float *const shi = accs + NW * tile, *const slo = shi + tile;
    __shared__ long long s_item, s_pt, s_lb, s_le;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned *queue = S.queue[warp];

    for (int i = tid; i < NW * tile; i += NT) accs[i] = 0.0f;
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
        for (int i = tid; i < tile; i += NT) {
            shi[i] = 0.0f;
            slo[i] = 0.0f;
        }
        __syncthreads();
        if (s_item < 0) break;
        const int64_t pt = s_pt;
        const int p = (int)(pt / ntiles);
        // the tile's first bin; with a halo the window starts H bins before the
        // central bins the tile owns (possibly before bin 0: those bins stay empty)
        const int64_t tix = pt - (int64_t)p * ntiles;
        const int t0 = g.halo ? (int)(tix * (tile - 2 * g.halo)) - g.halo : (int)(tix * tile);
        const int t1 = (int)min((int64_t)t0 + tile, g.nbins) - 1;  // last bin of the tile
        const int64_t l_begin = s_lb, l_end = s_le;
        const Prob &pr = probs[p];
        const int scale = *pr.scale_exp;
        const int tg0 = t0 >> 5, tg1 = t1 >> 5;           // the tile's groups
        float *accb = accs + warp * tile + lane;
        int rounds = 0;
        for (int64_t base = l_begin; base < l_end; base += NT) {
            // short lines: warp w owns lines base + 32 w + lane (consecutive lines,
            // whose batches share their structure); wide lines: base + w + 8 lane,
            // so that every warp of the block gets lines from the whole round and
            // the warps reach the fold barriers together (7 % at config 3)
            const int64_t l = (V & kVPeel) ? base + warp + NW * lane : base + tid;
            Rec q;
            if (l < l_end) {
                make_rec(pr, g, l, scale, &q);
                if (V & kVPeel)
                    q.pad = __int_as_float(wide_flags(q, tg0, tg1, g.profile == kProfVoigt));
            } else {  // past the item's lines: an empty record
                q.c = 0;
                q.lo = 0x3fffffff;
                q.hi = -0x3fffffff;
                q.gA = 1;
                q.gB = 0;
                q.L4 = q.cl = q.Lc = 1;
                q.R4 = q.ch = q.Rc = 0;
                q.pad = 0.0f;
            }
            // short lines: the round's series, when it can take one (before the
            // batch summary, which overwrites fields of the batches' first records)
            RoundSeries &rs = *reinterpret_cast<RoundSeries *>(S.queue[warp]);
            int mode = 0;
            if ((V & ~kVPlinth) == 0) {
                mode = round_series<V>(q, lane, rs);
                batch_summary(q, lane);
                if (mode == 4) {   // the batches' core and ring passes take the round's U, U8
                    if ((lane & (NLS - 1)) == 0) {
                        q.L2 = rs.ulo;
                        q.R2 = rs.uhi;
                    } else if ((lane & (NLS - 1)) == 1) {
                        q.Lc = rs.u8lo;
                        q.Rc = rs.u8hi;
                    }
                }
            }
            S.rec[warp][lane] = q;
            __syncwarp();
            int qn = 0;
            if ((V & ~kVPlinth) == 0) {   // short Voigt lines, with or without the plinth
                int RA = INT_MIN, RB = INT_MAX;
                if (mode == 4) {   // warp-uniform
                    const bool u8 = rs.u8lo <= rs.u8hi;
                    round_sweep<KMP4>(rs, rs.gA + 1, rs.gB - 1, tg0, tg1, accb, lane,
                                      u8 ? rs.u8lo : kNoBin, u8 ? rs.u8hi : kNoBin);
                } else if (mode == 2) {
                    round_sweep<KMP2>(rs, rs.gA + 1, rs.RA - 1, tg0, tg1, accb, lane, kNoBin,
                                      kNoBin);
                    round_sweep<KMP2>(rs, rs.RB + 1, rs.gB - 1, tg0, tg1, accb, lane, kNoBin,
                                      kNoBin);
                    RA = rs.RA;
                    RB = rs.RB;
                } else if (mode == 3) {
                    round_sweep<KMP4>(rs, rs.gA + 1, rs.RA - 1, tg0, tg1, accb, lane, kNoBin,
                                      kNoBin);
                    round_sweep<KMP4>(rs, rs.RB + 1, rs.gB - 1, tg0, tg1, accb, lane, kNoBin,
                                      kNoBin);
                    RA = rs.RA;
                    RB = rs.RB;
                }
                unsigned rmask = 0u;
                for (int j0 = 0; j0 < 32; j0 += NLS)
                    rmask |= do_batch<V, NLS>(S, warp, j0, tg0, tg1, accb, lane, queue, qn, t0,
                                              RA, RB, mode == 4)
                             << j0;
                drain_rest(queue, qn, S, warp, lane, t0, accb - lane);
                core_slots<NLS, false>(S, warp, lane, rmask, t0, t1, accb - lane);
                core_slots<NLS, true>(S, warp, lane, rmask, t0, t1, accb - lane);
            } else if ((V & kVPeel) && !(V & (kVDoppler | kVBinned))) {
                // the round's far groups as one series (Voigt), then the batches on
                // the rest of the tile
                int cv[4] = {1, 0, 1, 0};
                if (g.profile == kProfVoigt) wide_round<V>(q, l < l_end, lane, tg0, tg1, accb, cv);
                int pr0[3], pr1[3], np = 0, start = tg0;
                if (cv[0] <= cv[1]) {
                    if (start < cv[0]) {
                        pr0[np] = start;
                        pr1[np++] = cv[0] - 1;
                    }
                    start = cv[1] + 1;
                }
                if (cv[2] <= cv[3]) {
                    if (start < cv[2]) {
                        pr0[np] = start;
                        pr1[np++] = cv[2] - 1;
                    }
                    start = cv[3] + 1;
                }
                if (start <= tg1) {
                    pr0[np] = start;
                    pr1[np++] = tg1;
                }
                for (int k = 0; k < np; ++k)
                    for (int j0 = 0; j0 < 32; j0 += NLB)
                        do_batch_wide<V>(S, warp, j0, tg0, tg1, accb, lane, queue, qn, t0, pr0[k],
                                         pr1[k]);
            } else {
                for (int j = 0; j < 32; ++j) {
                    // a register copy: the record must not be re-read from shared
                    // memory after every store into the tile copy
                    const Rec q = S.rec[warp][j];
                    do_line<V>(q, j, tg0, tg1, accb, lane, queue, qn, S, warp, t0, tg0, tg1);
                }
            }
            drain_rest(queue, qn, S, warp, lane, t0, accb - lane);
            if (++rounds == FLUSH_ROUNDS) {
                rounds = 0;
                __syncthreads();
                fold(accs, shi, slo, tile, tid);
                __syncthreads();
            }
        }
        __syncthreads();
        fold(accs, shi, slo, tile, tid);
        __syncthreads();
        for (int i = tid; i <= t1 - t0; i += NT) {
            const double tot = (double)shi[i] + (double)slo[i];
            if (tot != 0.0 && t0 + i >= 0) atomicAdd(pr.acc + t0 + i, tot);
        }
        __syncthreads();
    }
}

}  // namespace f32g

// Each line's bin geometry as the FP32C records take it (c, rn, lo, hi; an
// empty range when no bin of the grid is inside the cut), for a line list
// whose problems share it: a fixed cut or none and no pressure shift, so that
// the geometry depends on the line and the grid only.
__global__ void k_line_geo(Prob p, GridD g, int4 *geo)
{
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < p.n;
         l += (int64_t)gridDim.x * blockDim.x) {
        int c, lo, hi;
        float rn;
        CutW cw;
        line_geometry_cut(p, g, l, &cw, &c, &rn, &lo, &hi);
        geo[l] = make_int4(c, __float_as_int(rn), lo, hi);
    }
}

int line_geo_launch(const Prob &p, const GridD &g, int4 *geo, cudaStream_t st, int num_sms)
{
    if (p.n <= 0) return HK_OK;
    k_line_geo<<<num_sms * 4, 256, 0, st>>>(p, g, geo);
    const cudaError_t e = cudaGetLastError();
    return e ? fail_cuda(e) : HK_OK;
}

// Dynamic shared memory of a launch with `tile`-bin tiles.
static size_t f32_smem(int tile) { return sizeof(f32g::Smem) + (size_t)(f32g::NW + 2) * tile * 4; }

bool gather_f32_tile_ok(int tile) { return tile == 1024 || tile == 2048; }

// Lines at least this many bins wide take the peeled sweeps.
constexpr double kPeelBins = 1024.0;

// Blocks per SM of a kernel instance on the current device for a dynamic
// shared-memory size, after raising the instance's shared-memory limit there
// to the widest tile's need (a per-device attribute): done once per (device,
// instance, size) under a lock, so concurrent first calls from several host
// threads, or a second device, each see a configured kernel.
static int configure_once(const void *fn, size_t smem, int threads, int *per_sm_out)
{
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, bool> limit_set;
    static std::map<std::pair<std::pair<int, const void *>, size_t>, int> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return fail_cuda(e);
    std::lock_guard<std::mutex> lk(mu);
    auto it = done.find({{dev, fn}, smem});
    if (it != done.end()) {
        *per_sm_out = it->second;
        return HK_OK;
    }
    if (!limit_set[{dev, fn}]) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)f32_smem(f32g::TILE_MAX));
        if (e) return fail_cuda(e);
        limit_set[{dev, fn}] = true;
    }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
    if (e) return fail_cuda(e);
    if (per_sm < 1) per_sm = 1;
    done[{{dev, fn}, smem}] = per_sm;
    *per_sm_out = per_sm;
    return HK_OK;
}

template <int V>
static int launch_variant(const Prob *probs_d, const GridD &g, int64_t ntiles, int64_t m,
                          const int64_t *item_off, const int64_t *tile_lb,
                          const int64_t *tile_le, int lmax, unsigned long long *counter,
                          cudaStream_t st, int num_sms, int tile)
{
    const size_t smem = f32_smem(tile);
    int per_sm = 0;
    int rc = configure_once((const void *)f32g::k_gather_f32<V>, smem, f32g::NT, &per_sm);
    if (rc) return rc;
    cudaError_t e;
    f32g::k_gather_f32<V><<<num_sms * per_sm, f32g::NT, smem, st>>>(
        probs_d, g, ntiles, m, item_off, tile_lb, tile_le, lmax, counter, tile);
    e = cudaGetLastError();
    return e ? fail_cuda(e) : HK_OK;
}

int gather_f32_launch(const Prob *probs_d, const GridD &g, int64_t ntiles, int64_t m,
                      const int64_t *item_off, const int64_t *tile_lb, const int64_t *tile_le,
                      int lmax, unsigned long long *counter, cudaStream_t st, int num_sms,
                      int tile)
{
    if (!gather_f32_tile_ok(tile)) return HK_EINVAL;
    const bool wide = g.W <= 0.0 || 2.0 * g.W + 1.0 >= kPeelBins;
    // the Lorentzian is the one-node rule itself: it needs the one-node passes
    // that only the peeled instance keeps
    int v = (wide || g.profile == kProfLorentz ? f32g::kVPeel : 0) |
            (g.plinth && has_cut(g) ? f32g::kVPlinth : 0);
    if (g.profile == kProfDoppler) v = f32g::kVPeel | f32g::kVPlinth | f32g::kVDoppler;
    if (g.profile == kProfBinned) v = f32g::kVPeel | f32g::kVPlinth | f32g::kVBinned;
    switch (v) {
    case f32g::kVPeel | f32g::kVPlinth | f32g::kVDoppler:
        return launch_variant<f32g::kVPeel | f32g::kVPlinth | f32g::kVDoppler>(
            probs_d, g, ntiles, m, item_off, tile_lb, tile_le, lmax, counter, st, num_sms, tile);
    case f32g::kVPeel | f32g::kVPlinth | f32g::kVBinned:
        return launch_variant<f32g::kVPeel | f32g::kVPlinth | f32g::kVBinned>(
            probs_d, g, ntiles, m, item_off, tile_lb, tile_le, lmax, counter, st, num_sms, tile);
    case 0:
        return launch_variant<0>(probs_d, g, ntiles, m, item_off, tile_lb, tile_le, lmax,
                                 counter, st, num_sms, tile);
    case 1:
        return launch_variant<1>(probs_d, g, ntiles, m, item_off, tile_lb, tile_le, lmax,
                                 counter, st, num_sms, tile);
    case 2:
        return launch_variant<2>(probs_d, g, ntiles, m, item_off, tile_lb, tile_le, lmax,
                                 counter, st, num_sms, tile);
    default:
        return launch_variant<3>(probs_d, g, ntiles, m, item_off, tile_lb, tile_le, lmax,
                                 counter, st, num_sms, tile);
    }
}

}  // namespace hk
