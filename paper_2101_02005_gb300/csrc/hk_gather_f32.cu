// hk_gather_f32.cu -- the FP32-compensated Voigt sum (HK_FP32C) on sm_103a.
//
// Line-major warps over a shared-memory tile of the grid:
//
// * Work items are (problem, tile of TILE bins, chunk of <= lmax lines), as
//   in the FP64 gather; a persistent grid pulls them from an atomic counter.
// * Inside an item every warp takes 32 lines at a time: lane i computes the
//   parameters of line i once (bin geometry in FP64, strength and widths in
//   FP32, band boundaries) into a per-warp record table; then the warp sweeps
//   each line's bins inside the tile, 32 consecutive bins per step (lane =
//   bin), so no lane ever tests whether its bin is inside the cut.
// * The Faddeeva band of a 32-bin group is the band of its bin nearest the
//   line centre.  The bands form nested intervals of group indices around
//   the centre, computed once per line, so each group runs one formula with
//   no divergence.  Bins of the central groups that fall in the core band
//   (r2 < 64) go to a per-warp queue and are evaluated 32 at a time.
// * Each warp adds into its own FP32 copy of the tile in shared memory
//   (consecutive bins, no bank conflicts, no atomics); every FLUSH_ROUNDS
//   rounds the copies are summed into a (hi, lo) two-sum pair per bin, and at
//   the end of the item hi + lo goes to the FP64 accumulator of the problem
//   with one atomicAdd per bin.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "hk_internal.cuh"
#include "hk_launch.h"

namespace hk {

namespace f32g {

constexpr int NW = 8;             // warps per block
constexpr int NT = NW * 32;
constexpr int TILE = 2048;        // bins per tile
constexpr int QCAP = 64;          // core-queue entries per warp
constexpr int FLUSH_ROUNDS = 2;   // rounds (32 lines per warp each) between two-sum folds

// Per-line record, computed once per (line, item) by one lane.
struct __align__(16) Rec {
    float b, rn, Y, s;          // x step per bin, centre offset from bin c, y^2, scaled strength
    int c, lo, hi, pad;         // nearest bin to the centre, inclusive bin range in the cut
    int kL2, kR2, kL3, kR3;     // offsets k = bin - c with r2 < 1.5e6 / 2500 (kL > kR: none)
    int kL4, kR4, kLc, kRc;     // ... r2 < 200 / 64
    float rnb, sy, sy2, Yq;     // rn b, s y / sqrt(pi), sy / 2, Y + 1/4          (2 nodes)
    float C3, s23, s13, Ca;     // 3 Y + 9/4, 2 sy / 3, sy / 3                      (3 nodes)
    float Cb, sa, sb, y;        // 2 tau Y + tau^2 for both 4-node pairs, 2 W sy    (4 nodes)
};

struct Smem {
    float acc[NW][TILE];
    float hi[TILE];
    float lo[TILE];
    Rec rec[NW][32];
    unsigned queue[NW][QCAP];
};

constexpr float kTa = 0.27525512860841106f, kTb = 2.724744871391589f;   // 4-node tau
constexpr float kWa = 2.0f * 0.4541241452319315f, kWb = 2.0f * 0.04587585476806851f;

// Offsets k with |k - rn| < D, D = sqrt(R - Y) / b widened by a relative 1e-4
// and 1e-3 bins so a bin on the edge takes the more accurate band.
__device__ __forceinline__ void band_k(float R, float Y, float b, float rn, int *kL, int *kR)
{
    const float d2 = R - Y;
    if (!(d2 > 0.0f)) {
        *kL = 1;
        *kR = 0;
        return;
    }
    const float D = fminf(sqrtf(d2) / b * 1.0001f + 1e-3f, 1.0e9f);
    *kL = (int)floorf(rn - D) + 1;
    *kR = (int)ceilf(rn + D) - 1;
}

__device__ __forceinline__ void make_rec(const Prob &pr, const GridD &g, int64_t l, int scale,
                                         Rec *out)
{
    Rec q;
    const double nu0 = pr.nu0[l];
    int i0, lo, hi;
    double r;
    bool any = line_geometry(nu0, g, &i0, &r, &lo, &hi);
    int c;
    double rn;
    nearest_bin(i0, r, &c, &rn);
    q.c = c;
    q.lo = lo;
    q.hi = hi;
    q.rn = (float)rn;
    q.pad = 0;
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
    band_k(1.5e6f, Y, b, q.rn, &q.kL2, &q.kR2);
    band_k(2500.0f, Y, b, q.rn, &q.kL3, &q.kR3);
    band_k(200.0f, Y, b, q.rn, &q.kL4, &q.kR4);
    band_k(64.0f, Y, b, q.rn, &q.kLc, &q.kRc);
    q.rnb = q.rn * b;
    q.sy = sy;
    q.sy2 = 0.5f * sy;
    q.Yq = Y + 0.25f;
    q.C3 = fmaf(3.0f, Y, 2.25f);
    q.s23 = sy * (2.0f / 3.0f);
    q.s13 = sy * (1.0f / 3.0f);
    q.Ca = fmaf(2.0f * kTa, Y, kTa * kTa);
    q.Cb = fmaf(2.0f * kTb, Y, kTb * kTb);
    q.sa = sy * kWa;
    q.sb = sy * kWb;
    *out = q;
}

// Groups whose nearest offset is inside [kL, kR], nested in [Lp, Rp].  Group g
// covers offsets [ka + 32 g, ka + 32 g + 31]; it meets [kL, kR] iff
// (kL - ka) >> 5 <= g <= (kR - ka) >> 5 (arithmetic shifts are floor
// divisions).  An empty band sits at Rp + 1.
__device__ __forceinline__ void band_groups(int kL, int kR, int ka, int Lp, int Rp, int *L, int *R)
{
    int lo = (kL - ka) >> 5, hi = (kR - ka) >> 5;
    lo = max(lo, Lp);
    hi = min(hi, Rp);
    if (kL > kR || lo > hi) {
        *L = Rp + 1;
        *R = Rp;
    } else {
        *L = lo;
        *R = hi;
    }
}

// Value of one pair in band BAND at offset kf (float bin offset from c).
template <int BAND> __device__ __forceinline__ float pair_f(const Rec &q, float kf)
{
    const float x = fmaf(kf, q.b, -q.rnb);
    const float X = x * x;
    const float r2 = X + q.Y;
    // __fdividef: one reciprocal and a multiply, within 2 ulp while the
    // divisor is below 2^126 (gh1 beyond that gives 0, far below any sum)
    if (BAND == kBandGH1) {
        return __fdividef(q.sy, r2);
    } else if (BAND == kBandGH2) {          // |z^2 - 1/2|^2 = r2^2 - X + Y + 1/4
        const float d = fmaf(r2, r2, q.Yq - X);
        return __fdividef(fmaf(r2, q.sy, q.sy2), d);
    } else if (BAND == kBandGH3) {          // |z^2 - 3/2|^2 = r2^2 - 3 X + 3 Y + 9/4
        const float d = fmaf(r2, r2, fmaf(-3.0f, X, q.C3));
        const float u = fmaf(r2, r2, 1.5f * r2);
        return __fdividef(fmaf(q.s23, d, q.s13 * u), r2 * d);
    } else {                                // both 4-node pairs
        const float da = fmaf(r2, r2, fmaf(-2.0f * kTa, X, q.Ca));
        const float db = fmaf(r2, r2, fmaf(-2.0f * kTb, X, q.Cb));
        return __fdividef(fmaf(q.sa * (r2 + kTa), db, q.sb * (r2 + kTb) * da), da * db);
    }
}

// One band over groups [g0, g1) of a line.  `acc` points at the warp's tile
// copy at the line's first bin plus this lane; `kf0` is this lane's offset in
// group 0; groups below gf are full, group gf (if any) has `rem` live lanes.
template <int BAND>
__device__ __forceinline__ void sweep(const Rec &q, int g0, int g1, int gf, int rem, float *acc,
                                      float kf0, int lane)
{
    const int gfull = min(g1, gf);
    int g = g0;
    float kf = kf0 + (float)(32 * g0);
    float *p = acc + 32 * g0;
    for (; g + 1 < gfull; g += 2, kf += 64.0f, p += 64) {
        const float v0 = pair_f<BAND>(q, kf);
        const float v1 = pair_f<BAND>(q, kf + 32.0f);
        p[0] += v0;
        p[32] += v1;
    }
    if (g < gfull) {
        p[0] += pair_f<BAND>(q, kf);
        ++g;
        kf += 32.0f;
        p += 32;
    }
    if (g1 > gf && g0 <= gf && lane < rem) {   // the partial last group
        const float kfl = kf0 + (float)(32 * gf);
        acc[32 * gf] += pair_f<BAND>(q, kfl);
    }
}

template <int BAND>
__device__ __forceinline__ void sweep2(const Rec &q, int a0, int a1, int b0, int b1, int gf,
                                       int rem, float *acc, float kf0, int lane)
{
    if (a0 < a1) sweep<BAND>(q, a0, a1, gf, rem, acc, kf0, lane);
    if (b0 < b1) sweep<BAND>(q, b0, b1, gf, rem, acc, kf0, lane);
}

__device__ __forceinline__ void core_entry(Smem &S, int warp, int t0, unsigned e)
{
    const Rec &qq = S.rec[warp][e >> 16];
    const int tidx = (int)(e & 0xffffu);
    const float kk = (float)(t0 + tidx - qq.c);
    const float xx = fmaf(kk, qq.b, -qq.rnb);
    atomicAdd(&S.acc[warp][tidx], qq.s * core_re<float>(xx, qq.y));
}

// Central groups [g0, g1): bins with r2 >= 64 take the 4-node rule in place,
// core bins (r2 < 64) are queued as (record slot, tile index) and evaluated
// 32 at a time.
__device__ __forceinline__ void sweep_core(const Rec &q, int slot, int g0, int g1, int nact,
                                           float *acc0, float kf0, int lane, int tidx0,
                                           unsigned *queue, int &qn, Smem &S, int warp, int t0)
{
    int off = 32 * g0 + lane;
    float kf = kf0 + (float)(32 * g0);
    for (int gi = g0; gi < g1; ++gi, off += 32, kf += 32.0f) {
        const bool act = off < nact;
        const float x = fmaf(kf, q.b, -q.rnb);
        const float r2 = fmaf(x, x, q.Y);
        const bool core = act && r2 < 64.0f;
        if (act && !core) acc0[off] += pair_f<kBandGH4>(q, kf);
        const unsigned m = __ballot_sync(0xffffffffu, core);
        if (m) {
            const int pos = qn + __popc(m & ((1u << lane) - 1u));
            if (core) queue[pos] = ((unsigned)slot << 16) | (unsigned)(tidx0 + off);
            qn += __popc(m);
            __syncwarp();
            if (qn >= 32) {
                core_entry(S, warp, t0, queue[lane]);
                __syncwarp();
                if (lane < qn - 32) queue[lane] = queue[lane + 32];
                qn -= 32;
                __syncwarp();
            }
        }
    }
}

__device__ __forceinline__ void drain_rest(unsigned *queue, int &qn, Smem &S, int warp, int lane,
                                           int t0)
{
    if (qn > 0) {
        if (lane < qn) core_entry(S, warp, t0, queue[lane]);
        qn = 0;
    }
    __syncwarp();
}

__device__ __forceinline__ void fold(Smem &S, int tid)
{
    for (int i = tid; i < TILE; i += NT) {
        float sum = 0.0f;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            sum += S.acc[w][i];
            S.acc[w][i] = 0.0f;
        }
        float h, e;
        two_sum(S.hi[i], sum, &h, &e);
        S.hi[i] = h;
        S.lo[i] += e;
    }
}

__global__ void __launch_bounds__(NT, 2)
    k_gather_f32(const Prob *__restrict__ probs, GridD g, int64_t ntiles, int64_t m,
                 const int64_t *__restrict__ item_off, const int64_t *__restrict__ tile_lb,
                 const int64_t *__restrict__ tile_le, int lmax, unsigned long long *counter)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem &S = *reinterpret_cast<Smem *>(smem_raw);
    __shared__ long long s_item, s_pt, s_lb, s_le;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned *queue = S.queue[warp];

    for (int i = tid; i < NW * TILE; i += NT) (&S.acc[0][0])[i] = 0.0f;
    for (;;) {
        if (tid == 0) {
            long long item = (long long)atomicAdd(counter, 1ull);
            long long total = item_off[m];
            if (item >= total) {
                s_item = -1;
            } else {
                long long a = 0, b = m;
                while (b - a > 1) {
                    long long c = (a + b) >> 1;
                    if (item_off[c] <= item) a = c; else b = c;
                }
                long long lb = tile_lb[a] + (item - item_off[a]) * lmax;
                s_item = item;
                s_pt = a;
                s_lb = lb;
                s_le = min((long long)tile_le[a], lb + lmax);
            }
        }
        for (int i = tid; i < TILE; i += NT) {
            S.hi[i] = 0.0f;
            S.lo[i] = 0.0f;
        }
        __syncthreads();
        if (s_item < 0) break;
        const int64_t pt = s_pt;
        const int p = (int)(pt / ntiles);
        const int t0 = (int)((pt - (int64_t)p * ntiles) * TILE);
        const int t1 = (int)min((int64_t)t0 + TILE, g.nbins) - 1;  // last bin of the tile
        const int64_t l_begin = s_lb, l_end = s_le;
        const Prob &pr = probs[p];
        const int scale = *pr.scale_exp;
        int rounds = 0;
        for (int64_t base = l_begin; base < l_end; base += NT) {
            const int64_t l = base + tid;  // warp w owns lines base + 32 w + lane
            Rec q;
            if (l < l_end) {
                make_rec(pr, g, l, scale, &q);
            } else {
                q.lo = 0x3fffffff;
                q.hi = -0x3fffffff;
            }
            S.rec[warp][lane] = q;
            __syncwarp();
            int qn = 0;
            for (int j = 0; j < 32; ++j) {
                const Rec &r = S.rec[warp][j];
                const int a = max(r.lo, t0), bb = min(r.hi, t1);
                if (a > bb) continue;  // warp-uniform
                const Rec q2 = r;
                const int ka = a - q2.c;
                const int nact = bb - a + 1;
                const int G = (nact + 31) >> 5, gf = nact >> 5, rem = nact & 31;
                int L2, R2, L3, R3, L4, R4, Lc, Rc;
                band_groups(q2.kL2, q2.kR2, ka, 0, G - 1, &L2, &R2);
                band_groups(q2.kL3, q2.kR3, ka, L2, R2, &L3, &R3);
                band_groups(q2.kL4, q2.kR4, ka, L3, R3, &L4, &R4);
                band_groups(q2.kLc, q2.kRc, ka, L4, R4, &Lc, &Rc);
                float *acc0 = &S.acc[warp][a - t0];
                float *acc = acc0 + lane;
                const float kf0 = (float)(ka + lane);
                sweep2<kBandGH1>(q2, 0, L2, R2 + 1, G, gf, rem, acc, kf0, lane);
                sweep2<kBandGH2>(q2, L2, L3, R3 + 1, R2 + 1, gf, rem, acc, kf0, lane);
                sweep2<kBandGH3>(q2, L3, L4, R4 + 1, R3 + 1, gf, rem, acc, kf0, lane);
                sweep2<kBandGH4>(q2, L4, Lc, Rc + 1, R4 + 1, gf, rem, acc, kf0, lane);
                if (Lc <= Rc)
                    sweep_core(q2, j, Lc, Rc + 1, nact, acc0, kf0, lane, a - t0, queue, qn, S,
                               warp, t0);
            }
            drain_rest(queue, qn, S, warp, lane, t0);
            if (++rounds == FLUSH_ROUNDS) {
                rounds = 0;
                __syncthreads();
                fold(S, tid);
                __syncthreads();
            }
        }
        __syncthreads();
        fold(S, tid);
        __syncthreads();
        for (int i = tid; i <= t1 - t0; i += NT) {
            const double tot = (double)S.hi[i] + (double)S.lo[i];
            if (tot != 0.0) atomicAdd(pr.acc + t0 + i, tot);
        }
        __syncthreads();
    }
}

}  // namespace f32g

int gather_f32_tile_bins() { return f32g::TILE; }

size_t gather_f32_smem() { return sizeof(f32g::Smem); }

int gather_f32_launch(const Prob *probs_d, const GridD &g, int64_t ntiles, int64_t m,
                      const int64_t *item_off, const int64_t *tile_lb, const int64_t *tile_le,
                      int lmax, unsigned long long *counter, cudaStream_t st, int num_sms)
{
    static bool configured = false;
    cudaError_t e;
    if (!configured) {
        e = cudaFuncSetAttribute(f32g::k_gather_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(f32g::Smem));
        if (e) return fail_cuda(e);
        configured = true;
    }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f32g::k_gather_f32, f32g::NT,
                                                      sizeof(f32g::Smem));
    if (e || per_sm < 1) per_sm = 1;
    f32g::k_gather_f32<<<num_sms * per_sm, f32g::NT, sizeof(f32g::Smem), st>>>(
        probs_d, g, ntiles, m, item_off, tile_lb, tile_le, lmax, counter);
    e = cudaGetLastError();
    return e ? fail_cuda(e) : HK_OK;
}

}  // namespace hk
