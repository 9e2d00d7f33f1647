// hk_backward.cu -- adjoint of the cross section for retrievals.
//
// L = sum_k sum_i g_k[i] sigma_k[i] over nTP (T, P) points of one species.
// Per line l and point k (A = S alpha_D^-1 / sqrt(pi), Re w = V):
//   dL/dS_ref,l  += (A / S_ref) sum_i g V
//   dL/dgamma,l  += A (dy/dgamma) sum_i g dV/dy
//   dL/dT_k      += A [ dlnS/dT sum g V - (1/2T)(sum g V + sum g x dV/dx) + dy/dT sum g dV/dy ]
//   dL/dP_k      += A (dy/dP) sum_i g dV/dy
// with dV/dx = Re w', dV/dy = -Im w', w' = -2 z w + 2i/sqrt(pi) (Faddeeva ODE)
// and, for the Gauss-Hermite bands, the exact derivative of the quadrature
// rule.  Profiles are recomputed, never stored.
//
// Mapping: one warp per line (lines in nu0 order).  The line's per-point
// scalars (widths, strength ratio, their T and P derivatives) are computed
// once per point by one lane each (lane j for point j, 32 points at a time);
// then for every point the lanes sweep the line's bins 32 at a time, the
// per-line sums are FP32 and reduced with warp shuffles, and the lane that
// owns the point combines them with its scalars in FP64.  A warp owns its
// line for all points, so per-line gradients need no atomics; the per-point
// scalars go through shared-memory FP64 atomics and one global FP64 atomic
// per block and point.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "hk_internal.cuh"
#include "hk_launch.h"

namespace hk {

constexpr int BW_WARPS = 8;

// Q = (u + tau) / (u - tau)^2, u = z^2 = (X - Y) + i b, b = 2xy:
//   a = X - Y - tau, c = X - Y + tau, d = |u - tau|^2 = a^2 + b^2,
//   Re Q = (c (a^2 - b^2) + 2 a b^2) / d^2,  Im Q = b (a^2 - b^2 - 2 a c) / d^2;
// id2 = 1 / d^2 comes from the caller's shared reciprocal.
__device__ __forceinline__ void pair_q(float a, float c, float b, float id2, float *re,
                                       float *im)
{
    const float a2b2 = fmaf(a, a, -b * b);
    *re = fmaf(c, a2b2, 2.0f * a * b * b) * id2;
    *im = b * fmaf(-2.0f * a, c, a2b2) * id2;
}

// V = Re w, Vx = dV/dx, Vy = dV/dy at (x, y), y >= 0, float.  The Gauss-
// Hermite bands of the forward sum, differentiated exactly (w of an n-node
// rule is sum_j W_j (i/pi) / (z - t_j); its z-derivative pairs +-t_j into
// Q above), each band with one hardware reciprocal; the core takes the full
// trapezoid w and the Faddeeva ODE w' = -2 z w + 2i/sqrt(pi).
__device__ __forceinline__ void voigt_grad(float x, float y, float *V, float *Vx, float *Vy)
{
    const float k = (float)kInvSqrtPi;
    const float X = x * x, Y = y * y, r2 = X + Y;
    const float b = 2.0f * x * y;
    const float XmY = X - Y;
    if (r2 >= BandLimits<float>::gh2) {              // 1 node
        const float ir2 = rcp_ftz(r2);
        const float ky = k * ir2, ky2 = ky * ir2;
        *V = y * ky;
        *Vx = -b * ky2;
        *Vy = XmY * ky2;
        return;
    }
    if (r2 >= BandLimits<float>::gh3) {              // 2 nodes, tau = 1/2, 2W = 1
        const float a = XmY - 0.5f, c = XmY + 0.5f;
        const float d = fmaf(a, a, b * b);
        const float id = rcp_ftz(d);
        float re, im;
        pair_q(a, c, b, id * id, &re, &im);
        *V = k * y * (r2 + 0.5f) * id;
        *Vx = k * im;
        *Vy = k * re;
        return;
    }
    if (r2 >= BandLimits<float>::gh4) {              // 3 nodes: 0 (W0 = 2/3), tau = 3/2 (W = 1/6 each)
        const float a = XmY - 1.5f, c = XmY + 1.5f;
        const float d = fmaf(a, a, b * b);
        const float ird = rcp_ftz(r2 * d);
        const float id = r2 * ird, ir2 = d * ird;
        float re, im;
        pair_q(a, c, b, id * id, &re, &im);
        const float F = fmaf(2.0f / 3.0f, ir2, (1.0f / 3.0f) * (r2 + 1.5f) * id);
        const float ir22 = ir2 * ir2;
        *V = k * y * F;
        *Vx = k * fmaf(1.0f / 3.0f, im, -(2.0f / 3.0f) * b * ir22);
        *Vy = k * fmaf(1.0f / 3.0f, re, (2.0f / 3.0f) * XmY * ir22);
        return;
    }
    if (r2 >= BandLimits<float>::core) {             // 4 nodes
        const float ta = 0.27525512860841106f, tb = 2.724744871391589f;
        const float wa = 2.0f * 0.4541241452319315f, wb = 2.0f * 0.04587585476806851f;
        const float a1 = XmY - ta, c1 = XmY + ta, a2 = XmY - tb, c2 = XmY + tb;
        const float b2 = b * b;
        const float d1 = fmaf(a1, a1, b2), d2 = fmaf(a2, a2, b2);
        const float idd = rcp_ftz(d1 * d2);
        const float id1 = d2 * idd, id2 = d1 * idd;
        float re1, im1, re2, im2;
        pair_q(a1, c1, b, id1 * id1, &re1, &im1);
        pair_q(a2, c2, b, id2 * id2, &re2, &im2);
        const float F = fmaf(wa * (r2 + ta), id1, wb * (r2 + tb) * id2);
        *V = k * y * F;
        *Vx = k * fmaf(wa, im1, wb * im2);
        *Vy = k * fmaf(wa, re1, wb * re2);
        return;
    }
    // core: full w from the trapezoid rule with pole correction, then w'
    constexpr double w0[23] = HK_TRAP_W0;
    constexpr double w1[23] = HK_TRAP_W1;
    const float ax = fabsf(x);
    const float u = ax * 2.0f;
    const float fr = u - floorf(u);
    const bool sh = !(fr > 0.25f && fr < 0.75f);
    const float off = sh ? 0.5f : 0.0f;
    float sr = 0.0f, si = 0.0f;
#pragma unroll
    for (int n = -11; n <= 11; ++n) {
        const float t = ((float)n + off) * 0.5f;
        const float wt = sh ? (float)w1[n + 11] : (float)w0[n + 11];
        const float d = ax - t;
        const float q = wt * rcp_ftz(fmaf(d, d, Y));
        sr += q;
        si = fmaf(q, d, si);
    }
    float re = (float)(0.5 * kInvPi) * y * sr;
    float im = (float)(0.5 * kInvPi) * si;
    if (y < 2.0f) {
        const float em = expm1f((float)(4 * kPI) * y);
        const float E = 1.0f + em;
        float sn, cs;
        sincospi_core(4.0f * ax, &sn, &cs);
        if (sh) {
            sn = -sn;
            cs = -cs;
        }
        float s2, c2;
        sincos_core(2.0f * ax * y, &s2, &c2);
        const float den = em * em + 2.0f * E * (1.0f - cs);
        const float gg = 2.0f * expf(Y - X) * rcp_ftz(den);
        re += gg * (c2 * (1.0f - E * cs) - s2 * E * sn);
        im -= gg * (c2 * E * sn + s2 * (1.0f - E * cs));
    }
    if (x < 0.0f) im = -im;
    *V = re;
    *Vx = -2.0f * (x * re - y * im);
    *Vy = 2.0f * (x * im + y * re) - 2.0f * k;
}

// Per (line, point) scalars, computed by one lane per point (the FP64 ones
// wait in shared memory while the warp sweeps the bins).
struct PointScal {
    float y, bstep;                 // Gamma_L / alpha_D, dnu / alpha_D
    double rb;                      // S(T) / S_ref * alpha_D^-1 / sqrt(pi) * mass_scale
    double dlnS, dy_dT, dy_dP, dy_dg, T;
};
struct PointScalD {
    double rb, dlnS, dy_dT, dy_dP, dy_dg, T;
};

__device__ __forceinline__ void point_scalars(const Prob &pk, const GridD &g, double T,
                                              double dlnQ, double nu0, float nu0f, float E_low,
                                              float gam, float nT, float nat, PointScal *o)
{
    const float aDinv = pk.aD_coef_f / nu0f;
    const float trn = exp2f(nT * pk.log2_tratio_f);
    const float GL = nat + gam * trn * pk.press_f;
    o->y = GL * aDinv;
    o->bstep = (float)g.dnu * aDinv;
    // strength ratio as in the forward: Boltzmann exponent as a float pair
    const float Lh = E_low * pk.K2_hi;
    const float Ll = fmaf(E_low, pk.K2_lo, fmaf(E_low, pk.K2_hi, -Lh));
    const float nL = rintf(Lh);
    const float bz = exp2f((Lh - nL) + Ll);
    const float stim = expm1f(-pk.c2T_f * nu0f) / expm1f(-pk.c2Tref_f * nu0f);
    const float rbf = pk.qratio_f * bz * stim * aDinv * (float)kInvSqrtPi * pk.mass_scale_f;
    o->rb = ldexp((double)rbf, (int)nL);
    // d ln S / dT = -dlnQ/dT + c2 E''/T^2 - (c2 nu0 / T^2) / expm1(c2 nu0 / T)
    const double c2T = pk.c2T;
    o->dlnS = -dlnQ + c2T * (double)E_low / T - (c2T * nu0 / T) / expm1(c2T * nu0);
    const double dGL_dT = -(double)nT * (double)(GL - nat) / T;
    o->dy_dT = dGL_dT * (double)aDinv - (double)o->y / (2.0 * T);
    o->dy_dP = (double)gam * (double)trn * pk.inv_Pref * (double)aDinv;
    o->dy_dg = (double)trn * pk.press * (double)aDinv;
    o->T = T;
}

__global__ void __launch_bounds__(BW_WARPS * 32, 4)
    k_backward(const Prob *__restrict__ probs, int nTP, GridD g, const float *__restrict__ grad,
               const double *__restrict__ kscal, double *dL_dT, double *dL_dP, double *dL_dSref,
               double *dL_dgamma, const int64_t *__restrict__ perm)
{
    extern __shared__ double s_acc[];  // [2 * nTP]: dT, dP partials of this block
    __shared__ PointScalD s_pt[BW_WARPS][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < 2 * nTP; k += blockDim.x) s_acc[k] = 0.0;
    __syncthreads();
    const Prob &p0 = probs[0];
    const int64_t n = p0.n;
    for (int64_t l = (int64_t)blockIdx.x * BW_WARPS + warp; l < n;
         l += (int64_t)gridDim.x * BW_WARPS) {
        const double nu0 = p0.nu0[l];
        int c, lo, hi;
        float rn;
        const bool any =
            line_geometry_f32(line_pos(p0, l), g, line_cut(p0, g, l, nu0), &c, &rn, &lo, &hi);
        double gS = 0.0, gG = 0.0;   // this lane's share of the line's gradients
        if (any) {
            const float nu0f = (float)nu0;
            const float E_low = p0.E_low[l], gam = p0.gamma[l], nT = p0.n_T[l];
            const float S_ref = p0.S_ref[l];
            const float nat = p0.A ? p0.A[l] * p0.nat_coef_f : 0.0f;
            const float k0 = (float)(lo - c);
            for (int kc = 0; kc < nTP; kc += 32) {
                const int npt = min(32, nTP - kc);
                // lane j: the scalars of point kc + j
                float py = 1.0f, pb = 0.0f;
                if (lane < npt) {
                    const int kk = kc + lane;
                    PointScal ps;
                    point_scalars(probs[kk], g, kscal[2 * kk], kscal[2 * kk + 1], nu0, nu0f,
                                  E_low, gam, nT, nat, &ps);
                    py = ps.y;
                    pb = ps.bstep;
                    s_pt[warp][lane] = PointScalD{ps.rb, ps.dlnS, ps.dy_dT, ps.dy_dP, ps.dy_dg, ps.T};
                }
                float mV = 0.0f, mXVx = 0.0f, mVy = 0.0f;   // sums of this lane's point
                for (int j = 0; j < npt; ++j) {
                    const float y = __shfl_sync(0xffffffffu, py, j);
                    const float bstep = __shfl_sync(0xffffffffu, pb, j);
                    const float rnb = rn * bstep;
                    const float *gk = grad + (int64_t)(kc + j) * g.nbins;
                    float sV = 0.0f, sXVx = 0.0f, sVy = 0.0f;
                    float kf = k0 + (float)lane;
                    int i = lo + lane;
                    // four bins per lane and step, their upstream-gradient loads
                    // issued before any profile work (the loop is load-latency bound)
                    for (; i + 96 <= hi; i += 128, kf += 128.0f) {
                        float gv[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) gv[u] = __ldg(gk + i + 32 * u);
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const float x = fmaf(kf + 32.0f * u, bstep, -rnb);
                            float V, Vx, Vy;
                            voigt_grad(x, y, &V, &Vx, &Vy);
                            sV = fmaf(gv[u], V, sV);
                            sXVx = fmaf(gv[u] * x, Vx, sXVx);
                            sVy = fmaf(gv[u], Vy, sVy);
                        }
                    }
                    for (; i <= hi; i += 32, kf += 32.0f) {
                        const float gi = __ldg(gk + i);
                        const float x = fmaf(kf, bstep, -rnb);
                        float V, Vx, Vy;
                        voigt_grad(x, y, &V, &Vx, &Vy);
                        sV = fmaf(gi, V, sV);
                        sXVx = fmaf(gi * x, Vx, sXVx);
                        sVy = fmaf(gi, Vy, sVy);
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        sV += __shfl_xor_sync(0xffffffffu, sV, o);
                        sXVx += __shfl_xor_sync(0xffffffffu, sXVx, o);
                        sVy += __shfl_xor_sync(0xffffffffu, sVy, o);
                    }
                    if (lane == j) {
                        mV = sV;
                        mXVx = sXVx;
                        mVy = sVy;
                    }
                }
                if (lane < npt) {
                    const PointScalD ps = s_pt[warp][lane];
                    const double A = ps.rb * (double)S_ref;
                    const double V = mV, XVx = mXVx, Vy = mVy;
                    gS += ps.rb * V;
                    gG += A * Vy * ps.dy_dg;
                    const double dT = A * (ps.dlnS * V - (V + XVx) / (2.0 * ps.T) + ps.dy_dT * Vy);
                    const double dP = A * Vy * ps.dy_dP;
                    atomicAdd(&s_acc[kc + lane], dT);
                    atomicAdd(&s_acc[nTP + kc + lane], dP);
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            gS += __shfl_xor_sync(0xffffffffu, gS, o);
            gG += __shfl_xor_sync(0xffffffffu, gG, o);
        }
        if (lane == 0) {
            int64_t o = perm ? perm[l] : l;
            dL_dSref[o] = gS;
            dL_dgamma[o] = gG;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nTP; k += blockDim.x) {
        if (s_acc[k] != 0.0) atomicAdd(&dL_dT[k], s_acc[k]);
        if (s_acc[nTP + k] != 0.0) atomicAdd(&dL_dP[k], s_acc[nTP + k]);
    }
}

size_t backward_workspace(int64_t n, int nTP, int64_t nbins)
{
    (void)n;
    (void)nbins;
    return ((sizeof(Prob) * nTP + 255) & ~(size_t)255) +
           ((sizeof(double) * 2 * nTP + 255) & ~(size_t)255);
}

int backward_run(Prob *probs_h, int nTP, const GridD &g, const float *grad_sigma,
                 const double *dlnQ_dT, const double *T, const double *P, double *dL_dT,
                 double *dL_dP, double *dL_dSref, double *dL_dgamma, const int64_t *perm,
                 char *ws, size_t ws_bytes, cudaStream_t st, int num_sms)
{
    (void)P;
    if (backward_workspace(probs_h[0].n, nTP, g.nbins) > ws_bytes) return HK_ENOMEM;
    if ((size_t)nTP * 2 * sizeof(double) > 48 * 1024) return HK_ENOTSUP;
    Prob *probs_d = (Prob *)ws;
    double *kscal = (double *)(ws + ((sizeof(Prob) * nTP + 255) & ~(size_t)255));
    // kscal[2k] = T, kscal[2k+1] = dlnQ/dT
    std::vector<double> hs(2 * (size_t)nTP);
    for (int k = 0; k < nTP; ++k) {
        hs[2 * k] = T[k];
        hs[2 * k + 1] = dlnQ_dT[k];
    }
    cudaError_t e;
    int urc = upload_probs(probs_d, probs_h, nTP, st);
    if (!urc) urc = upload_doubles(kscal, hs.data(), 2 * nTP, st);
    if (urc) return urc;
    if ((e = cudaMemsetAsync(dL_dT, 0, sizeof(double) * nTP, st))) return fail_cuda(e);
    if ((e = cudaMemsetAsync(dL_dP, 0, sizeof(double) * nTP, st))) return fail_cuda(e);
    int64_t n = probs_h[0].n;
    if (n == 0) return HK_OK;
    int64_t blocks = (n + BW_WARPS - 1) / BW_WARPS;
    int64_t cap = (int64_t)num_sms * 8;
    if (blocks > cap) blocks = cap;
    size_t shm = sizeof(double) * 2 * nTP;
    k_backward<<<(unsigned)blocks, BW_WARPS * 32, shm, st>>>(probs_d, nTP, g, grad_sigma, kscal,
                                                            dL_dT, dL_dP, dL_dSref, dL_dgamma,
                                                            perm);
    if ((e = cudaGetLastError())) return fail_cuda(e);
    return HK_OK;
}

}  // namespace hk
