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
// Mapping: one warp per line (lines in nu0 order), lanes sweep the line's
// bins 32 at a time for every point k; per-line sums are FP32 and reduced
// with warp shuffles; everything across lines or points is FP64.  A warp
// owns its line for all k, so per-line gradients need no atomics; the
// per-point scalars go through shared-memory FP64 atomics and one global
// FP64 atomic per block and point.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "hk_internal.cuh"
#include "hk_launch.h"

namespace hk {

constexpr int BW_WARPS = 8;

// (Re Q, Im Q) with Q = (u + tau) / (u - tau)^2, u = z^2 = (X - Y) + i 2xy.
__device__ __forceinline__ void pair_q(float tau, float X, float Y, float b, float *re,
                                       float *im)
{
    float a = X - Y - tau;
    float c = X - Y + tau;
    float a2b2 = a * a - b * b;
    float d = a * a + b * b;
    float id2 = 1.0f / (d * d);
    *re = (c * a2b2 + 2.0f * a * b * b) * id2;
    *im = b * (a2b2 - 2.0f * a * c) * id2;
}

// V = Re w, Vx = dV/dx, Vy = dV/dy at (x, y), y >= 0.
__device__ __forceinline__ void voigt_grad(float x, float y, float *V, float *Vx, float *Vy)
{
    const float k = (float)kInvSqrtPi;
    float X = x * x, Y = y * y, r2 = X + Y;
    float b = 2.0f * x * y;
    if (r2 >= BandLimits<float>::gh2) {
        float ir2 = 1.0f / r2;
        *V = k * y * ir2;
        *Vx = -k * b * ir2 * ir2;
        *Vy = k * (X - Y) * ir2 * ir2;
        return;
    }
    if (r2 >= BandLimits<float>::core) {
        float re, im, vx = 0.0f, vy = 0.0f, F;
        if (r2 >= BandLimits<float>::gh3) {          // 2 nodes, 2W = 1
            F = gh2_F<float>(X, Y, r2);
            pair_q(0.5f, X, Y, b, &re, &im);
            vx = im;
            vy = re;
        } else if (r2 >= BandLimits<float>::gh4) {   // 3 nodes
            F = gh3_F<float>(X, Y, r2);
            pair_q(1.5f, X, Y, b, &re, &im);
            float ir2 = 1.0f / r2;
            vx = (1.0f / 3.0f) * im - (2.0f / 3.0f) * b * ir2 * ir2;
            vy = (1.0f / 3.0f) * re + (2.0f / 3.0f) * (X - Y) * ir2 * ir2;
        } else {                                     // 4 nodes
            F = gh4_F<float>(X, Y, r2);
            float re2, im2;
            pair_q(0.27525512860841106f, X, Y, b, &re, &im);
            pair_q(2.724744871391589f, X, Y, b, &re2, &im2);
            const float wa = 2.0f * 0.4541241452319315f, wb = 2.0f * 0.04587585476806851f;
            vx = wa * im + wb * im2;
            vy = wa * re + wb * re2;
        }
        *V = k * y * F;
        *Vx = k * vx;
        *Vy = k * vy;
        return;
    }
    // core: full w from the trapezoid rule with pole correction, then w'
    constexpr double w0[23] = HK_TRAP_W0;
    constexpr double w1[23] = HK_TRAP_W1;
    float ax = fabsf(x);
    float u = ax * 2.0f;
    float fr = u - floorf(u);
    bool sh = !(fr > 0.25f && fr < 0.75f);
    float off = sh ? 0.5f : 0.0f;
    float sr = 0.0f, si = 0.0f;
#pragma unroll
    for (int n = -11; n <= 11; ++n) {
        float t = ((float)n + off) * 0.5f;
        float wt = sh ? (float)w1[n + 11] : (float)w0[n + 11];
        float d = ax - t;
        float q = __fdividef(wt, d * d + Y);
        sr += q;
        si += q * d;
    }
    float re = (float)(0.5 * kInvPi) * y * sr;
    float im = (float)(0.5 * kInvPi) * si;
    if (y < 2.0f) {
        float em = expm1f((float)(4 * kPI) * y);
        float E = 1.0f + em;
        float sn, cs;
        sincospif(4.0f * ax, &sn, &cs);
        if (sh) {
            sn = -sn;
            cs = -cs;
        }
        float s2, c2;
        sincosf(2.0f * ax * y, &s2, &c2);
        float den = em * em + 2.0f * E * (1.0f - cs);
        float g = 2.0f * expf(Y - X) / den;
        re += g * (c2 * (1.0f - E * cs) - s2 * E * sn);
        im -= g * (c2 * E * sn + s2 * (1.0f - E * cs));
    }
    if (x < 0.0f) im = -im;
    *V = re;
    *Vx = -2.0f * (x * re - y * im);
    *Vy = 2.0f * (x * im + y * re) - 2.0f * k;
}

__global__ void __launch_bounds__(BW_WARPS * 32)
    k_backward(const Prob *__restrict__ probs, int nTP, GridD g, const float *__restrict__ grad,
               const double *__restrict__ kscal, double *dL_dT, double *dL_dP, double *dL_dSref,
               double *dL_dgamma, const int64_t *__restrict__ perm)
{
    extern __shared__ double s_acc[];  // [2 * nTP]: dT, dP partials of this block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < 2 * nTP; k += blockDim.x) s_acc[k] = 0.0;
    __syncthreads();
    const Prob &p0 = probs[0];
    const int64_t n = p0.n;
    for (int64_t l = (int64_t)blockIdx.x * BW_WARPS + warp; l < n;
         l += (int64_t)gridDim.x * BW_WARPS) {
        const double nu0 = p0.nu0[l];
        int i0, lo, hi;
        double r64;
        bool any = line_geometry(nu0, g, &i0, &r64, &lo, &hi);
        double gS = 0.0, gG = 0.0;
        if (any) {
            double rn;
            nearest_bin(i0, r64, &i0, &rn);
            const float r = (float)rn;
            const float nu0f = (float)nu0;
            const float E_low = p0.E_low[l], gam = p0.gamma[l], nT = p0.n_T[l];
            const float S_ref = p0.S_ref[l];
            const float nat = p0.A ? p0.A[l] * (float)p0.nat_coef : 0.0f;
            for (int k = 0; k < nTP; ++k) {
                const Prob &pk = probs[k];
                const double T = kscal[2 * k], dlnQ = kscal[2 * k + 1];
                const float aDinv = (float)pk.aD_coef / nu0f;
                const float trn = exp2f(nT * (float)pk.log2_tratio);
                const float GL = nat + gam * trn * (float)pk.press;
                const float y = GL * aDinv;
                const float bstep = (float)g.dnu * aDinv;
                const float* gk = grad + (int64_t)k * g.nbins;
                float sV = 0.0f, sXVx = 0.0f, sVy = 0.0f;
                for (int i = lo + lane; i <= hi; i += 32) {
                    const float x = ((float)(i - i0) - r) * bstep;
                    float V, Vx, Vy;
                    voigt_grad(x, y, &V, &Vx, &Vy);
                    const float gi = __ldg(gk + i);
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
                // strength pieces: ratio_base = S(T)/S_ref * alphaD_inv / sqrt(pi) * mass_scale
                const double L = (double)E_low * pk.K2;
                const double nL = rint(L);
                const float bz = exp2f((float)(L - nL));
                const float stim = expm1f(-(float)pk.c2T * nu0f) / expm1f(-(float)pk.c2Tref * nu0f);
                const float rbf = (float)pk.qratio * bz * stim * aDinv * (float)kInvSqrtPi *
                                  (float)pk.mass_scale;
                const double rb = ldexp((double)rbf, (int)nL);
                const double A = rb * (double)S_ref;
                // d ln S / dT = -dlnQ/dT + c2 E''/T^2 - (c2 nu0 / T^2) / expm1(c2 nu0 / T)
                const double c2T = pk.c2T;
                const double dlnS = -dlnQ + c2T * (double)E_low / T -
                                    (c2T * nu0 / T) / expm1(c2T * nu0);
                const double dGL_dT = -(double)nT * (double)(GL - nat) / T;
                const double dy_dT = dGL_dT * (double)aDinv - (double)y / (2.0 * T);
                const double dy_dP = (double)gam * (double)trn * pk.inv_Pref * (double)aDinv;
                const double dy_dg = (double)trn * pk.press * (double)aDinv;
                gS += rb * (double)sV;
                gG += A * (double)sVy * dy_dg;
                if (lane == 0) {
                    double dT = A * (dlnS * (double)sV - ((double)sV + (double)sXVx) / (2.0 * T) +
                                     dy_dT * (double)sVy);
                    double dP = A * (double)sVy * dy_dP;
                    atomicAdd(&s_acc[k], dT);
                    atomicAdd(&s_acc[nTP + k], dP);
                }
            }
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
