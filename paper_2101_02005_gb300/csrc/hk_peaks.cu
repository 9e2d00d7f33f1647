// hk_peaks.cu -- throughput microbenchmarks of the pipes the Voigt kernels
// run on (FP32 FMA, scalar and packed FP32x2, the MUFU reciprocal and exp2,
// FP64 FMA), so that their
// rooflines are stated against measured peaks of this GPU rather than
// nominal unit counts.
//
// Each thread runs NCH independent dependency chains of one operation, so the
// pipe, not the latency of a chain, sets the rate; the grid fills every SM
// (8 blocks of 256 threads per SM).  The chains stay bounded (fixed points of
// the iterated maps), and a test no value can pass keeps the compiler from
// removing them.
#include <cuda_runtime.h>

#include <cstdint>

#include "hk_internal.cuh"
#include "hk_launch.h"

namespace hk {

namespace peaks {

constexpr int NT = 256;
constexpr int NCH = 8;      // independent chains per thread
constexpr int UNROLL = 16;  // operations per chain per loop iteration

__device__ __forceinline__ float ex2_approx(float a)
{
    float r;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}

__device__ __forceinline__ float rcp_approx(float a)
{
    float r;
    asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}

// KIND 0: FFMA a = a m + c.  1: MUFU reciprocal a = 1/a + 1/2.  2: MUFU exp2
// a = 2^a - 3/2.  The FADD after each MUFU op keeps consecutive operations
// from cancelling (1/(1/a) = a) and costs the FMA pipe a small share of what
// the MUFU pipe spends.
template <int KIND> __global__ void __launch_bounds__(NT) k_peak_f32(float *out, int iters, float seed)
{
    float a[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) a[c] = seed + 0.01f * (float)(threadIdx.x + c);
    const float m = 0.9999f, k = 1e-5f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                if (KIND == 0) a[c] = fmaf(a[c], m, k);
                else if (KIND == 1) a[c] = rcp_approx(a[c]) + 0.5f;
                else a[c] = ex2_approx(a[c]) - 1.5f;
            }
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < NCH; ++c) s += a[c];
    if (s == -12345.678f) out[blockIdx.x * NT + threadIdx.x] = s;
}

// Packed FP32x2 FMA (sm_100 and later: one instruction, two FMAs per lane):
// a = a m + c on both halves of NCH register pairs.
__global__ void __launch_bounds__(NT) k_peak_f32x2(float *out, int iters, float seed)
{
    float2 a[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c)
        a[c] = make_float2(seed + 0.01f * (float)(threadIdx.x + c), seed - 0.01f * (float)c);
    const float2 m = make_float2(0.9999f, 0.9998f), k = make_float2(1e-5f, 2e-5f);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
#pragma unroll
            for (int c = 0; c < NCH; ++c) a[c] = __ffma2_rn(a[c], m, k);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < NCH; ++c) s += a[c].x + a[c].y;
    if (s == -12345.678f) out[blockIdx.x * NT + threadIdx.x] = s;
}

__global__ void __launch_bounds__(NT) k_peak_f64(double *out, int iters, double seed)
{
    double a[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) a[c] = seed + 0.01 * (double)(threadIdx.x + c);
    const double m = 0.9999, k = 1e-5;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
#pragma unroll
            for (int c = 0; c < NCH; ++c) a[c] = fma(a[c], m, k);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < NCH; ++c) s += a[c];
    if (s == -12345.678) out[blockIdx.x * NT + threadIdx.x] = s;
}

}  // namespace peaks

// Launches one microbenchmark; *ops = operations it performs (FMA counted
// once).
int peak_launch(int kind, int iters, int num_sms, void *scratch, double *ops, cudaStream_t st)
{
    const int blocks = num_sms * 8;
    *ops = (double)blocks * peaks::NT * iters * peaks::UNROLL * peaks::NCH;
    switch (kind) {
    case 0:
        peaks::k_peak_f32<0><<<blocks, peaks::NT, 0, st>>>((float *)scratch, iters, 0.5f);
        break;
    case 1:
        peaks::k_peak_f32<1><<<blocks, peaks::NT, 0, st>>>((float *)scratch, iters, 0.5f);
        break;
    case 2:
        peaks::k_peak_f32<2><<<blocks, peaks::NT, 0, st>>>((float *)scratch, iters, 0.5f);
        break;
    case 3:
        peaks::k_peak_f64<<<blocks, peaks::NT, 0, st>>>((double *)scratch, iters, 0.5);
        break;
    case 4:   // two FMAs per lane and instruction
        *ops *= 2.0;
        peaks::k_peak_f32x2<<<blocks, peaks::NT, 0, st>>>((float *)scratch, iters, 0.5f);
        break;
    default:
        return HK_EINVAL;
    }
    cudaError_t e = cudaGetLastError();
    return e ? fail_cuda(e) : HK_OK;
}

}  // namespace hk
