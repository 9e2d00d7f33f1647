// hk_launch.h -- host-side interfaces between the libhk translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "hk.h"
#include "hk_internal.cuh"

namespace hk {

// Records a CUDA error for hk_last_cuda_error() and returns HK_ECUDA.
int fail_cuda(cudaError_t e);

// Host arrays to device memory through kernel parameters (stream-ordered,
// capturable, no pageable-memory copy).
int upload_probs(Prob *dst, const Prob *src, int n, cudaStream_t st);
int upload_doubles(double *dst, const double *src, int n, cudaStream_t st);

// Gather (hk_gather.cu).  Tile width in bins: FP64, 512 (bpt 2 bins per
// thread); FP32C, `bpt` itself is the tile width (1024 or 2048).
int gather_tile_bins(int precision, int bpt);
// Workspace bytes of gather_run for nprob sigma arrays of nbins bins.
size_t gather_workspace(int nprob, const GridD &g, int precision, int bpt);
// Runs the Voigt sum for nprob problems.  precision 0: FP32C, out is
// float[nprob][nbins]; precision 1: FP64, out is double[nprob][nbins].
// accumulate: add into out instead of overwriting.  probs_h is modified
// (device pointers of the workspace are filled in).
// out_f64: with precision 0, write double instead of float.  status_d: the
// device status word (overflow of a float output is flagged there).
int gather_run(Prob *probs_h, int nprob, const GridD &g, int precision, int bpt, int lmax,
               void *out, int out_f64, int accumulate, char *ws, size_t ws_bytes,
               unsigned *status_d, cudaStream_t st, int num_sms);

// The per-device status word (allocated on first use).  Returns nullptr on failure.
unsigned *status_word();

// FP32-compensated line-major gather (hk_gather_f32.cu).  tile: bins per
// tile, one of the widths gather_f32_tile_ok accepts (1024, 2048).
bool gather_f32_tile_ok(int tile);
int gather_f32_launch(const Prob *probs_d, const GridD &g, int64_t ntiles, int64_t m,
                      const int64_t *item_off, const int64_t *tile_lb, const int64_t *tile_le,
                      int lmax, unsigned long long *counter, cudaStream_t st, int num_sms,
                      int tile);

// Profiling of the gather launches (hk_profile).
void gather_profile_record(cudaStream_t st, bool begin);
int gather_profile(int mode, double *ms, int64_t *launches);
// Per-line bin geometry shared by the problems of a line list (hk_gather_f32.cu).
int line_geo_launch(const Prob &p, const GridD &g, int4 *geo, cudaStream_t st, int num_sms);
// Pair and band counts (hk_count_pairs).
int count_pairs_run(const Prob &p, const GridD &g, unsigned long long *counts_d, cudaStream_t st,
                    int num_sms);

// Pipe-throughput microbenchmarks (hk_peaks.cu).  kind 0 FFMA, 1 MUFU
// reciprocal, 2 MUFU exp2, 3 DFMA; scratch: >= num_sms * 8 * 256 doubles.
int peak_launch(int kind, int iters, int num_sms, void *scratch, double *ops, cudaStream_t st);

// Adjoint (hk_backward.cu).
size_t backward_workspace(int64_t n, int nTP, int64_t nbins);
int backward_run(Prob *probs_h, int nTP, const GridD &g, const float *grad_sigma,
                 const double *dlnQ_dT, const double *T, const double *P, double *dL_dT,
                 double *dL_dP, double *dL_dSref, double *dL_dgamma, const int64_t *perm,
                 char *ws, size_t ws_bytes, cudaStream_t st, int num_sms);

}  // namespace hk
