// hk_api.cu -- the C ABI of libhk (declared in include/hk.h): argument
// checks, scalar preparation in FP64, the scratch pool, the optional sort of
// unsorted line lists, and the small per-line kernels.
#include <cuda_runtime.h>

#include <cub/cub.cuh>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "hk_internal.cuh"
#include "hk_launch.h"

namespace hk {

static thread_local int g_last_cuda = 0;

int fail_cuda(cudaError_t e)
{
    g_last_cuda = (int)e;
    (void)cudaGetLastError();  // clear a non-sticky launch error
    return HK_ECUDA;
}

// ---- scratch pool: one grow-only device buffer per device -----------------
struct Pool {
    char *ptr = nullptr;
    size_t cap = 0;
};
static std::mutex g_pool_mu;
static std::map<int, Pool> g_pools;

static size_t pool_limit()
{
    const char *s = getenv("HK_POOL_LIMIT_MB");
    double mb = s ? atof(s) : 16384.0;
    if (!(mb > 0)) mb = 16384.0;
    return (size_t)(mb * 1048576.0);
}

// Returns HK_OK and a buffer of at least `bytes`, or HK_ENOMEM.
static int pool_get(size_t bytes, char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return fail_cuda(e);
    std::lock_guard<std::mutex> lk(g_pool_mu);
    Pool &p = g_pools[dev];
    if (bytes > p.cap) {
        if (bytes > pool_limit()) return HK_ENOMEM;
        if (p.ptr) {
            // cudaFree waits for work in flight on the device that may still use it
            cudaFree(p.ptr);
            p.ptr = nullptr;
            p.cap = 0;
        }
        size_t want = std::max(bytes, (size_t)64 << 20);
        want = std::min(std::max(want, bytes + bytes / 4), std::max(pool_limit(), bytes));
        if (cudaMalloc(&p.ptr, want) != cudaSuccess) {
            (void)cudaGetLastError();
            if (cudaMalloc(&p.ptr, bytes) != cudaSuccess) {
                (void)cudaGetLastError();
                p.ptr = nullptr;
                return HK_ENOMEM;
            }
            want = bytes;
        }
        p.cap = want;
    }
    *out = p.ptr;
    return HK_OK;
}

// ---- per-device status word ---------------------------------------------------
static std::mutex g_status_mu;
static std::map<int, unsigned *> g_status;

unsigned *status_word()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_status_mu);
    auto it = g_status.find(dev);
    if (it != g_status.end()) return it->second;
    unsigned *p = nullptr;
    if (cudaMalloc(&p, sizeof(unsigned)) != cudaSuccess || cudaMemset(p, 0, sizeof(unsigned)) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    g_status[dev] = p;
    return p;
}

static int num_sms()
{
    static std::mutex mu;
    static std::map<int, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
        (void)cudaGetLastError();
        n = 148;
    }
    cache[dev] = n;
    return n;
}

// ---- tuning cache (hk_autotune) --------------------------------------------
struct Tune {
    int bpt = 4;        // FP64: bins per thread; FP32C: tile width in bins
    int lmax = 16384;   // lines per work item
};
static std::mutex g_tune_mu;
static std::map<std::pair<int, int>, Tune> g_tune;  // (device, precision) -> tuning

static Tune get_tune(int precision)
{
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find({dev, precision});
    if (it != g_tune.end()) return it->second;
    Tune t;
    if (precision == HK_FP64) {
        t.bpt = 2;
    } else {
        t.bpt = 1024;
        t.lmax = 2048;
    }
    return t;
}

// ---- validation ------------------------------------------------------------
static bool finite_pos(double v) { return std::isfinite(v) && v > 0; }

static int check_lines(const hk_lines *L, bool need_fields)
{
    if (!L || L->n < 0) return HK_EINVAL;
    if (L->n == 0) return HK_OK;
    if (!L->nu0 || !finite_pos(L->mass_amu)) return HK_EINVAL;
    if (L->s_mode != HK_S_REF && L->s_mode != HK_S_EINSTEIN_A) return HK_EINVAL;
    if (!need_fields) return HK_OK;
    if (!L->E_low || !L->gamma_ref || !L->n_T) return HK_EINVAL;
    if (L->s_mode == HK_S_REF && !L->S_ref) return HK_EINVAL;
    if (L->s_mode == HK_S_EINSTEIN_A && (!L->A || !L->g_up)) return HK_EINVAL;
    return HK_OK;
}

static int check_grid(const hk_grid *g)
{
    if (!g || g->nbins <= 0 || g->nbins > 2000000000LL || !finite_pos(g->dnu) ||
        !std::isfinite(g->nu_min))
        return HK_EINVAL;
    return HK_OK;
}

static int check_state(const hk_state *s)
{
    if (!s || !finite_pos(s->T) || !std::isfinite(s->P) || s->P < 0 || !finite_pos(s->Q_T) ||
        !std::isfinite(s->dlnQ_dT) || !std::isfinite(s->P_self) || s->P_self < 0)
        return HK_EINVAL;
    return HK_OK;
}

static int check_opts(const hk_opts *o)
{
    if (!o || !finite_pos(o->T_ref) || !finite_pos(o->P_ref) || !finite_pos(o->Q_Tref) ||
        !std::isfinite(o->cut))
        return HK_EINVAL;
    if (o->cut_mode != HK_CUT_FIXED && o->cut_mode != HK_CUT_NONE &&
        o->cut_mode != HK_CUT_DOPPLER && o->cut_mode != HK_CUT_LORENTZ)
        return HK_EINVAL;
    if ((o->cut_mode == HK_CUT_DOPPLER || o->cut_mode == HK_CUT_LORENTZ) && !(o->cut > 0.0))
        return HK_EINVAL;
    if (o->precision != HK_FP32C && o->precision != HK_FP64) return HK_EINVAL;
    if (o->flags & ~(HK_PER_GRAM | HK_SIGMA_F64 | HK_REMOVE_PLINTH)) return HK_EINVAL;
    if (o->profile < HK_PROFILE_VOIGT || o->profile > HK_PROFILE_BINNED_GAUSS) return HK_EINVAL;
    return HK_OK;
}
static_assert(kCutFixed == HK_CUT_FIXED && kCutNone == HK_CUT_NONE &&
                  kCutDoppler == HK_CUT_DOPPLER && kCutLorentz == HK_CUT_LORENTZ,
              "cut mode values");
static_assert(kProfVoigt == HK_PROFILE_VOIGT && kProfLorentz == HK_PROFILE_LORENTZ &&
                  kProfDoppler == HK_PROFILE_DOPPLER && kProfBinned == HK_PROFILE_BINNED_GAUSS,
              "profile values");

// The FP32 fast path of the cut bounds: W = Wi + Wf for 0 < W < 2^30.
static void set_cut_split(GridD *d)
{
    if (d->W > 0.0 && d->W < 1073741824.0) {
        d->Wi = (int)std::floor(d->W);
        d->Wf = (float)(d->W - (double)d->Wi);
    } else {
        d->Wi = -1;
        d->Wf = 0.0f;
    }
}

static GridD make_grid(const hk_grid *g, const hk_opts *o)
{
    GridD d;
    d.nu_min = g->nu_min;
    d.dnu = g->dnu;
    d.inv_dnu = 1.0 / g->dnu;
    d.nbins = g->nbins;
    const int mode = o ? o->cut_mode : HK_CUT_NONE;
    const bool perline = mode == HK_CUT_DOPPLER || mode == HK_CUT_LORENTZ;
    bool nocut = mode == HK_CUT_NONE || perline;   // no fixed cut
    d.cut = nocut ? 0.0 : o->cut;
    d.W = (d.cut > 0.0) ? d.cut * d.inv_dnu : 0.0;
    if (d.cut <= 0.0) d.cut = 0.0;
    set_cut_split(&d);
    d.cut_mode = d.W > 0.0 ? HK_CUT_FIXED : (perline ? mode : HK_CUT_NONE);
    d.cut_factor = perline ? o->cut : 0.0;
    d.plinth = (o && (o->flags & HK_REMOVE_PLINTH)) ? 1 : 0;
    d.profile = o ? o->profile : HK_PROFILE_VOIGT;
    d.halo = 0;
    return d;
}

static GridD make_grid_cut(const hk_grid *g, double cut)
{
    GridD d;
    d.nu_min = g->nu_min;
    d.dnu = g->dnu;
    d.inv_dnu = 1.0 / g->dnu;
    d.nbins = g->nbins;
    d.cut = cut > 0.0 ? cut : 0.0;
    d.W = cut > 0.0 ? cut * d.inv_dnu : 0.0;
    set_cut_split(&d);
    d.cut_mode = d.W > 0.0 ? HK_CUT_FIXED : HK_CUT_NONE;
    d.cut_factor = 0.0;
    d.plinth = 0;
    d.profile = HK_PROFILE_VOIGT;
    d.halo = 0;
    return d;
}

// Float copies of a problem's scalars (the FP32 strength uses only these).
static void set_f32_scalars(Prob *p)
{
    p->qratio_f = (float)p->qratio;
    p->c2T_f = (float)p->c2T;
    p->c2Tref_f = (float)p->c2Tref;
    p->mass_scale_f = (float)p->mass_scale;
    p->aD_coef_f = (float)p->aD_coef;
    p->log2_tratio_f = (float)p->log2_tratio;
    p->press_f = (float)p->press;
    p->nat_coef_f = (float)p->nat_coef;
    p->press_air_f = (float)p->press_air;
    p->press_self_f = (float)p->press_self;
    p->K2_hi = (float)p->K2;
    p->K2_lo = (float)(p->K2 - (double)p->K2_hi);
}

// FP64 scalars of one (species, T, P) problem.
static Prob make_prob(const hk_lines *L, const hk_state *s, const hk_opts *o)
{
    Prob p;
    memset(&p, 0, sizeof(p));
    p.nu0 = L->nu0;
    p.S_ref = L->S_ref;
    p.A = L->A;
    p.g_up = L->g_up;
    p.E_low = L->E_low;
    p.gamma = L->gamma_ref;
    p.n_T = L->n_T;
    p.n = L->n;
    p.s_mode = L->s_mode;
    p.pre = 0;
    const double T = s->T;
    if (L->s_mode == HK_S_REF) {
        p.K2 = -kC2 * (1.0 / T - 1.0 / o->T_ref) * kInvLn2;
        p.qratio = o->Q_Tref / s->Q_T;
    } else {
        p.K2 = -kC2 / T * kInvLn2;
        p.qratio = 1.0 / (8.0 * kPI * kC * s->Q_T);
    }
    p.c2T = kC2 / T;
    p.c2Tref = kC2 / o->T_ref;
    const double m_g = L->mass_amu * kAMU;
    p.mass_scale = (o->flags & HK_PER_GRAM) ? 1.0 / m_g : 1.0;
    p.aD_coef = kC * std::sqrt(m_g / (2.0 * kKB * T));
    p.log2_tratio = std::log2(o->T_ref / T);
    p.press = s->P / o->P_ref;
    p.inv_Pref = 1.0 / o->P_ref;
    p.nat_coef = 1.0 / (4.0 * kPI * kC);
    p.tratio = o->T_ref / T;
    p.gamma_self = L->gamma_self;
    p.delta = L->delta;
    p.press_air = (s->P - s->P_self) / o->P_ref;
    p.press_self = s->P_self / o->P_ref;
    // the same operations, in the same order, as the oracle's Doppler cut width
    p.K_D = std::sqrt(0.6931471805599453) * std::sqrt(2.0 * kKB * T / m_g) / kC;
    set_f32_scalars(&p);
    return p;
}

// ---- small per-line kernels -------------------------------------------------
__global__ void k_strength(Prob p, double *S_out)
{
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < p.n;
         l += (int64_t)gridDim.x * blockDim.x) {
        double S, aDinv, y;
        line_strength_f64(p, l, &S, &aDinv, &y);
        S_out[l] = S;
    }
}

__global__ void k_widths(Prob p, float *aDinv_out, float *y_out)
{
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < p.n;
         l += (int64_t)gridDim.x * blockDim.x) {
        double S, aDinv, y;
        line_strength_f64(p, l, &S, &aDinv, &y);
        aDinv_out[l] = (float)aDinv;
        y_out[l] = (float)y;
    }
}

// Sort support: order-preserving 64-bit keys of the nu0 doubles.
__global__ void k_sort_keys(const double *nu0, int64_t n, unsigned long long *keys, int64_t *idx)
{
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n;
         l += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long b = (unsigned long long)__double_as_longlong(nu0[l]);
        keys[l] = (b >> 63) ? ~b : (b | 0x8000000000000000ull);
        idx[l] = l;
    }
}

__global__ void k_gather_fields(const hk_lines L, const int64_t *perm, int64_t n, double *nu0,
                                float *S_ref, float *A, float *g_up, float *E_low, float *gamma,
                                float *n_T, float *gamma_self, float *delta)
{
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n;
         l += (int64_t)gridDim.x * blockDim.x) {
        int64_t s = perm[l];
        nu0[l] = L.nu0[s];
        if (L.S_ref) S_ref[l] = L.S_ref[s];
        if (L.A) A[l] = L.A[s];
        if (L.g_up) g_up[l] = L.g_up[s];
        E_low[l] = L.E_low[s];
        gamma[l] = L.gamma_ref[s];
        n_T[l] = L.n_T[s];
        if (L.gamma_self) gamma_self[l] = L.gamma_self[s];
        if (L.delta) delta[l] = L.delta[s];
    }
}

static inline size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

// Bytes needed to hold a sorted copy of a line list (plus the permutation).
size_t sort_bytes(int64_t n, size_t *cub_bytes)
{
    size_t tb = 0;
    cub::DeviceRadixSort::SortPairs((void *)nullptr, tb, (const unsigned long long *)nullptr,
                                    (unsigned long long *)nullptr, (const int64_t *)nullptr,
                                    (int64_t *)nullptr, (int64_t)n, 0, 64, (cudaStream_t)0);
    *cub_bytes = tb;
    return al(tb) + 2 * al(n * 8) + 2 * al(n * 8) + al(n * 8) + 8 * al(n * 4);
}

// Builds a sorted copy of `L` in `ws`; fills `S` with device pointers into ws and
// `perm_out` with sorted-position -> original-index.
int sort_lines(const hk_lines *L, char *ws, hk_lines *S, int64_t **perm_out, cudaStream_t st)
{
    int64_t n = L->n;
    size_t tb;
    sort_bytes(n, &tb);
    char *cur = ws;
    auto take = [&](size_t b) {
        char *r = cur;
        cur += al(b);
        return r;
    };
    void *temp = take(tb);
    auto *k_in = (unsigned long long *)take(n * 8), *k_out = (unsigned long long *)take(n * 8);
    auto *i_in = (int64_t *)take(n * 8), *i_out = (int64_t *)take(n * 8);
    auto *nu0 = (double *)take(n * 8);
    auto *S_ref = (float *)take(n * 4), *A = (float *)take(n * 4), *g_up = (float *)take(n * 4);
    auto *E = (float *)take(n * 4), *gam = (float *)take(n * 4), *nT = (float *)take(n * 4);
    auto *gself = (float *)take(n * 4), *dlt = (float *)take(n * 4);
    int sms = num_sms();
    k_sort_keys<<<sms * 4, 256, 0, st>>>(L->nu0, n, k_in, i_in);
    cudaError_t e = cudaGetLastError();
    if (e) return fail_cuda(e);
    e = cub::DeviceRadixSort::SortPairs(temp, tb, k_in, k_out, i_in, i_out, n, 0, 64, st);
    if (e) return fail_cuda(e);
    k_gather_fields<<<sms * 4, 256, 0, st>>>(*L, i_out, n, nu0, S_ref, A, g_up, E, gam, nT,
                                             gself, dlt);
    if ((e = cudaGetLastError())) return fail_cuda(e);
    *S = *L;
    S->nu0 = nu0;
    S->S_ref = L->S_ref ? S_ref : nullptr;
    S->A = L->A ? A : nullptr;
    S->g_up = L->g_up ? g_up : nullptr;
    S->E_low = E;
    S->gamma_ref = gam;
    S->n_T = nT;
    S->gamma_self = L->gamma_self ? gself : nullptr;
    S->delta = L->delta ? dlt : nullptr;
    S->sorted = 1;
    *perm_out = i_out;
    return HK_OK;
}

}  // namespace hk

using namespace hk;

// ============================================================================
extern "C" {

int hk_version(void) { return 100; }

const char *hk_strerror(int s)
{
    switch (s) {
    case HK_OK: return "ok";
    case HK_EINVAL: return "invalid argument";
    case HK_ENOMEM: return "scratch pool or workspace too small";
    case HK_ECUDA: return "CUDA error";
    case HK_ETIMEOUT: return "bounded device wait gave up";
    case HK_ENOTSUP: return "unsupported combination of options";
    case HK_ERANGE: return "a float sigma output overflowed (use HK_SIGMA_F64)";
    case HK_ESIZE: return "grid too large for the fixed scratch of hk_cross_section_noalloc";
    default: return "unknown status";
    }
}

int hk_last_cuda_error(void) { return g_last_cuda; }

int hk_constants(double *out6)
{
    if (!out6) return HK_EINVAL;
    out6[0] = kC;
    out6[1] = kKB;
    out6[2] = kH;
    out6[3] = kAMU;
    out6[4] = kC2;
    out6[5] = kPI;
    return HK_OK;
}

int hk_release(void)
{
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_pools.find(dev);
    if (it != g_pools.end()) {
        if (it->second.ptr) {
            cudaError_t e = cudaFree(it->second.ptr);
            if (e) return fail_cuda(e);
        }
        g_pools.erase(it);
    }
    return HK_OK;
}

int hk_count_pairs(const hk_lines *lines, const hk_grid *grid, const hk_state *state,
                   const hk_opts *opts, int64_t *counts, void *stream)
{
    int rc;
    if ((rc = check_lines(lines, true)) || (rc = check_grid(grid)) || (rc = check_state(state)) ||
        (rc = check_opts(opts)))
        return rc;
    if (!counts) return HK_EINVAL;
    for (int t = 0; t < 6; ++t) counts[t] = 0;
    if (lines->n == 0) return HK_OK;
    char *ws;
    if ((rc = pool_get(256, &ws))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Prob p = make_prob(lines, state, opts);
    GridD g = make_grid(grid, opts);
    if ((rc = count_pairs_run(p, g, (unsigned long long *)ws, st, num_sms()))) return rc;
    unsigned long long h[6];
    cudaError_t e = cudaMemcpyAsync(h, ws, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (e) return fail_cuda(e);
    for (int t = 0; t < 6; ++t) counts[t] = (int64_t)h[t];
    return HK_OK;
}

int hk_count_ring_pairs(const hk_lines *lines, const hk_grid *grid, const hk_state *state,
                        const hk_opts *opts, int64_t *ring, void *stream)
{
    int rc;
    if ((rc = check_lines(lines, true)) || (rc = check_grid(grid)) || (rc = check_state(state)) ||
        (rc = check_opts(opts)))
        return rc;
    if (!ring) return HK_EINVAL;
    *ring = 0;
    const GridD g = make_grid(grid, opts);
    // the FP32C short-line batches: a fixed cut of fewer than 1024 bins, Voigt
    const bool short_lines = opts->precision == HK_FP32C && g.profile == kProfVoigt &&
                             g.W > 0.0 && 2.0 * g.W + 1.0 < 1024.0;
    if (lines->n == 0 || !short_lines) return HK_OK;
    char *ws;
    if ((rc = pool_get(256, &ws))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Prob p = make_prob(lines, state, opts);
    if ((rc = count_pairs_run(p, g, (unsigned long long *)ws, st, num_sms()))) return rc;
    unsigned long long h[7];
    cudaError_t e = cudaMemcpyAsync(h, ws, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (e) return fail_cuda(e);
    *ring = (int64_t)h[6];
    return HK_OK;
}

int hk_profile(int mode, double *ms, int64_t *launches)
{
    if (mode != 0 && mode != 1) return HK_EINVAL;
    return gather_profile(mode, ms, launches);
}

int hk_sync_status(void *stream)
{
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e) return fail_cuda(e);
    unsigned *sw = status_word();
    if (!sw) return HK_ENOMEM;
    unsigned v = 0;
    e = cudaMemcpy(&v, sw, sizeof(v), cudaMemcpyDeviceToHost);
    if (!e && v) e = cudaMemset(sw, 0, sizeof(v));
    if (e) return fail_cuda(e);
    if (v & kStatusTimeout) return HK_ETIMEOUT;
    if (v & kStatusRange) return HK_ERANGE;
    return HK_OK;
}

int hk_line_strength(const hk_lines *lines, const hk_state *state, const hk_opts *opts,
                     double *S_out, void *stream)
{
    int rc;
    if ((rc = check_lines(lines, true)) || (rc = check_state(state)) || (rc = check_opts(opts)))
        return rc;
    if (lines->n == 0) return HK_OK;
    if (!S_out) return HK_EINVAL;
    Prob p = make_prob(lines, state, opts);
    k_strength<<<num_sms() * 4, 256, 0, (cudaStream_t)stream>>>(p, S_out);
    cudaError_t e = cudaGetLastError();
    return e ? fail_cuda(e) : HK_OK;
}

int hk_widths(const hk_lines *lines, const hk_state *state, const hk_opts *opts,
              float *alphaD_inv_out, float *y_out, void *stream)
{
    int rc;
    if ((rc = check_lines(lines, true)) || (rc = check_state(state)) || (rc = check_opts(opts)))
        return rc;
    if (lines->n == 0) return HK_OK;
    if (!alphaD_inv_out || !y_out) return HK_EINVAL;
    Prob p = make_prob(lines, state, opts);
    k_widths<<<num_sms() * 4, 256, 0, (cudaStream_t)stream>>>(p, alphaD_inv_out, y_out);
    cudaError_t e = cudaGetLastError();
    return e ? fail_cuda(e) : HK_OK;
}

int hk_voigt_accumulate(const double *nu0, const double *S, const float *alphaD_inv,
                        const float *y, int64_t n, const hk_grid *grid, double cut,
                        void *sigma_inout, int precision, void *stream)
{
    int rc;
    if ((rc = check_grid(grid))) return rc;
    if (n < 0 || !std::isfinite(cut) || (precision != HK_FP32C && precision != HK_FP64))
        return HK_EINVAL;
    if (n == 0) return HK_OK;
    if (!nu0 || !S || !alphaD_inv || !y || !sigma_inout) return HK_EINVAL;
    Prob p;
    memset(&p, 0, sizeof(p));
    p.nu0 = nu0;
    p.S_pre = S;
    p.aDinv_pre = alphaD_inv;
    p.y_pre = y;
    p.n = n;
    p.pre = 1;
    GridD g = make_grid_cut(grid, cut);
    Tune t = get_tune(precision);
    size_t need = gather_workspace(1, g, precision, t.bpt);
    char *ws;
    if ((rc = pool_get(need, &ws))) return rc;
    unsigned *sw = status_word();
    if (!sw) return HK_ENOMEM;
    return gather_run(&p, 1, g, precision, t.bpt, t.lmax, sigma_inout, 0, 1, ws, need, sw,
                      (cudaStream_t)stream, num_sms());
}

static int cross_section_impl(const hk_lines *lines, const hk_grid *grid, const hk_state *state,
                              const hk_opts *opts, void *sigma_out, cudaStream_t st, int bpt,
                              int lmax)
{
    int rc;
    GridD g = make_grid(grid, opts);
    int prec = opts->precision;
    const int out_f64 = (opts->flags & HK_SIGMA_F64) ? 1 : 0;
    if (lines->n == 0) {
        size_t b = (size_t)grid->nbins * ((prec == HK_FP64 || out_f64) ? 8 : 4);
        cudaError_t e = cudaMemsetAsync(sigma_out, 0, b, st);
        return e ? fail_cuda(e) : HK_OK;
    }
    size_t need = gather_workspace(1, g, prec, bpt);
    size_t sort_need = 0, cub_b = 0;
    if (!lines->sorted) sort_need = al(sort_bytes(lines->n, &cub_b));
    char *ws;
    if ((rc = pool_get(need + sort_need, &ws))) return rc;
    hk_lines L = *lines;
    if (!lines->sorted) {
        int64_t *perm;
        if ((rc = sort_lines(lines, ws + need, &L, &perm, st))) return rc;
    }
    Prob p = make_prob(&L, state, opts);
    unsigned *sw = status_word();
    if (!sw) return HK_ENOMEM;
    return gather_run(&p, 1, g, prec, bpt, lmax, sigma_out, out_f64, 0, ws, need, sw, st,
                      num_sms());
}

int hk_cross_section(const hk_lines *lines, const hk_grid *grid, const hk_state *state,
                     const hk_opts *opts, void *sigma_out, void *stream)
{
    int rc;
    if ((rc = check_lines(lines, true)) || (rc = check_grid(grid)) || (rc = check_state(state)) ||
        (rc = check_opts(opts)))
        return rc;
    if (!sigma_out) return HK_EINVAL;
    Tune t = get_tune(opts->precision);
    return cross_section_impl(lines, grid, state, opts, sigma_out, (cudaStream_t)stream, t.bpt,
                              t.lmax);
}

// ---- hk_cross_section_host: host line list streamed in blocks ----------------
// Per device: a copy stream, a second compute stream and five events.  Blocks
// alternate between buffer/stream pair 0 (the caller's stream) and pair 1
// (the second compute stream), each pair with its own gather workspace and
// FP64 partial sigma, so one block's kernels can fill the SMs that the
// previous block's persistent launch leaves idle at its end.  `start` orders
// all of it after earlier work on the caller's stream (which may still read
// the pool); copied[b] / done[b] hand buffer b between the copy stream and
// compute stream b; the caller's stream finally waits for done[1] and adds
// the two partial sums.
struct CopyCtx {
    cudaStream_t cs = nullptr, st2 = nullptr;
    cudaEvent_t start = nullptr, copied[2] = {nullptr, nullptr}, done[2] = {nullptr, nullptr};
};
static std::mutex g_copy_mu;
static std::map<int, CopyCtx> g_copy;

static int copy_ctx(CopyCtx **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return fail_cuda(e);
    std::lock_guard<std::mutex> lk(g_copy_mu);
    auto it = g_copy.find(dev);
    if (it != g_copy.end()) {
        *out = &it->second;
        return HK_OK;
    }
    CopyCtx c;
    e = cudaStreamCreateWithFlags(&c.cs, cudaStreamNonBlocking);
    if (!e) e = cudaStreamCreateWithFlags(&c.st2, cudaStreamNonBlocking);
    cudaEvent_t *evs[5] = {&c.start, &c.copied[0], &c.copied[1], &c.done[0], &c.done[1]};
    for (int i = 0; i < 5 && !e; ++i) e = cudaEventCreateWithFlags(evs[i], cudaEventDisableTiming);
    if (e) return fail_cuda(e);
    *out = &(g_copy[dev] = c);
    return HK_OK;
}

// out = a (+ b), as double (o64) or float (o32, with the overflow flag).
__global__ void k_combine(const double *__restrict__ a, const double *__restrict__ b,
                          double *o64, float *o32, int64_t n, unsigned *status)
{
    bool over = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = b ? a[i] + b[i] : a[i];
        if (o64) {
            o64[i] = v;
        } else {
            const float f = (float)v;
            over |= isinf(f) && !isinf(v);
            o32[i] = f;
        }
    }
    if (over) atomicOr(status, kStatusRange);
}

int hk_cross_section_host(const hk_lines *lines, const hk_grid *grid, const hk_state *state,
                          const hk_opts *opts, void *sigma_out, int64_t chunk_lines,
                          void *stream)
{
    int rc;
    if ((rc = check_lines(lines, true)) || (rc = check_grid(grid)) || (rc = check_state(state)) ||
        (rc = check_opts(opts)))
        return rc;
    if (!sigma_out || chunk_lines < 0) return HK_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const int prec = opts->precision;
    const int out_f64 = (prec == HK_FP64 || (opts->flags & HK_SIGMA_F64)) ? 1 : 0;
    const int64_t n = lines->n, nbins = grid->nbins;
    const int64_t C = std::max<int64_t>(1, std::min<int64_t>(chunk_lines > 0 ? chunk_lines
                                                                             : (int64_t)1 << 26,
                                                             std::max<int64_t>(n, 1)));
    // float fields present (S_ref, E_low, gamma_ref, n_T, A, g_up, gamma_self, delta)
    const float *hf[8] = {lines->S_ref, lines->E_low, lines->gamma_ref, lines->n_T, lines->A,
                          lines->g_up,  lines->gamma_self, lines->delta};
    Tune t = get_tune(prec);
    const GridD g = make_grid(grid, opts);
    const size_t need_g = al(gather_workspace(1, g, prec, t.bpt));
    size_t cub_b = 0;
    const size_t sort_need = lines->sorted ? 0 : al(sort_bytes(C, &cub_b));
    size_t buf = al((size_t)C * 8);
    for (int f = 0; f < 8; ++f)
        if (hf[f]) buf += al((size_t)C * 4);
    const size_t sig_b = al((size_t)nbins * 8);
    const size_t out_b = out_f64 ? sig_b : al((size_t)nbins * 4);
    const size_t per_pair = need_g + sort_need + buf + sig_b;
    char *ws;
    if ((rc = pool_get(2 * per_pair + out_b, &ws))) return rc;
    char *ws_g[2], *ws_sort[2], *bufs[2];
    double *sig[2];
    for (int b = 0; b < 2; ++b) {
        char *base = ws + b * per_pair;
        ws_g[b] = base;
        ws_sort[b] = base + need_g;
        bufs[b] = base + need_g + sort_need;
        sig[b] = (double *)(base + need_g + sort_need + buf);
    }
    char *outbuf = ws + 2 * per_pair;
    unsigned *sw = status_word();
    if (!sw) return HK_ENOMEM;
    CopyCtx *cx;
    if ((rc = copy_ctx(&cx))) return rc;
    cudaStream_t cst[2] = {st, cx->st2};
    cudaError_t e;
    if ((e = cudaEventRecord(cx->start, st))) return fail_cuda(e);
    if ((e = cudaStreamWaitEvent(cx->cs, cx->start, 0))) return fail_cuda(e);
    if ((e = cudaStreamWaitEvent(cx->st2, cx->start, 0))) return fail_cuda(e);
    const int nsms = num_sms();
    // blocks grow from C/8 to C so the first copy, which nothing hides, is short
    int64_t nblk = 0;
    for (int64_t off = 0, i = 0; off < n; ++i, ++nblk) {
        const int b = (int)(i & 1);
        const int64_t cap = i < 3 ? std::max<int64_t>(1, C >> (3 - i)) : C;
        const int64_t cnt = std::min(cap, n - off);
        if (i >= 2 && (e = cudaStreamWaitEvent(cx->cs, cx->done[b], 0))) return fail_cuda(e);
        hk_lines L = *lines;
        L.n = cnt;
        char *cur = bufs[b];
        L.nu0 = (const double *)cur;
        if ((e = cudaMemcpyAsync(cur, lines->nu0 + off, sizeof(double) * cnt, cudaMemcpyDefault,
                                 cx->cs)))
            return fail_cuda(e);
        cur += al((size_t)C * 8);
        const float **lf[8] = {&L.S_ref, &L.E_low, &L.gamma_ref, &L.n_T,
                               &L.A,     &L.g_up,  &L.gamma_self, &L.delta};
        for (int f = 0; f < 8; ++f) {
            if (!hf[f]) continue;
            *lf[f] = (const float *)cur;
            if ((e = cudaMemcpyAsync(cur, hf[f] + off, sizeof(float) * cnt, cudaMemcpyDefault,
                                     cx->cs)))
                return fail_cuda(e);
            cur += al((size_t)C * 4);
        }
        if ((e = cudaEventRecord(cx->copied[b], cx->cs))) return fail_cuda(e);
        if ((e = cudaStreamWaitEvent(cst[b], cx->copied[b], 0))) return fail_cuda(e);
        hk_lines Ls = L;
        if (!lines->sorted) {
            int64_t *perm;
            if ((rc = sort_lines(&L, ws_sort[b], &Ls, &perm, cst[b]))) return rc;
        }
        Prob p = make_prob(&Ls, state, opts);
        if ((rc = gather_run(&p, 1, g, prec, t.bpt, t.lmax, sig[b], 1, i >= 2 ? 1 : 0, ws_g[b],
                             need_g, sw, cst[b], nsms)))
            return rc;
        if ((e = cudaEventRecord(cx->done[b], cst[b]))) return fail_cuda(e);
        off += cnt;
    }
    if (nblk == 0 && (e = cudaMemsetAsync(sig[0], 0, sizeof(double) * (size_t)nbins, st)))
        return fail_cuda(e);
    if (nblk >= 2 && (e = cudaStreamWaitEvent(st, cx->done[1], 0))) return fail_cuda(e);
    k_combine<<<nsms * 4, 256, 0, st>>>(sig[0], nblk >= 2 ? sig[1] : nullptr,
                                        out_f64 ? (double *)outbuf : nullptr,
                                        out_f64 ? nullptr : (float *)outbuf, nbins, sw);
    if ((e = cudaGetLastError())) return fail_cuda(e);
    const size_t bytes = (out_f64 ? sizeof(double) : sizeof(float)) * (size_t)nbins;
    if ((e = cudaMemcpyAsync(sigma_out, outbuf, bytes, cudaMemcpyDefault, st))) return fail_cuda(e);
    return HK_OK;
}

// ---- hk_cross_section_noalloc: scratch in a fixed device array ---------------
// The array lives in device memory of every GPU that loads the library.  Host
// code must never hand the symbol itself to a kernel (on the host it names a
// host-side shadow); the device address comes from cudaGetSymbolAddress, looked
// up once per device with that device current.  Layout: [0, 256) a status word
// for the finalize kernel, [256, HK_NOALLOC_SCRATCH_BYTES) the gather's scratch.
static __device__ __align__(256) unsigned char g_noalloc_scratch[HK_NOALLOC_SCRATCH_BYTES];
static std::mutex g_noalloc_mu;
static std::map<int, char *> g_noalloc_addr;

static int noalloc_scratch(char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return fail_cuda(e);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    auto it = g_noalloc_addr.find(dev);
    if (it != g_noalloc_addr.end()) {
        *out = it->second;
        return HK_OK;
    }
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return fail_cuda(e ? e : cudaErrorInvalidSymbol);
    g_noalloc_addr[dev] = (char *)p;
    *out = (char *)p;
    return HK_OK;
}

int hk_cross_section_noalloc(const hk_lines *lines, const hk_grid *grid, const hk_state *state,
                             const hk_opts *opts, void *sigma_out, void *stream)
{
    int rc;
    if ((rc = check_lines(lines, true)) || (rc = check_grid(grid)) || (rc = check_state(state)) ||
        (rc = check_opts(opts)))
        return rc;
    if (!sigma_out) return HK_EINVAL;
    if (lines->n > 0 && !lines->sorted) return HK_ENOTSUP;
    const int prec = opts->precision;
    Tune t = get_tune(prec);
    const size_t need = gather_workspace(1, make_grid(grid, opts), prec, t.bpt);
    if (need + 256 > (size_t)HK_NOALLOC_SCRATCH_BYTES) return HK_ESIZE;
    char *scratch;
    if ((rc = noalloc_scratch(&scratch))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int out_f64 = (opts->flags & HK_SIGMA_F64) ? 1 : 0;
    cudaError_t e;
    if (lines->n == 0) {
        size_t b = (size_t)grid->nbins * ((prec == HK_FP64 || out_f64) ? 8 : 4);
        e = cudaMemsetAsync(sigma_out, 0, b, st);
        return e ? fail_cuda(e) : HK_OK;
    }
    unsigned *status = (unsigned *)scratch;
    if ((e = cudaMemsetAsync(status, 0, sizeof(unsigned), st))) return fail_cuda(e);
    GridD g = make_grid(grid, opts);
    Prob p = make_prob(lines, state, opts);
    // gather_run clears the accumulator, the scale slot and the work counter
    return gather_run(&p, 1, g, prec, t.bpt, t.lmax, sigma_out, out_f64, 0, scratch + 256, need,
                      status, st, num_sms());
}

int hk_noalloc_status(void *stream)
{
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e) return fail_cuda(e);
    int dev = 0;
    if ((e = cudaGetDevice(&dev))) return fail_cuda(e);
    char *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        auto it = g_noalloc_addr.find(dev);
        if (it == g_noalloc_addr.end()) return HK_OK;   // no call on this device yet
        scratch = it->second;
    }
    unsigned v = 0;
    e = cudaMemcpy(&v, scratch, sizeof(v), cudaMemcpyDeviceToHost);
    if (!e && v) e = cudaMemset(scratch, 0, sizeof(v));
    if (e) return fail_cuda(e);
    if (v & kStatusTimeout) return HK_ETIMEOUT;
    if (v & kStatusRange) return HK_ERANGE;
    return HK_OK;
}

// Whether the problems of one species in a batched call share each line's
// bin geometry (a fixed cut or none, no pressure shift), and there are enough
// of them for a geometry prepass to pay.
static bool shared_geometry(const hk_lines &L, int nTP, const hk_opts *opts)
{
    return nTP >= 2 && L.n > 0 && !L.delta && opts->cut_mode != HK_CUT_DOPPLER &&
           opts->cut_mode != HK_CUT_LORENTZ;
}

int hk_workspace_size(int kind, const hk_lines *species, int nspecies, int nTP,
                      const hk_grid *grid, const hk_opts *opts, size_t *bytes)
{
    int rc;
    if (!bytes || !species || nspecies <= 0 || nTP <= 0 || (kind != 0 && kind != 1)) return HK_EINVAL;
    if ((rc = check_grid(grid)) || (rc = check_opts(opts))) return rc;
    size_t total = 0;
    if (kind == 0) {
        Tune t = get_tune(opts->precision);
        total = gather_workspace(nspecies * nTP, make_grid(grid, opts), HK_FP32C, t.bpt);
        for (int s = 0; s < nspecies; ++s) {
            if ((rc = check_lines(&species[s], true))) return rc;
            if (!species[s].sorted && species[s].n > 0) {
                size_t cb;
                total += al(sort_bytes(species[s].n, &cb));
            }
            if (shared_geometry(species[s], nTP, opts))
                total += al((size_t)species[s].n * sizeof(int4));
        }
    } else {
        if ((rc = check_lines(&species[0], true))) return rc;
        total = backward_workspace(species[0].n, nTP, grid->nbins);
        if (!species[0].sorted && species[0].n > 0) {
            size_t cb;
            total += al(sort_bytes(species[0].n, &cb));
        }
    }
    *bytes = total;
    return HK_OK;
}

int hk_cross_section_batched(const hk_lines *species, int nspecies, const hk_state *TP, int nTP,
                             const hk_grid *grid, const hk_opts *opts, void *sigma_out,
                             void *workspace, size_t ws_bytes, void *stream)
{
    int rc;
    if (!species || nspecies <= 0 || !TP || nTP <= 0 || !sigma_out) return HK_EINVAL;
    if ((rc = check_grid(grid)) || (rc = check_opts(opts))) return rc;
    if (opts->precision != HK_FP32C) return HK_ENOTSUP;
    for (int s = 0; s < nspecies; ++s)
        if ((rc = check_lines(&species[s], true))) return rc;
    for (int k = 0; k < nTP; ++k)
        if ((rc = check_state(&TP[k]))) return rc;
    size_t need;
    if ((rc = hk_workspace_size(0, species, nspecies, nTP, grid, opts, &need))) return rc;
    if (!workspace || ws_bytes < need) return HK_ENOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    Tune t = get_tune(HK_FP32C);
    size_t gneed = gather_workspace(nspecies * nTP, make_grid(grid, opts), HK_FP32C, t.bpt);
    char *sort_ws = (char *)workspace + gneed;
    std::vector<hk_lines> L(species, species + nspecies);
    for (int s = 0; s < nspecies; ++s) {
        if (!species[s].sorted && species[s].n > 0) {
            int64_t *perm;
            if ((rc = sort_lines(&species[s], sort_ws, &L[s], &perm, st))) return rc;
            size_t cb;
            sort_ws += al(sort_bytes(species[s].n, &cb));
        }
    }
    GridD g = make_grid(grid, opts);
    std::vector<Prob> probs;
    probs.reserve((size_t)nspecies * nTP);
    for (int s = 0; s < nspecies; ++s) {
        // each line's bin geometry once for all (T, P) points when they share it
        int4 *geo = nullptr;
        if (shared_geometry(species[s], nTP, opts)) {
            geo = (int4 *)sort_ws;
            sort_ws += al((size_t)species[s].n * sizeof(int4));
            if ((rc = line_geo_launch(make_prob(&L[s], &TP[0], opts), g, geo, st, num_sms())))
                return rc;
        }
        for (int k = 0; k < nTP; ++k) {
            probs.push_back(make_prob(&L[s], &TP[k], opts));
            probs.back().geo = geo;
        }
    }
    unsigned *sw = status_word();
    if (!sw) return HK_ENOMEM;
    return gather_run(probs.data(), (int)probs.size(), g, HK_FP32C, t.bpt, t.lmax, sigma_out,
                      (opts->flags & HK_SIGMA_F64) ? 1 : 0, 0, (char *)workspace, gneed, sw, st,
                      num_sms());
}

int hk_cross_section_backward(const hk_lines *lines, const hk_grid *grid, const hk_state *TP,
                              int nTP, const hk_opts *opts, const float *grad_sigma,
                              double *dL_dT, double *dL_dP, double *dL_dSref,
                              double *dL_dgamma_ref, void *workspace, size_t ws_bytes,
                              void *stream)
{
    int rc;
    if ((rc = check_lines(lines, true)) || (rc = check_grid(grid)) || (rc = check_opts(opts)))
        return rc;
    if (!TP || nTP <= 0 || !grad_sigma || !dL_dT || !dL_dP) return HK_EINVAL;
    if (lines->n > 0 && (!dL_dSref || !dL_dgamma_ref)) return HK_EINVAL;
    if (lines->s_mode != HK_S_REF) return HK_ENOTSUP;
    if (opts->cut_mode == HK_CUT_DOPPLER || opts->cut_mode == HK_CUT_LORENTZ ||
        (opts->flags & HK_REMOVE_PLINTH) || opts->profile != HK_PROFILE_VOIGT ||
        lines->gamma_self || lines->delta)
        return HK_ENOTSUP;
    for (int k = 0; k < nTP; ++k)
        if ((rc = check_state(&TP[k]))) return rc;
    size_t need;
    if ((rc = hk_workspace_size(1, lines, 1, nTP, grid, opts, &need))) return rc;
    if (!workspace || ws_bytes < need) return HK_ENOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    size_t bneed = backward_workspace(lines->n, nTP, grid->nbins);
    hk_lines L = *lines;
    const int64_t *perm = nullptr;
    if (!lines->sorted && lines->n > 0) {
        int64_t *pm;
        if ((rc = sort_lines(lines, (char *)workspace + bneed, &L, &pm, st))) return rc;
        perm = pm;
    }
    std::vector<Prob> probs;
    std::vector<double> dlnQ(nTP), T(nTP), P(nTP);
    for (int k = 0; k < nTP; ++k) {
        probs.push_back(make_prob(&L, &TP[k], opts));
        dlnQ[k] = TP[k].dlnQ_dT;
        T[k] = TP[k].T;
        P[k] = TP[k].P;
    }
    GridD g = make_grid(grid, opts);
    return backward_run(probs.data(), nTP, g, grad_sigma, dlnQ.data(), T.data(), P.data(), dL_dT,
                        dL_dP, dL_dSref, dL_dgamma_ref, perm, (char *)workspace, bneed, st,
                        num_sms());
}

int hk_autotune(const hk_lines *lines, const hk_grid *grid, const hk_state *state,
                const hk_opts *opts, void *stream)
{
    int rc;
    if ((rc = check_lines(lines, true)) || (rc = check_grid(grid)) || (rc = check_state(state)) ||
        (rc = check_opts(opts)))
        return rc;
    if (lines->n == 0) return HK_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int prec = opts->precision;
    // lines per work item: small items balance uneven line density across the
    // SMs, large ones cut the per-item cost (record setup, one FP64 atomic per
    // bin of the tile); FP32C also the tile width: 1024 bins (3 blocks of 8
    // warps per SM) or 2048 (2 blocks; half the tile visits of a wide line)
    const int lmaxs[] = {1024, 2048, 4096, 16384, 65536};
    const int nl = (int)(sizeof(lmaxs) / sizeof(lmaxs[0]));
    const int tiles[] = {1024, 2048};
    const int nt = prec == HK_FP32C ? 2 : 1;
    const int ncand = nl * nt;
    size_t out_b = (size_t)grid->nbins * 8;
    // the output buffer lives in its own cudaMalloc (the pool is used by the runs)
    void *out = nullptr;
    if (cudaMalloc(&out, out_b) != cudaSuccess) {
        (void)cudaGetLastError();
        return HK_ENOMEM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaEventCreate(&e0);
    if (!ce) ce = cudaEventCreate(&e1);
    if (ce) {
        rc = fail_cuda(ce);
        if (e0) cudaEventDestroy(e0);
        cudaFree(out);
        return rc;
    }
    hk_opts o = *opts;
    o.flags |= HK_SIGMA_F64;  // time without any float-overflow concern
    Tune best = get_tune(prec);
    float best_ms = 1e30f;
    for (int j = 0; j < ncand && rc == HK_OK; ++j) {
        const int bpt = prec == HK_FP32C ? tiles[j / nl] : get_tune(prec).bpt;
        const int lmax = lmaxs[j % nl];
        rc = cross_section_impl(lines, grid, state, &o, out, st, bpt, lmax);  // warm-up
        if (rc) break;
        if ((ce = cudaEventRecord(e0, st))) {
            rc = fail_cuda(ce);
            break;
        }
        rc = cross_section_impl(lines, grid, state, &o, out, st, bpt, lmax);
        if (rc) break;
        float ms = 0;
        if ((ce = cudaEventRecord(e1, st)) || (ce = cudaEventSynchronize(e1)) ||
            (ce = cudaEventElapsedTime(&ms, e0, e1))) {
            rc = fail_cuda(ce);
            break;
        }
        if (ms < best_ms) {
            best_ms = ms;
            best.bpt = bpt;
            best.lmax = lmax;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ce = cudaStreamSynchronize(st);
    if (ce && !rc) rc = fail_cuda(ce);
    ce = cudaFree(out);
    if (ce && !rc) rc = fail_cuda(ce);
    if (rc) return rc;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[{dev, prec}] = best;
    return HK_OK;
}

int hk_measure_peak(int kind, double target_ms, double *ops_per_s, void *stream)
{
    if (kind < 0 || kind > 4 || !ops_per_s || !(target_ms > 0.0) || target_ms > 60000.0)
        return HK_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const int sms = num_sms();
    char *scratch;
    int rc = pool_get((size_t)sms * 8 * 256 * sizeof(double), &scratch);
    if (rc) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (!e) e = cudaEventCreate(&e1);
    double ops = 0.0, total_ops = 0.0;
    float ms = 0.0f;
    int iters = 256;
    // calibration launch (also the warm-up), then launches of ~100 ms each
    if (!e && !(rc = peak_launch(kind, iters, sms, scratch, &ops, st))) {
        if (!(e = cudaEventRecord(e0, st)) &&
            !(rc = peak_launch(kind, iters, sms, scratch, &ops, st)) &&
            !(e = cudaEventRecord(e1, st)) && !(e = cudaEventSynchronize(e1)) &&
            !(e = cudaEventElapsedTime(&ms, e0, e1))) {
            // at most 2000x the calibration launch, so a launch stays bounded
            const double scale = std::min(100.0 / std::max((double)ms, 1e-3), 2000.0);
            iters = (int)std::max(iters * scale, 256.0);
            const int reps = std::max(1, (int)std::ceil(target_ms / 100.0));
            if (!(e = cudaEventRecord(e0, st))) {
                for (int r = 0; r < reps && !rc; ++r) {
                    rc = peak_launch(kind, iters, sms, scratch, &ops, st);
                    total_ops += ops;
                }
                if (!rc && !(e = cudaEventRecord(e1, st)) && !(e = cudaEventSynchronize(e1)))
                    e = cudaEventElapsedTime(&ms, e0, e1);
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rc) return rc;
    if (e) return fail_cuda(e);
    *ops_per_s = total_ops / (ms * 1e-3);
    return HK_OK;
}

int hk_tuning(int precision, int *lmax, int *tile_bins)
{
    if ((precision != HK_FP32C && precision != HK_FP64) || !lmax) return HK_EINVAL;
    const Tune t = get_tune(precision);
    *lmax = t.lmax;
    if (tile_bins) *tile_bins = gather_tile_bins(precision, t.bpt);
    return HK_OK;
}

int hk_set_tuning(int precision, int lmax, int tile_bins)
{
    if ((precision != HK_FP32C && precision != HK_FP64) || lmax < 32 || lmax > (1 << 24))
        return HK_EINVAL;
    if (tile_bins != 0 && (precision == HK_FP64 ? tile_bins != gather_tile_bins(HK_FP64, 2)
                                                : !gather_f32_tile_ok(tile_bins)))
        return HK_EINVAL;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return fail_cuda(e);
    Tune t = get_tune(precision);
    t.lmax = lmax;
    if (tile_bins != 0 && precision == HK_FP32C) t.bpt = tile_bins;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[{dev, precision}] = t;
    return HK_OK;
}

}  // extern "C"
