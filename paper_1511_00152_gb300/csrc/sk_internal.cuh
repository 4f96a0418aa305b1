// sk_internal.cuh -- device helpers shared by the library's kernels.
//
// Philox4x32-10 follows Salmon, Moraes, Dror and Shaw, "Parallel random
// numbers: as easy as 1, 2, 3" (SC'11): ten rounds of two 32x32->64-bit
// multiplies with the Weyl key schedule.  The word layout of the sign and
// mask streams is the library's written spec (see include/sk.h).
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/sk.h"

namespace sk {

constexpr uint32_t kTagSign = 0x5349474Eu;  // "SIGN"
constexpr uint32_t kTagMask = 0x4D41534Bu;  // "MASK"

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(kPhiloxM0, c.x);
        const uint32_t lo0 = kPhiloxM0 * c.x;
        const uint32_t hi1 = __umulhi(kPhiloxM1, c.z);
        const uint32_t lo1 = kPhiloxM1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return c;
}

__device__ __forceinline__ uint32_t pick_word(uint4 v, uint32_t lane) {
    return lane == 0 ? v.x : lane == 1 ? v.y : lane == 2 ? v.z : v.w;
}

// Word w of the mask stream of global row g.
__device__ __forceinline__ uint32_t mask_word(uint32_t k0, uint32_t k1, uint64_t g,
                                              uint32_t w) {
    const uint4 o = philox4x32_10(
        make_uint4(w >> 2, (uint32_t)g, (uint32_t)(g >> 32), kTagMask), k0, k1);
    return pick_word(o, w & 3u);
}

// Sign bit (1 = negative) of coordinate j of D.
__device__ __forceinline__ uint32_t sign_bit(uint32_t k0, uint32_t k1, uint32_t j) {
    const uint4 o = philox4x32_10(make_uint4(j >> 7, 0u, 0u, kTagSign), k0, k1);
    return (pick_word(o, (j >> 5) & 3u) >> (j & 31u)) & 1u;
}

// float64 reciprocal square root and reciprocal by Newton-Raphson.
// The argument is split as m 2^(2k) (m in [1, 4)) or m 2^e (m in [1, 2)) so
// the float32 estimate of the mantissa part is always in range; two
// Newton-Raphson steps (y <- y (3 - m y^2) / 2, resp. y <- y (2 - m y)) take
// its ~22 correct bits past float64 precision; the exponent is then restored.
// For positive (resp. nonzero) normal x with |exponent| <= 1022; accurate to
// a few units in the last place, not correctly rounded.
__device__ __forceinline__ double pow2(int e) {  // 2^e for -1022 <= e <= 1023
    return __longlong_as_double((long long)(e + 1023) << 52);
}

__device__ __forceinline__ double rsqrt_nr(double x) {
    const long long bits = __double_as_longlong(x);
    const int e = (int)((bits >> 52) & 0x7ff) - 1023;
    const int k = e >> 1;  // floor(e / 2)
    const double m = __longlong_as_double((bits & 0x000fffffffffffffLL) |
                                          ((long long)(e - 2 * k + 1023) << 52));
    double y = (double)rsqrtf((float)m);
    const double hm = 0.5 * m;
    y = y * (1.5 - hm * y * y);
    y = y * (1.5 - hm * y * y);
    return y * pow2(-k);
}

__device__ __forceinline__ double rcp_nr(double x) {
    const long long bits = __double_as_longlong(x);
    const int e = (int)((bits >> 52) & 0x7ff) - 1023;
    const double m = __longlong_as_double((bits & 0x800fffffffffffffLL) | (1023LL << 52));
    double y = (double)__frcp_rn((float)m);
    y = y * (2.0 - m * y);
    y = y * (2.0 - m * y);
    return y * pow2(-e);
}

// Index j of a caller's ELL entry kept inside [0, pt): the identity for
// valid input (sk_compress writes indices below pt); a bad index is clamped
// rather than reaching outside the library's arrays.  pt need not be a power
// of two (the DCT preconditioner keeps pt = p).
__device__ __forceinline__ int clamp_index(int j, int pt) {
    return (int)min((unsigned)j, (unsigned)(pt - 1));
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned lanemask_gt() {
    unsigned r;
    asm("mov.u32 %0, %%lanemask_gt;" : "=r"(r));
    return r;
}

}  // namespace sk

// Host-side launchers (defined in the kernel files, called by sk_api.cu).
struct sk_ctx {
    int64_t p;
    int64_t pt;
    int log2pt;
    int64_t m;
    uint64_t seed;
    uint32_t flags;  // SK_FLAG_* of sk_init_ex
    // autotuned launch choices (0: the built-in heuristics)
    int gram_n;      // Gram tile width, 128 or 256
    int split_mult;  // multiplier on the Gram row-split count
    int compress_ctas;  // compress CTAs per SM (1 or 2)
    // SK_FLAG_DCT: radices of the FFT of length p / 2 (pt = p, no padding;
    // log2pt is then the exponent of the next power of two, for sizing only)
    int dct_nf;
    int dct_fac[16];
};

namespace sk {
// Records the calling thread's message for sk_last_error (sk_api.cu).
void set_last_error(const char *msg);

// ---- many data sets in one launch (batch.cu holds the plan; each kernel
// file builds its part of the device table and launches from it)
struct BatchRows {  // one data set's rows and ELL output
    const float *X;
    int64_t n, ldx, row0;
    int32_t *idx;
    float *val;
};
struct CompressBatchInfo {
    size_t params_off, tasks_off, ticket_off, smem;
    int ntasks, grid;
};
bool compress_batchable(const sk_ctx &c, const float *X, int64_t ldx);
cudaError_t compress_batch_build(const sk_ctx *ctxs, const BatchRows *rows, int nd,
                                 int units_per_group, std::vector<unsigned char> &table,
                                 CompressBatchInfo &info);
cudaError_t compress_batch_launch(const CompressBatchInfo &info, unsigned char *dev_table,
                                  cudaStream_t s);
struct BatchGram {  // one data set's ELL rows, Gram accumulator and workspace
    const int32_t *idx;
    const float *val;
    int64_t n;
    double *G;
    void *work;
};
struct GramBatchInfo {
    size_t tc_off, bk_off, slab_off, cta_off, smem;
    int64_t slabs, ctas;
    int nd, first;
};
cudaError_t gram_batch_build(const sk_ctx *ctxs, const BatchGram *rows, int nd, int mode,
                             std::vector<unsigned char> &table, GramBatchInfo &info);
cudaError_t gram_batch_launch(const GramBatchInfo &info, unsigned char *dev_table, cudaStream_t s);
struct BatchKmeans {  // one data set's ELL rows and K-means state
    const int32_t *idx;
    const float *val;
    int64_t n;
    int K;
    float *mu;
    float *mu_t;
    int32_t *labels;
    double *S;
    int32_t *cnt;
    int64_t *nk;
    int64_t *changed;
};
struct KmeansBatchInfo {
    size_t params_off, tasks_off, start_off, ticket_off, smem;
    int64_t total;
    int nd, ntasks, grid, mu_cap;
    // tasks [ntasks_smem, ntasks) read their centre table from global memory
    // and run as a second launch with the staging region alone (smem_g
    // bytes, grid_g CTAs), leaving the rest of the SM's memory to L1
    int ntasks_smem, grid_g;
    size_t smem_g;
};
cudaError_t kmeans_batch_build(const sk_ctx *ctxs, const BatchKmeans *it, int nd,
                               std::vector<unsigned char> &table, KmeansBatchInfo &info);
// op: 0 reset the sums, 1 full pass, 2 incremental pass, 3 finalize the centres
cudaError_t kmeans_batch_launch(const KmeansBatchInfo &info, unsigned char *dev_table, int op,
                                cudaStream_t s);

// The DCT preconditioner (dct.cu): factorisation of p / 2 at sk_init_ex; the
// forward rows (Y != NULL: dense y = H D x; else val = y[idx] with the masks
// already in idx) and the un-mixing rows D H^T (float32 or float64).
bool dct_factor(int64_t L, int *fac, int *nf);
size_t dct_forward_smem(const sk_ctx &c);
cudaError_t launch_dct_forward(const sk_ctx &c, const float *X, int64_t n, int64_t ldx,
                               const int32_t *idx, float *val, float *Y, cudaStream_t s);
cudaError_t launch_dct_inverse(const sk_ctx &c, const void *in, int64_t r, void *out, bool f64,
                               cudaStream_t s);

cudaError_t launch_compress(const sk_ctx &c, const float *X, int64_t n, int64_t ldx,
                            int64_t row0, int32_t *idx, float *val, float *Y,
                            cudaStream_t s);
cudaError_t launch_kmeans(const sk_ctx &c, const int32_t *idx, const float *val,
                          int64_t n, const float *mu, int K, int32_t *labels, float *dist,
                          double *S, int32_t *cnt, int64_t *nk, bool do_assign,
                          int do_update, int64_t *changed, cudaStream_t s);
// Adaptive pass (sk_kmeans_step_auto): full or incremental sums, chosen on
// the device from state[0], the previous pass's count of changed labels.
cudaError_t launch_kmeans_auto(const sk_ctx &c, const int32_t *idx, const float *val,
                               int64_t n, const float *mu, int K, int32_t *labels, float *dist,
                               double *S, int32_t *cnt, int64_t *nk, int64_t *state, int first,
                               cudaStream_t s);
cudaError_t launch_kmeans_finalize(const sk_ctx &c, int K, const double *S,
                                   const int32_t *cnt, float *mu, cudaStream_t s);
cudaError_t launch_gram_fp32(const sk_ctx &c, const int32_t *idx, const float *val,
                             int64_t n, double *G, cudaStream_t s);
cudaError_t launch_gram_tc(const sk_ctx &c, int mode, const int32_t *idx,
                           const float *val, int64_t n, double *G, void *work, cudaStream_t s);
int64_t gram_tc_workspace(const sk_ctx &c, int64_t n);
// mean == NULL: C_n; else the centred estimate with mean the sample-mean estimate
cudaError_t launch_cov_finalize(const sk_ctx &c, const double *G, int64_t n_total,
                                const double *mean, double *C, cudaStream_t s);
cudaError_t launch_unmix(const sk_ctx &c, const void *in, int64_t r, void *out,
                         bool f64, cudaStream_t s);
// K-means++ seeding and the objective J' (kmeanspp.cu).
int64_t kmeanspp_workspace(int64_t n);
cudaError_t launch_kmeanspp(const sk_ctx &c, const int32_t *idx, const float *val, int64_t n,
                            int K, uint32_t restart, float *mu, int64_t *rows, void *work,
                            cudaStream_t s);
cudaError_t launch_objective(const float *dist, int64_t n, double *J, cudaStream_t s);
cudaError_t launch_kmeans_hk(const sk_ctx &c, int K, const int32_t *cnt, const int64_t *nk,
                             double *dev, cudaStream_t s);
// Algorithm 2's second pass and the sample mean (extras.cu).
cudaError_t launch_kmeans2_assign(const sk_ctx &c, const float *X, int64_t n, int64_t ldx,
                                  const float *mu, int K, int32_t *labels, float *dist,
                                  cudaStream_t s);
cudaError_t launch_kmeans2_sums(const sk_ctx &c, const float *X, int64_t n, int64_t ldx,
                                const int32_t *labels, int K, double *sums, int64_t *counts,
                                cudaStream_t s);
cudaError_t launch_kmeans2_finalize(const sk_ctx &c, int K, const double *sums,
                                    const int64_t *counts, float *mu, cudaStream_t s);
cudaError_t launch_mean_accumulate(const sk_ctx &c, const int32_t *idx, const float *val,
                                   int64_t n, double *sums, cudaStream_t s);
cudaError_t launch_mean_finalize(const sk_ctx &c, const double *sums, int64_t n_total,
                                 double *mean, cudaStream_t s);
cudaError_t launch_topk(const sk_ctx &c, const double *C, int k, int iters,
                        double *evals, double *U, double *work, cudaStream_t s);
int64_t topk_workspace(int64_t pt, int k);
// Fixed top-k scratch (a static device array of topk_static_capacity() doubles):
// its device address for the current device (looked up on every call).
int64_t topk_static_capacity();
cudaError_t topk_static_scratch(double **out);
// Limit of the kernels' bounded device waits, in SM clock cycles (default
// 4e9, about 2 s; sk_debug_set_wait_cycles changes it for later launches).
long long wait_limit_cycles();
// Reads and clears the device error word of the kernels with bounded waits
// (bit 0: an mbarrier wait ran out).  Returns cudaSuccess or the copy error.
cudaError_t take_device_error(unsigned int *flag);
// Device address of the error word (NULL if it cannot be resolved).
unsigned int *device_error_word();
}  // namespace sk
