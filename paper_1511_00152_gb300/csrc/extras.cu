// extras.cu -- the second pass of the 2-pass sparsified K-means (Algorithm 2)
// and the sample-mean estimator (Sec. IV).
//
// Algorithm 2 re-reads the raw rows once: every row is assigned to the nearest
// 1-pass centre (dense squared distance over all p coordinates, in the data
// domain) and added to the mean of its *1-pass* cluster.  Both are streams
// over X (4 p bytes per row), so both are HBM-bound:
//   * dense_assign_kernel: a warp per group of kRowsPerWarp rows, lanes over
//     coordinates (16-byte loads when aligned).  The centres sit in shared
//     memory when K p floats fit (else they are read through L1/L2); each
//     centre element loaded is used for kRowsPerWarp rows.  Per-lane partial
//     distances are reduced across the warp; ties go to the smallest k.
//   * dense_sums_kernel: a CTA per (1024-column block, kSumRows-row block);
//     each thread owns 4 columns and adds a row's values into the shared-memory
//     sums of that row's cluster (FP32, at most kSumRows rows), which are then
//     added into the caller's FP64 sums.  Column block 0 also counts rows.
// The sample mean is (pt/m)(1/n) sum_i R_i R_i^T y_i: a scatter of the ELL
// values into CTA-private shared-memory sums, flushed with FP64 atomics.
#include "sk_internal.cuh"

namespace sk {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kRowsPerWarp = 4;
constexpr int kSumRows = 1024;    // rows per CTA of the sums kernel
constexpr int kSumCols = 1024;    // columns per CTA of the sums kernel
constexpr int kMaxSumK = 48;      // clusters per sums launch (48 x 4 KiB shared memory)
constexpr int kMeanRows = 4096;   // rows per CTA of the mean scatter

// KC: centres per register block (kRowsPerWarp x KC partial distances live in
// registers); the launcher picks the smallest of 4, 8, 12, 16 that covers K.
template <int KC, bool VEC, bool MU_SMEM>
__global__ void __launch_bounds__(256, 2) dense_assign_kernel(const float *__restrict__ X, int64_t n,
                                                          int p, int64_t ldx,
                                                          const float *__restrict__ mu, int K,
                                                          int32_t *labels, float *dist) {
    extern __shared__ __align__(16) float smu[];
    if constexpr (MU_SMEM) {
        for (int e = threadIdx.x; e < K * p; e += blockDim.x) smu[e] = mu[e];
        __syncthreads();
    }
    const float *cen = MU_SMEM ? smu : mu;
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t ngroups = (n + kRowsPerWarp - 1) / kRowsPerWarp;
    for (int64_t g = gw; g < ngroups; g += nw) {
        const int64_t i0 = g * kRowsPerWarp;
        float bd[kRowsPerWarp];
        int bk[kRowsPerWarp];
#pragma unroll
        for (int r = 0; r < kRowsPerWarp; ++r) {
            bd[r] = INFINITY;
            bk[r] = 0;
        }
        for (int k0 = 0; k0 < K; k0 += KC) {
            float d[kRowsPerWarp][KC];
#pragma unroll
            for (int r = 0; r < kRowsPerWarp; ++r)
#pragma unroll
                for (int q = 0; q < KC; ++q) d[r][q] = 0.f;
            if constexpr (VEC) {
                for (int j = 4 * lane; j < p; j += 128) {
                    float4 x4[kRowsPerWarp];
#pragma unroll
                    for (int r = 0; r < kRowsPerWarp; ++r)
                        x4[r] = (i0 + r < n) ? __ldcs(reinterpret_cast<const float4 *>(
                                                   X + (i0 + r) * ldx + j))
                                             : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int q = 0; q < KC; ++q) {
                        if (k0 + q < K) {
                            const float4 c4 =
                                *reinterpret_cast<const float4 *>(cen + (int64_t)(k0 + q) * p + j);
#pragma unroll
                            for (int r = 0; r < kRowsPerWarp; ++r) {
                                float t = x4[r].x - c4.x;
                                d[r][q] = fmaf(t, t, d[r][q]);
                                t = x4[r].y - c4.y;
                                d[r][q] = fmaf(t, t, d[r][q]);
                                t = x4[r].z - c4.z;
                                d[r][q] = fmaf(t, t, d[r][q]);
                                t = x4[r].w - c4.w;
                                d[r][q] = fmaf(t, t, d[r][q]);
                            }
                        }
                    }
                }
            } else {
                for (int j = lane; j < p; j += 32) {
                    float xv[kRowsPerWarp];
#pragma unroll
                    for (int r = 0; r < kRowsPerWarp; ++r)
                        xv[r] = (i0 + r < n) ? __ldcs(X + (i0 + r) * ldx + j) : 0.f;
#pragma unroll
                    for (int q = 0; q < KC; ++q) {
                        if (k0 + q < K) {
                            const float c = cen[(int64_t)(k0 + q) * p + j];
#pragma unroll
                            for (int r = 0; r < kRowsPerWarp; ++r) {
                                const float t = xv[r] - c;
                                d[r][q] = fmaf(t, t, d[r][q]);
                            }
                        }
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < kRowsPerWarp; ++r)
#pragma unroll
                for (int q = 0; q < KC; ++q) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) d[r][q] += __shfl_xor_sync(kFull, d[r][q], o);
                    // strict < keeps the smallest k among equal distances
                    if (k0 + q < K && d[r][q] < bd[r]) {
                        bd[r] = d[r][q];
                        bk[r] = k0 + q;
                    }
                }
        }
        if (lane < kRowsPerWarp) {
            float dd = bd[0];
            int kk = bk[0];
#pragma unroll
            for (int r = 1; r < kRowsPerWarp; ++r)
                if (lane == r) {
                    dd = bd[r];
                    kk = bk[r];
                }
            if (i0 + lane < n) {
                labels[i0 + lane] = kk;
                if (dist) dist[i0 + lane] = dd;
            }
        }
    }
}

// Columns of this thread within its 1024-column block: 4*t..4*t+3 (VEC) or
// t, t+256, t+512, t+768.
template <bool VEC>
__device__ __forceinline__ int sum_col(int t, int q) {
    return VEC ? 4 * t + q : t + 256 * q;
}

template <bool VEC>
__global__ void __launch_bounds__(256) dense_sums_kernel(const float *__restrict__ X, int64_t n,
                                                        int p, int64_t ldx,
                                                        const int32_t *__restrict__ labels,
                                                        int k0, int kc, double *sums,
                                                        int64_t *counts) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *sacc = reinterpret_cast<float *>(smem_raw);                       // kc x 1024
    int *slab = reinterpret_cast<int *>(smem_raw + (size_t)kc * kSumCols * 4);  // kSumRows
    int *scnt = slab + kSumRows;                                             // kc
    const int t = threadIdx.x;
    const int c0 = blockIdx.x * kSumCols;
    const int64_t r0 = (int64_t)blockIdx.y * kSumRows;
    const int rows = (int)((n - r0) < kSumRows ? (n - r0) : kSumRows);
    for (int e = t; e < kc * kSumCols; e += blockDim.x) sacc[e] = 0.f;
    for (int e = t; e < kc; e += blockDim.x) scnt[e] = 0;
    for (int e = t; e < rows; e += blockDim.x) slab[e] = __ldg(labels + r0 + e) - k0;
    __syncthreads();
    bool live[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) live[q] = c0 + sum_col<VEC>(t, q) < p;
    const bool vec_live = VEC && live[0];  // p % 4 == 0: all four or none
    constexpr int U = 4;
    for (int b = 0; b < rows; b += U) {
        float4 x4[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            x4[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (b + u < rows) {
                const float *src = X + (r0 + b + u) * ldx + c0;
                if constexpr (VEC) {
                    if (vec_live) x4[u] = __ldcs(reinterpret_cast<const float4 *>(src + 4 * t));
                } else {
                    if (live[0]) x4[u].x = __ldcs(src + t);
                    if (live[1]) x4[u].y = __ldcs(src + t + 256);
                    if (live[2]) x4[u].z = __ldcs(src + t + 512);
                    if (live[3]) x4[u].w = __ldcs(src + t + 768);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (b + u >= rows) break;
            const int lab = slab[b + u];
            if ((unsigned)lab < (unsigned)kc) {
                float *a = sacc + (size_t)lab * kSumCols;
                if constexpr (VEC) {
                    float4 s4 = *reinterpret_cast<float4 *>(a + 4 * t);
                    s4.x += x4[u].x;
                    s4.y += x4[u].y;
                    s4.z += x4[u].z;
                    s4.w += x4[u].w;
                    *reinterpret_cast<float4 *>(a + 4 * t) = s4;
                } else {
                    a[t] += x4[u].x;
                    a[t + 256] += x4[u].y;
                    a[t + 512] += x4[u].z;
                    a[t + 768] += x4[u].w;
                }
            }
        }
    }
    if (blockIdx.x == 0) {
        for (int e = t; e < rows; e += blockDim.x) {
            const int lab = slab[e];
            if ((unsigned)lab < (unsigned)kc) atomicAdd(scnt + lab, 1);
        }
    }
    __syncthreads();
    for (int e = t; e < kc * kSumCols; e += blockDim.x) {
        const int k = e / kSumCols, c = c0 + (e % kSumCols);
        if (c < p && sacc[e] != 0.f) atomicAdd(sums + (int64_t)(k0 + k) * p + c, (double)sacc[e]);
    }
    if (blockIdx.x == 0)
        for (int e = t; e < kc; e += blockDim.x)
            if (scnt[e])
                atomicAdd(reinterpret_cast<unsigned long long *>(counts + k0 + e),
                          (unsigned long long)scnt[e]);
}

// mu_k = sums_k / counts_k; an empty cluster keeps its 1-pass centre.
__global__ void dense_finalize_kernel(int64_t total, int p, const double *sums,
                                      const int64_t *counts, float *mu) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = counts[e / p];
        if (c > 0) mu[e] = (float)(sums[e] / (double)c);
    }
}

__global__ void __launch_bounds__(512) mean_scatter_kernel(const int32_t *__restrict__ idx,
                                                           const float *__restrict__ val,
                                                           int64_t n, int m, int pt,
                                                           double *sums) {
    extern __shared__ float ssum[];
    for (int e = threadIdx.x; e < pt; e += blockDim.x) ssum[e] = 0.f;
    __syncthreads();
    const int64_t r0 = (int64_t)blockIdx.x * kMeanRows;
    const int64_t r1 = (r0 + kMeanRows < n) ? r0 + kMeanRows : n;
    const int64_t e1 = r1 * m;
    for (int64_t e = r0 * m + threadIdx.x; e < e1; e += blockDim.x)
        atomicAdd(ssum + clamp_index(__ldg(idx + e), pt), __ldg(val + e));
    __syncthreads();
    for (int e = threadIdx.x; e < pt; e += blockDim.x)
        if (ssum[e] != 0.f) atomicAdd(sums + e, (double)ssum[e]);
}

__global__ void mean_finalize_kernel(int pt, double scale, const double *sums, double *mean) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < pt; e += gridDim.x * blockDim.x)
        mean[e] = scale * sums[e];
}

int num_sms() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

int smem_optin() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

template <int KC, bool VEC, bool MU_SMEM>
cudaError_t assign_launch(const sk_ctx &c, const float *X, int64_t n, int64_t ldx,
                          const float *mu, int K, int32_t *labels, float *dist, cudaStream_t s) {
    const size_t smem = MU_SMEM ? (size_t)K * c.p * 4 : 0;
    auto kern = dense_assign_kernel<KC, VEC, MU_SMEM>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
    if (per_sm < 1) per_sm = 1;
    const int64_t groups = (n + kRowsPerWarp - 1) / kRowsPerWarp;
    int64_t blocks = (groups + 7) / 8;
    const int64_t cap = (int64_t)num_sms() * per_sm;
    if (blocks > cap) blocks = cap;
    kern<<<(unsigned)blocks, 256, smem, s>>>(X, n, (int)c.p, ldx, mu, K, labels, dist);
    return cudaGetLastError();
}

// ||H_k - I||_2 per cluster: H_k (Eq. (Hkmk)) is diagonal with entries
// (pt/m) cnt[k][j] / n_k, so the norm is the largest |entry - 1|; -1 for an
// empty cluster.  One CTA per cluster.
__global__ void hk_kernel(const int32_t *cnt, const int64_t *nk, int pt, double ratio,
                          double *dev) {
    __shared__ double red[256];
    const int k = blockIdx.x;
    const int64_t n = nk[k];
    double worst = 0.0;
    if (n > 0)
        for (int j = threadIdx.x; j < pt; j += blockDim.x) {
            const double h = ratio * (double)cnt[(int64_t)k * pt + j] / (double)n;
            worst = fmax(worst, fabs(h - 1.0));
        }
    red[threadIdx.x] = worst;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + h]);
        __syncthreads();
    }
    if (threadIdx.x == 0) dev[k] = n > 0 ? red[0] : -1.0;
}

}  // namespace

cudaError_t launch_kmeans_hk(const sk_ctx &c, int K, const int32_t *cnt, const int64_t *nk,
                             double *dev, cudaStream_t s) {
    hk_kernel<<<K, 256, 0, s>>>(cnt, nk, (int)c.pt, (double)c.pt / (double)c.m, dev);
    return cudaGetLastError();
}

cudaError_t launch_kmeans2_assign(const sk_ctx &c, const float *X, int64_t n, int64_t ldx,
                                  const float *mu, int K, int32_t *labels, float *dist,
                                  cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const bool vec = ((reinterpret_cast<uintptr_t>(X) & 15) == 0) &&
                     ((reinterpret_cast<uintptr_t>(mu) & 15) == 0) && (c.p % 4 == 0) &&
                     (ldx % 4 == 0);
    // centres in shared memory when they leave room for a second CTA's worth
    const bool in_smem = (int64_t)K * c.p * 4 <= (int64_t)smem_optin() - 1024;
    if (vec && in_smem) {
        if (K <= 4) return assign_launch<4, true, true>(c, X, n, ldx, mu, K, labels, dist, s);
        if (K <= 8) return assign_launch<8, true, true>(c, X, n, ldx, mu, K, labels, dist, s);
        if (K <= 12) return assign_launch<12, true, true>(c, X, n, ldx, mu, K, labels, dist, s);
        return assign_launch<16, true, true>(c, X, n, ldx, mu, K, labels, dist, s);
    }
    if (vec) return assign_launch<16, true, false>(c, X, n, ldx, mu, K, labels, dist, s);
    return in_smem ? assign_launch<16, false, true>(c, X, n, ldx, mu, K, labels, dist, s)
                   : assign_launch<16, false, false>(c, X, n, ldx, mu, K, labels, dist, s);
}

static cudaError_t sums_launch(const sk_ctx &c, const float *X, int64_t n, int64_t ldx,
                        const int32_t *labels, int K, double *sums, int64_t *counts, bool vec,
                        cudaStream_t s);

cudaError_t launch_kmeans2_sums(const sk_ctx &c, const float *X, int64_t n, int64_t ldx,
                                const int32_t *labels, int K, double *sums, int64_t *counts,
                                cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const bool vec = ((reinterpret_cast<uintptr_t>(X) & 15) == 0) && (c.p % 4 == 0) &&
                     (ldx % 4 == 0);
    // grid.y is limited to 65535 row blocks: longer inputs go in several launches
    constexpr int64_t kLaunchRows = (int64_t)65535 * kSumRows;
    for (int64_t a = 0; a < n; a += kLaunchRows) {
        const int64_t na = (n - a) < kLaunchRows ? (n - a) : kLaunchRows;
        cudaError_t e = sums_launch(c, X + a * ldx, na, ldx, labels + a, K, sums, counts, vec, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static cudaError_t sums_launch(const sk_ctx &c, const float *X, int64_t n, int64_t ldx,
                        const int32_t *labels, int K, double *sums, int64_t *counts, bool vec,
                        cudaStream_t s) {
    const dim3 grid((unsigned)((c.p + kSumCols - 1) / kSumCols),
                    (unsigned)((n + kSumRows - 1) / kSumRows));
    for (int k0 = 0; k0 < K; k0 += kMaxSumK) {
        const int kc = (K - k0) < kMaxSumK ? (K - k0) : kMaxSumK;
        const size_t smem = (size_t)kc * kSumCols * 4 + (size_t)kSumRows * 4 + (size_t)kc * 4;
        cudaError_t e;
        if (vec) {
            e = cudaFuncSetAttribute(dense_sums_kernel<true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            dense_sums_kernel<true><<<grid, 256, smem, s>>>(X, n, (int)c.p, ldx, labels, k0, kc,
                                                            sums, counts);
        } else {
            e = cudaFuncSetAttribute(dense_sums_kernel<false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            dense_sums_kernel<false><<<grid, 256, smem, s>>>(X, n, (int)c.p, ldx, labels, k0, kc,
                                                             sums, counts);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_kmeans2_finalize(const sk_ctx &c, int K, const double *sums,
                                    const int64_t *counts, float *mu, cudaStream_t s) {
    const int64_t total = (int64_t)K * c.p;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    dense_finalize_kernel<<<(unsigned)blocks, 256, 0, s>>>(total, (int)c.p, sums, counts, mu);
    return cudaGetLastError();
}

cudaError_t launch_mean_accumulate(const sk_ctx &c, const int32_t *idx, const float *val,
                                   int64_t n, double *sums, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const size_t smem = (size_t)c.pt * 4;
    cudaError_t e = cudaFuncSetAttribute(mean_scatter_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (n + kMeanRows - 1) / kMeanRows;
    mean_scatter_kernel<<<(unsigned)blocks, 512, smem, s>>>(idx, val, n, (int)c.m, (int)c.pt, sums);
    return cudaGetLastError();
}

cudaError_t launch_mean_finalize(const sk_ctx &c, const double *sums, int64_t n_total,
                                 double *mean, cudaStream_t s) {
    const double scale = (double)c.pt / (double)c.m / (double)n_total;
    mean_finalize_kernel<<<(unsigned)((c.pt + 255) / 256), 256, 0, s>>>((int)c.pt, scale, sums,
                                                                       mean);
    return cudaGetLastError();
}

}  // namespace sk
