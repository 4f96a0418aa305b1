// kmeans.cu -- sparsified K-means assign and centre-update passes (Sec. VI-B,
// Eqs. (assignments), (mu_update_one), (mu_update_two)).
//
// Assignment: a row's restricted distance to centre k is
// sum_t (val_t - mu'_k[idx_t])^2 over its m sampled coordinates only.  A row
// is handled by LPR lanes, each owning KPL consecutive centres; the centres
// live in shared memory transposed to [pt][Kpad] so the lanes of one row read
// consecutive words of one coordinate (no bank conflicts inside a row).  Each
// lane accumulates its KPL distances directly -- a difference, then a fused
// multiply-add -- so no cross-lane reduction over t is needed; the argmin over
// the LPR lanes of a row (ties to the smallest k) takes a few shuffles.
//
// Update: in the same pass, each (row, t) entry adds val to S[label][idx] and
// 1 to cnt[label][idx] in CTA-private shared-memory accumulators, flushed to
// the caller's float64 / int32 sums with one atomic per touched entry.
#include "sk_internal.cuh"

namespace sk {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = 1024;

struct KmParams {
    const int32_t *idx;
    const float *val;
    int64_t n;
    int m;
    int pt;
    int K, Kpad, LPR, RW;
    const float *mu;
    int32_t *labels;
    float *dist;
    double *S;
    int32_t *cnt;
    int64_t *nk;
    int do_assign, do_update;
};

template <int KPL, bool MU_SMEM, bool PRIV>
__global__ void __launch_bounds__(kThreads) kmeans_kernel(KmParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *mus = reinterpret_cast<float *>(smem_raw);
    const size_t mu_bytes = (MU_SMEM && P.do_assign) ? (size_t)P.pt * P.Kpad * 4 : 0;
    float *sS = reinterpret_cast<float *>(smem_raw + mu_bytes);
    int32_t *sC = reinterpret_cast<int32_t *>(smem_raw + mu_bytes + (PRIV ? (size_t)P.K * P.pt * 4 : 0));
    int32_t *snk = reinterpret_cast<int32_t *>(smem_raw + mu_bytes + (PRIV ? (size_t)P.K * P.pt * 8 : 0));

    const int tid = threadIdx.x;
    const int KP = P.K * P.pt;
    if (MU_SMEM && P.do_assign) {
        for (int e = tid; e < P.pt * P.Kpad; e += blockDim.x) {
            const int j = e / P.Kpad, k = e - j * P.Kpad;
            mus[e] = (k < P.K) ? P.mu[(int64_t)k * P.pt + j] : 0.f;
        }
    }
    if (PRIV && P.do_update) {
        for (int e = tid; e < KP; e += blockDim.x) {
            sS[e] = 0.f;
            sC[e] = 0;
        }
        for (int e = tid; e < P.K; e += blockDim.x) snk[e] = 0;
    }
    __syncthreads();

    const int lane = tid & 31;
    const int sub = lane / P.LPR;            // row slot of this lane in the warp
    const int kl = lane - sub * P.LPR;       // centre group of this lane
    const int kbase = kl * KPL;
    const bool lane_used = sub < P.RW;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + tid) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int m = P.m;

    for (int64_t base = gwarp * P.RW; base < P.n; base += nwarps * P.RW) {
        const int64_t i = base + sub;
        const bool row_ok = lane_used && i < P.n;
        int label = 0;
        if (P.do_assign) {
            float acc[KPL];
#pragma unroll
            for (int q = 0; q < KPL; ++q) acc[q] = 0.f;
            if (row_ok) {
                const int32_t *ri = P.idx + i * m;
                const float *rv = P.val + i * m;
#pragma unroll 4
                for (int t = 0; t < m; ++t) {
                    // indices outside [0, pt) (not produced by sk_compress) wrap
                    const int j = __ldg(ri + t) & (P.pt - 1);
                    const float v = __ldg(rv + t);
                    if constexpr (MU_SMEM) {
                        const float *c = mus + j * P.Kpad + kbase;
#pragma unroll
                        for (int q = 0; q < KPL; q += 2) {
                            const float2 c2 = *reinterpret_cast<const float2 *>(c + q);
                            const float d0 = v - c2.x, d1 = v - c2.y;
                            acc[q] = fmaf(d0, d0, acc[q]);
                            acc[q + 1] = fmaf(d1, d1, acc[q + 1]);
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < KPL; ++q) {
                            const int k = kbase + q;
                            const float c = (k < P.K) ? __ldg(P.mu + (int64_t)k * P.pt + j) : 0.f;
                            const float d = v - c;
                            acc[q] = fmaf(d, d, acc[q]);
                        }
                    }
                }
            }
            // local argmin over this lane's centres (ascending k: strict < keeps the first)
            float bd = INFINITY;
            int bk = 0x7fffffff;
#pragma unroll
            for (int q = 0; q < KPL; ++q) {
                const int k = kbase + q;
                if (k < P.K && acc[q] < bd) {
                    bd = acc[q];
                    bk = k;
                }
            }
            // argmin across the LPR lanes of the row: the row's first lane gathers
            const int lead = sub * P.LPR;
            for (int o = 1; o < P.LPR; ++o) {
                const int srcl = (lead + o < 32) ? lead + o : lane;
                const float od = __shfl_sync(kFull, bd, srcl);
                const int ok = __shfl_sync(kFull, bk, srcl);
                if (kl == 0 && (od < bd || (od == bd && ok < bk))) {
                    bd = od;
                    bk = ok;
                }
            }
            const int leadl = (lead < 32) ? lead : lane;
            bd = __shfl_sync(kFull, bd, leadl);
            bk = __shfl_sync(kFull, bk, leadl);
            label = bk;
            if (row_ok && kl == 0) {
                P.labels[i] = label;
                if (P.dist) P.dist[i] = bd;
            }
        }
        if (P.do_update) {
            // labels of this warp's RW rows: slot sub's label lives in lane sub*LPR
            const int rows_here = (int)((P.n - base) < P.RW ? (P.n - base) : P.RW);
            for (int rs = 0; rs < rows_here; ++rs) {
                int lab;
                if (P.do_assign) {
                    lab = __shfl_sync(kFull, label, rs * P.LPR);
                } else {
                    lab = __ldg(P.labels + base + rs);
                }
                if ((unsigned)lab >= (unsigned)P.K) continue;  // invalid caller label: skipped
                const int64_t ii = base + rs;
                const int32_t *ri = P.idx + ii * m;
                const float *rv = P.val + ii * m;
                for (int t = lane; t < m; t += 32) {
                    const int j = __ldg(ri + t) & (P.pt - 1);
                    const float v = __ldg(rv + t);
                    const int64_t slot = (int64_t)lab * P.pt + j;
                    if constexpr (PRIV) {
                        atomicAdd(sS + slot, v);
                        atomicAdd(sC + slot, 1);
                    } else {
                        atomicAdd(P.S + slot, (double)v);
                        atomicAdd(P.cnt + slot, 1);
                    }
                }
                if (lane == 0) {
                    if constexpr (PRIV) {
                        atomicAdd(snk + lab, 1);
                    } else {
                        atomicAdd(reinterpret_cast<unsigned long long *>(P.nk + lab), 1ull);
                    }
                }
            }
        }
    }
    if (PRIV && P.do_update) {
        __syncthreads();
        for (int e = tid; e < KP; e += blockDim.x) {
            const int c = sC[e];
            if (c) {
                atomicAdd(P.S + e, (double)sS[e]);
                atomicAdd(P.cnt + e, c);
            }
        }
        for (int e = tid; e < P.K; e += blockDim.x)
            if (snk[e]) atomicAdd(reinterpret_cast<unsigned long long *>(P.nk + e),
                                  (unsigned long long)snk[e]);
    }
}

__global__ void kmeans_finalize_kernel(int64_t KP, const double *S, const int32_t *cnt,
                                       float *mu) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < KP;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = cnt[e];
        if (c > 0) mu[e] = (float)(S[e] / (double)c);
    }
}

template <int KPL, bool MU_SMEM, bool PRIV>
cudaError_t launch_variant(const KmParams &P, size_t smem, cudaStream_t s) {
    auto kern = kmeans_kernel<KPL, MU_SMEM, PRIV>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t warps_needed = (P.n + P.RW - 1) / P.RW;
    int64_t blocks = (warps_needed + 31) / 32;
    if (blocks > sms) blocks = sms;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, kThreads, smem, s>>>(P);
    return cudaGetLastError();
}

template <int KPL>
cudaError_t launch_kpl(KmParams &P, cudaStream_t s) {
    P.LPR = (P.K + KPL - 1) / KPL;
    P.Kpad = P.LPR * KPL;
    P.RW = 32 / P.LPR;
    int dev = 0, smem_max = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t mu_b = P.do_assign ? (size_t)P.pt * P.Kpad * 4 : 0;
    const size_t priv_b = P.do_update ? (size_t)P.K * P.pt * 8 + (size_t)P.K * 4 : 0;
    const size_t budget = (size_t)smem_max;
    if (mu_b + priv_b <= budget) return launch_variant<KPL, true, true>(P, mu_b + priv_b, s);
    if (mu_b <= budget) return launch_variant<KPL, true, false>(P, mu_b, s);
    if (priv_b <= budget) return launch_variant<KPL, false, true>(P, priv_b, s);
    return launch_variant<KPL, false, false>(P, 0, s);
}

}  // namespace

cudaError_t launch_kmeans(const sk_ctx &c, const int32_t *idx, const float *val,
                          int64_t n, const float *mu, int K, int32_t *labels, float *dist,
                          double *S, int32_t *cnt, int64_t *nk, bool do_assign,
                          bool do_update, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    KmParams P;
    P.idx = idx;
    P.val = val;
    P.n = n;
    P.m = (int)c.m;
    P.pt = (int)c.pt;
    P.K = K;
    P.mu = mu;
    P.labels = labels;
    P.dist = dist;
    P.S = S;
    P.cnt = cnt;
    P.nk = nk;
    P.do_assign = do_assign;
    P.do_update = do_update;
    if (K <= 64) return launch_kpl<2>(P, s);
    if (K <= 128) return launch_kpl<4>(P, s);
    return launch_kpl<8>(P, s);
}

cudaError_t launch_kmeans_finalize(const sk_ctx &c, int K, const double *S,
                                   const int32_t *cnt, float *mu, cudaStream_t s) {
    const int64_t KP = (int64_t)K * c.pt;
    int blocks = (int)((KP + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    kmeans_finalize_kernel<<<blocks, 256, 0, s>>>(KP, S, cnt, mu);
    return cudaGetLastError();
}

}  // namespace sk
