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
// Bank-disjoint centre copies: with LPR <= 16 the rows of a warp are laid out
// per half-warp (G = 16 / LPR row slots in each half).  When the table fits,
// coordinate j owns one 32-word line of shared memory holding G copies of its
// Kpad centre values, copy s at words s*Kpad .. s*Kpad + Kpad - 1; the row in
// slot s reads copy s.  The G rows of a half-warp then touch disjoint banks
// whatever their coordinates, so a centre load is one wavefront per half-warp
// instead of a random number of conflicting ones.
//
// Update: in the same pass, each (row, t) entry adds val to S[label][idx] and
// 1 to cnt[label][idx] in CTA-private shared-memory accumulators, flushed to
// the caller's float64 / int32 sums with one atomic per touched entry.
#include "sk_internal.cuh"

namespace sk {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = 1024;
constexpr int kWarpsK = kThreads / 32;

struct KmParams {
    const int32_t *idx;
    const float *val;
    int64_t n;
    int m;
    int pt;
    int K, Kpad, LPR, RW;
    int G;          // row slots per half-warp (0: rows laid out over the whole warp)
    int stage_cap;  // staged (idx, val) entries per warp
    const float *mu;
    int32_t *labels;
    float *dist;
    double *S;
    int32_t *cnt;
    int64_t *nk;
    unsigned long long *changed;  // delta mode: rows whose label changed (may be NULL)
    int do_assign;
    int do_update;  // 0 none, 1 full sums, 2 incremental (changed rows only)
};

// Packed FP32 pairs (two independent IEEE round-to-nearest operations).
__device__ __forceinline__ uint64_t pack2(float lo, float hi) {
    return ((uint64_t)__float_as_uint(hi) << 32) | __float_as_uint(lo);
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t sqacc2(uint64_t d, uint64_t acc) {
    uint64_t r;
    asm("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(r) : "l"(d), "l"(acc));
    return r;
}

// Lane of the first centre group of row slot rs, and row slot of a lane.
__device__ __forceinline__ int lead_lane(const KmParams &P, int rs) {
    return P.G ? (rs / P.G) * 16 + (rs % P.G) * P.LPR : rs * P.LPR;
}
__device__ __forceinline__ int slot_of_lane(const KmParams &P, int l) {
    return P.G ? (l >> 4) * P.G + (l & 15) / P.LPR : l / P.LPR;
}

template <int KPL, bool MU_SMEM, bool PRIV, bool STAGE, bool COPIES>
__global__ void __launch_bounds__(kThreads) kmeans_kernel(KmParams P) {
    constexpr int NP = KPL / 2;  // packed pairs per lane
    extern __shared__ __align__(16) unsigned char smem_raw[];
    size_t off = 0;
    float *mus = reinterpret_cast<float *>(smem_raw + off);
    if (MU_SMEM && P.do_assign) off += (size_t)P.pt * (COPIES ? 32 : P.Kpad) * 4;
    float *sS = reinterpret_cast<float *>(smem_raw + off);
    int32_t *sC = reinterpret_cast<int32_t *>(smem_raw + off + (size_t)P.K * P.pt * 4);
    int32_t *snk = reinterpret_cast<int32_t *>(smem_raw + off + (size_t)P.K * P.pt * 8);
    if (PRIV && P.do_update == 1) off += (size_t)P.K * P.pt * 8 + (((size_t)P.K * 4 + 15) & ~(size_t)15);
    int2 *stage_all = reinterpret_cast<int2 *>(smem_raw + off);

    const int tid = threadIdx.x;
    const int KP = P.K * P.pt;
    if (MU_SMEM && P.do_assign) {
        if constexpr (COPIES) {
            for (int e = tid; e < P.pt * 32; e += blockDim.x) {
                const int j = e >> 5, w = e & 31;
                const int c = w / P.Kpad, k = w - c * P.Kpad;
                mus[e] = (c < P.G && k < P.K) ? P.mu[(int64_t)k * P.pt + j] : 0.f;
            }
        } else {
            for (int e = tid; e < P.pt * P.Kpad; e += blockDim.x) {
                const int j = e / P.Kpad, k = e - j * P.Kpad;
                mus[e] = (k < P.K) ? P.mu[(int64_t)k * P.pt + j] : 0.f;
            }
        }
    }
    if (PRIV && P.do_update == 1) {
        for (int e = tid; e < KP; e += blockDim.x) {
            sS[e] = 0.f;
            sC[e] = 0;
        }
        for (int e = tid; e < P.K; e += blockDim.x) snk[e] = 0;
    }
    __syncthreads();

    const int lane = tid & 31, warp = tid >> 5;
    // row slot of this lane in the warp, its centre group, and (per half-warp
    // layout) the slot's position in its half, which selects the copy
    int sub, kl, hs = 0;
    bool lane_used;
    if (P.G) {
        hs = (lane & 15) / P.LPR;
        sub = (lane >> 4) * P.G + hs;
        kl = (lane & 15) - hs * P.LPR;
        lane_used = hs < P.G;
    } else {
        sub = lane / P.LPR;
        kl = lane - sub * P.LPR;
        lane_used = sub < P.RW;
    }
    const int kbase = kl * KPL;
    int2 *stage = stage_all + (size_t)warp * P.stage_cap;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + tid) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int m = P.m;
    const int pmask = P.pt - 1;

    for (int64_t base = gwarp * P.RW; base < P.n; base += nwarps * P.RW) {
        const int rows_here = (int)((P.n - base) < P.RW ? (P.n - base) : P.RW);
        if constexpr (STAGE) {
            // this pass's rows are contiguous in the ELL arrays: coalesced copy
            const int total = rows_here * m;
            const int32_t *gi = P.idx + base * m;
            const float *gv = P.val + base * m;
            for (int e = lane; e < total; e += 32)
                stage[e] = make_int2(__ldg(gi + e), __float_as_int(__ldg(gv + e)));
            __syncwarp();
        }
        const int64_t i = base + sub;
        const bool row_ok = lane_used && sub < rows_here;
        int label = 0;
        // previous label (incremental mode), loaded before the distance loop so
        // the load latency overlaps it
        int old_pref = -1;
        if (P.do_update == 2 && row_ok && kl == 0) old_pref = P.labels[i];
        if (P.do_assign) {
            uint64_t acc[NP];
#pragma unroll
            for (int q = 0; q < NP; ++q) acc[q] = 0ull;
            if (row_ok) {
                const int2 *rs = stage + sub * m;
                const int32_t *ri = P.idx + i * m;
                const float *rv = P.val + i * m;
#pragma unroll 4
                for (int t = 0; t < m; ++t) {
                    int j;
                    float v;
                    if constexpr (STAGE) {
                        const int2 iv = rs[t];
                        j = iv.x & pmask;  // indices outside [0, pt) wrap
                        v = __int_as_float(iv.y);
                    } else {
                        j = __ldg(ri + t) & pmask;
                        v = __ldg(rv + t);
                    }
                    const uint64_t vv = pack2(v, v);
                    if constexpr (MU_SMEM) {
                        const float *line = COPIES ? mus + j * 32 + hs * P.Kpad : mus + j * P.Kpad;
                        const uint64_t *c = reinterpret_cast<const uint64_t *>(line + kbase);
#pragma unroll
                        for (int q = 0; q < NP; ++q) acc[q] = sqacc2(sub2(vv, c[q]), acc[q]);
                    } else {
#pragma unroll
                        for (int q = 0; q < NP; ++q) {
                            const int k0 = kbase + 2 * q;
                            const float c0 = (k0 < P.K) ? __ldg(P.mu + (int64_t)k0 * P.pt + j) : 0.f;
                            const float c1 = (k0 + 1 < P.K) ? __ldg(P.mu + (int64_t)(k0 + 1) * P.pt + j) : 0.f;
                            acc[q] = sqacc2(sub2(vv, pack2(c0, c1)), acc[q]);
                        }
                    }
                }
            }
            // local argmin over this lane's centres (ascending k, strict <)
            float bd = INFINITY;
            int bk = 0x7fffffff;
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const float d0 = __uint_as_float((uint32_t)acc[q]);
                const float d1 = __uint_as_float((uint32_t)(acc[q] >> 32));
                const int k0 = kbase + 2 * q;
                if (k0 < P.K && d0 < bd) {
                    bd = d0;
                    bk = k0;
                }
                if (k0 + 1 < P.K && d1 < bd) {
                    bd = d1;
                    bk = k0 + 1;
                }
            }
            // argmin across the LPR lanes of the row (ties to the smaller k)
            const int lead = lane_used ? lead_lane(P, sub) : 32;
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
            int old = old_pref;
            if (row_ok && kl == 0) {
                P.labels[i] = label;
                if (P.dist) P.dist[i] = bd;
            }
            if (P.do_update == 2) {
                // incremental sums: a row whose label moved from old to label
                // leaves cluster old and joins cluster label (exact in FP64 for
                // float inputs up to rounding of the running sums)
                old = __shfl_sync(kFull, old, (lead < 32) ? lead : lane);
                const bool moved = row_ok && kl == 0 && old != label;
                const unsigned mv = __ballot_sync(kFull, moved);
                if (P.changed && lane == 0 && mv)
                    atomicAdd(P.changed, (unsigned long long)__popc(mv));
                unsigned pending = mv;
                while (pending) {
                    const int src = __ffs(pending) - 1;
                    pending &= pending - 1;
                    const int rs = slot_of_lane(P, src);
                    const int newl = __shfl_sync(kFull, label, src);
                    const int oldl = __shfl_sync(kFull, old, src);
                    for (int t = lane; t < m; t += 32) {
                        int j;
                        float v;
                        if constexpr (STAGE) {
                            const int2 iv = stage[rs * m + t];
                            j = iv.x & pmask;
                            v = __int_as_float(iv.y);
                        } else {
                            j = __ldg(P.idx + (base + rs) * m + t) & pmask;
                            v = __ldg(P.val + (base + rs) * m + t);
                        }
                        if (PRIV && P.do_update == 1) {
                            atomicAdd(sS + newl * P.pt + j, v);
                            atomicAdd(sC + newl * P.pt + j, 1);
                            if ((unsigned)oldl < (unsigned)P.K) {
                                atomicAdd(sS + oldl * P.pt + j, -v);
                                atomicAdd(sC + oldl * P.pt + j, -1);
                            }
                        } else {
                            atomicAdd(P.S + (int64_t)newl * P.pt + j, (double)v);
                            atomicAdd(P.cnt + (int64_t)newl * P.pt + j, 1);
                            if ((unsigned)oldl < (unsigned)P.K) {
                                atomicAdd(P.S + (int64_t)oldl * P.pt + j, -(double)v);
                                atomicAdd(P.cnt + (int64_t)oldl * P.pt + j, -1);
                            }
                        }
                    }
                    if (lane == 0) {
                        if (PRIV && P.do_update == 1) {
                            atomicAdd(snk + newl, 1);
                            if ((unsigned)oldl < (unsigned)P.K) atomicAdd(snk + oldl, -1);
                        } else {
                            atomicAdd(reinterpret_cast<unsigned long long *>(P.nk + newl), 1ull);
                            if ((unsigned)oldl < (unsigned)P.K)
                                atomicAdd(reinterpret_cast<unsigned long long *>(P.nk + oldl),
                                          (unsigned long long)(-1LL));
                        }
                    }
                }
            }
        }
        if (P.do_update == 1) {
            for (int rs = 0; rs < rows_here; ++rs) {
                int lab;
                if (P.do_assign) {
                    lab = __shfl_sync(kFull, label, lead_lane(P, rs));
                } else {
                    lab = __ldg(P.labels + base + rs);
                }
                if ((unsigned)lab >= (unsigned)P.K) continue;  // invalid caller label: skipped
                const int64_t ii = base + rs;
                for (int t = lane; t < m; t += 32) {
                    int j;
                    float v;
                    if constexpr (STAGE) {
                        const int2 iv = stage[rs * m + t];
                        j = iv.x & pmask;
                        v = __int_as_float(iv.y);
                    } else {
                        j = __ldg(P.idx + ii * m + t) & pmask;
                        v = __ldg(P.val + ii * m + t);
                    }
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
        if constexpr (STAGE) __syncwarp();  // stage is rewritten by the next pass
    }
    if (PRIV && P.do_update == 1) {
        __syncthreads();
        // a slot can carry a nonzero float sum with a zero net count (a row
        // that left and another that joined): flush both independently
        for (int e = tid; e < KP; e += blockDim.x) {
            const int c = sC[e];
            const float x = sS[e];
            if (x != 0.f) atomicAdd(P.S + e, (double)x);
            if (c) atomicAdd(P.cnt + e, c);
        }
        for (int e = tid; e < P.K; e += blockDim.x)
            if (snk[e]) atomicAdd(reinterpret_cast<unsigned long long *>(P.nk + e),
                                  (unsigned long long)(long long)snk[e]);
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

template <int KPL, bool MU_SMEM, bool PRIV, bool STAGE, bool COPIES>
cudaError_t launch_variant(const KmParams &P, size_t smem, cudaStream_t s) {
    auto kern = kmeans_kernel<KPL, MU_SMEM, PRIV, STAGE, COPIES>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
    if (per_sm < 1) per_sm = 1;
    const int64_t warps_needed = (P.n + P.RW - 1) / P.RW;
    int64_t blocks = (warps_needed + kWarpsK - 1) / kWarpsK;
    if (blocks > (int64_t)sms * per_sm) blocks = (int64_t)sms * per_sm;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, kThreads, smem, s>>>(P);
    return cudaGetLastError();
}

template <int KPL, bool MU_SMEM, bool PRIV, bool COPIES = false>
cudaError_t launch_stage(KmParams &P, size_t fixed, size_t budget, cudaStream_t s) {
    const size_t stage_b = (size_t)kWarpsK * P.RW * P.m * 8;
    if (fixed + stage_b <= budget) {
        P.stage_cap = P.RW * P.m;
        return launch_variant<KPL, MU_SMEM, PRIV, true, COPIES>(P, fixed + stage_b, s);
    }
    P.stage_cap = 0;
    return launch_variant<KPL, MU_SMEM, PRIV, false, COPIES>(P, fixed, s);
}

template <int KPL>
cudaError_t launch_kpl(KmParams &P, cudaStream_t s) {
    P.LPR = (P.K + KPL - 1) / KPL;
    P.Kpad = P.LPR * KPL;
    // rows per half-warp when a row needs at most 16 lanes
    P.G = P.LPR <= 16 ? 16 / P.LPR : 0;
    P.RW = P.G ? 2 * P.G : 32 / P.LPR;
    int dev = 0, smem_max = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if constexpr (KPL == 2) {
        // bank-disjoint copies: worth it with two or more rows per half-warp,
        // when the assignment runs without the shared-memory update sums and
        // the 32-word lines plus the row staging fit
        const size_t lines_b = (size_t)P.pt * 32 * 4;
        const size_t stage_b = (size_t)kWarpsK * P.RW * P.m * 8;
        if (P.do_assign && P.do_update != 1 && P.G >= 2 && lines_b + stage_b <= (size_t)smem_max)
            return launch_stage<KPL, true, false, true>(P, lines_b, (size_t)smem_max, s);
    }
    const size_t mu_b = P.do_assign ? (size_t)P.pt * P.Kpad * 4 : 0;
    // the incremental mode touches only rows whose label changed (few after the
    // first passes): it adds straight into the global sums and keeps the
    // assignment's shared-memory footprint small (room in L1 for the loads)
    const size_t priv_b =
        P.do_update == 1 ? (size_t)P.K * P.pt * 8 + (((size_t)P.K * 4 + 15) & ~(size_t)15) : 0;
    const size_t budget = (size_t)smem_max;
    if (mu_b + priv_b <= budget) return launch_stage<KPL, true, true>(P, mu_b + priv_b, budget, s);
    if (mu_b <= budget) return launch_stage<KPL, true, false>(P, mu_b, budget, s);
    if (priv_b <= budget) return launch_stage<KPL, false, true>(P, priv_b, budget, s);
    return launch_stage<KPL, false, false>(P, 0, budget, s);
}

}  // namespace

cudaError_t launch_kmeans(const sk_ctx &c, const int32_t *idx, const float *val,
                          int64_t n, const float *mu, int K, int32_t *labels, float *dist,
                          double *S, int32_t *cnt, int64_t *nk, bool do_assign,
                          int do_update, int64_t *changed, cudaStream_t s) {
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
    P.changed = reinterpret_cast<unsigned long long *>(changed);
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
