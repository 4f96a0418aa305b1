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
#include <algorithm>
#include <cstring>
#include <vector>

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
    float *mu_t;  // batch only: transposed centres pt x Kpad in global memory (or NULL)
    int32_t *labels;
    float *dist;
    double *S;
    int32_t *cnt;
    int64_t *nk;
    unsigned long long *changed;  // delta mode: rows whose label changed (may be NULL)
    int do_assign;
    int do_update;  // 0 none, 1 full sums, 2 incremental (changed rows only)
    // adaptive passes: the kernel runs only if *mode == expect (mode NULL:
    // always); a full pass with changed != NULL counts the rows whose label
    // differs from the one labels held before the pass
    const int64_t *mode;
    int expect;
    // adaptive pass run by the rotated-copies kernel (auto_state NULL: not
    // adaptive): the kernel itself chooses the kind of pass (see RcParams)
    int64_t *auto_state = nullptr;
    int auto_first = 0;
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

// The rows of one pass set: warp w handles the RW-row groups starting at
// base0 (its first) and every step rows after, below r_end.  mus / sS, sC,
// snk / stage_all are the shared-memory centre table, update sums and row
// staging (each used only by the variants that have them).
template <int KPL, bool MU_SMEM, bool PRIV, bool STAGE, bool COPIES>
__device__ __forceinline__ void kmeans_rows(const KmParams &P, const float *mus, float *sS,
                                            int32_t *sC, int32_t *snk, int2 *stage_all,
                                            int64_t base0, int64_t step, int64_t r_end) {
    constexpr int NP = KPL / 2;  // packed pairs per lane
    const int tid = threadIdx.x;
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
    const int m = P.m;

    for (int64_t base = base0; base < r_end; base += step) {
        const int rows_here = (int)((r_end - base) < P.RW ? (r_end - base) : P.RW);
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
        if ((P.do_update == 2 || P.changed) && row_ok && kl == 0) old_pref = P.labels[i];
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
                        j = clamp_index(iv.x, P.pt);  // indices outside [0, pt) are clamped
                        v = __int_as_float(iv.y);
                    } else {
                        j = clamp_index(__ldg(ri + t), P.pt);
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
            if (P.do_update != 2 && P.changed) {
                const unsigned mv = __ballot_sync(kFull, row_ok && kl == 0 && old != label);
                if (lane == 0 && mv) atomicAdd(P.changed, (unsigned long long)__popc(mv));
            }
            if (P.do_update == 2) {
                // incremental sums: a row whose label moved from old to label
                // leaves cluster old and joins cluster label (exact in FP64 for
                // float inputs up to rounding of the running sums)
                old = __shfl_sync(kFull, old, (lead < 32) ? lead : lane);
                const bool moved = row_ok && kl == 0 && old != label &&
                                   (unsigned)label < (unsigned)P.K;
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
                            j = clamp_index(iv.x, P.pt);
                            v = __int_as_float(iv.y);
                        } else {
                            j = clamp_index(__ldg(P.idx + (base + rs) * m + t), P.pt);
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
                        j = clamp_index(iv.x, P.pt);
                        v = __int_as_float(iv.y);
                    } else {
                        j = clamp_index(__ldg(P.idx + ii * m + t), P.pt);
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
}

template <int KPL, bool MU_SMEM, bool PRIV, bool STAGE, bool COPIES>
__global__ void __launch_bounds__(kThreads) kmeans_kernel(KmParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (P.mode && *P.mode != P.expect) return;  // the other kind of pass runs
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

    {
        const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + tid) >> 5;
        const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
        kmeans_rows<KPL, MU_SMEM, PRIV, STAGE, COPIES>(P, mus, sS, sC, snk, stage_all,
                                                       gwarp * P.RW, nwarps * P.RW, P.n);
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

// Adaptive pass, first step (one CTA; used where the rotated-copies kernel,
// which makes this choice itself, does not apply): state[0] holds the
// number of rows whose label changed in the previous pass.  If that is more
// than thr (or this is the first pass), this pass rebuilds the sums from
// zero: the sums are zeroed here and state[1] = 1 selects the full pass;
// otherwise state[1] = 2 selects the incremental pass.  state[2] restarts at
// 0 and the pass that runs adds its own count of changed rows to it.
__global__ void kmeans_auto_decide_kernel(int64_t *state, int64_t thr, int first, int64_t KP,
                                          int K, double *S, int32_t *cnt, int64_t *nk) {
    __shared__ int full;
    if (threadIdx.x == 0) full = (first || state[0] > thr) ? 1 : 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        state[1] = full ? 1 : 2;
        state[2] = 0;
    }
    if (full) {
        for (int64_t e = threadIdx.x; e < KP; e += blockDim.x) {
            S[e] = 0.0;
            cnt[e] = 0;
        }
        for (int e = threadIdx.x; e < K; e += blockDim.x) nk[e] = 0;
    }
}

// Adaptive pass, last step where kmeans_auto_decide_kernel ran: this pass's
// count of changed rows becomes the next pass's state[0].
__global__ void kmeans_auto_carry_kernel(int64_t *state) {
    if (threadIdx.x == 0) {
        state[0] = state[2];
        state[2] = 0;
    }
}

// ---- many data sets in one persistent launch (K <= 64)
//
// Tasks (data set, row range) are taken in order from a ticket counter.  A
// data set's centres sit in shared memory when they fit the table region
// (reloaded only when the CTA moves to another data set), and its rows are
// staged when the per-warp staging fits; otherwise the variant reads them
// through L1/L2.  Sums go to the caller's float64 / int32 arrays with global
// atomics (no shared-memory privatisation across data sets).
struct KmTask {
    int32_t d;
    int32_t variant;  // bit 0: centre table in shared memory, bit 1: staged rows,
                      // bit 2: centre table = the transposed copy in global memory
    int64_t r_begin, r_end;
};

__global__ void __launch_bounds__(kThreads, 1) kmeans_batch_kernel(const KmParams *Ps,
                                                               const KmTask *tasks, int ntasks,
                                                               unsigned int *ticket,
                                                               int mu_cap_bytes, int do_update) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_task, s_last;
    float *mus = reinterpret_cast<float *>(smem_raw);
    int2 *stage_all = reinterpret_cast<int2 *>(smem_raw + mu_cap_bytes);
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) s_last = -1;
    for (;;) {
        if (tid == 0) s_task = (int)atomicAdd(ticket, 1u);
        __syncthreads();
        const int t = s_task;
        const int last = s_last;
        if (t >= ntasks) break;
        const KmTask T = tasks[t];
        KmParams P = Ps[T.d];
        P.do_assign = 1;
        P.do_update = do_update;
        if ((T.variant & 1) && T.d != last) {
            for (int e = tid; e < P.pt * P.Kpad; e += blockDim.x) {
                const int j = e / P.Kpad, k = e - j * P.Kpad;
                mus[e] = (k < P.K) ? P.mu[(int64_t)k * P.pt + j] : 0.f;
            }
        }
        __syncthreads();
        if (tid == 0) s_last = (T.variant & 1) ? T.d : -1;
        const int64_t base0 = T.r_begin + (int64_t)warp * P.RW;
        const int64_t step = (int64_t)kWarpsK * P.RW;
        switch (T.variant) {
            case 6:
                kmeans_rows<2, true, false, true, false>(P, P.mu_t, nullptr, nullptr, nullptr,
                                                         stage_all, base0, step, T.r_end);
                break;
            case 4:
                kmeans_rows<2, true, false, false, false>(P, P.mu_t, nullptr, nullptr, nullptr,
                                                          stage_all, base0, step, T.r_end);
                break;
            case 3:
                kmeans_rows<2, true, false, true, false>(P, mus, nullptr, nullptr, nullptr,
                                                         stage_all, base0, step, T.r_end);
                break;
            case 1:
                kmeans_rows<2, true, false, false, false>(P, mus, nullptr, nullptr, nullptr,
                                                          stage_all, base0, step, T.r_end);
                break;
            case 2:
                kmeans_rows<2, false, false, true, false>(P, mus, nullptr, nullptr, nullptr,
                                                          stage_all, base0, step, T.r_end);
                break;
            default:
                kmeans_rows<2, false, false, false, false>(P, mus, nullptr, nullptr, nullptr,
                                                           stage_all, base0, step, T.r_end);
                break;
        }
        // rows done before the centre table, the staging or the ticket is reused
        __syncthreads();
    }
}

// Zero (mode 0) or finalize (mode 1: mu = S / cnt where cnt > 0) the sums of
// every data set: element e of the concatenated K x pt arrays (start[] is the
// prefix), plus each data set's nk in mode 0.
__global__ void kmeans_sums_batch_kernel(const KmParams *Ps, const int64_t *start, int nd,
                                         int64_t total, int mode) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = nd - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (start[mid] <= e) lo = mid; else hi = mid - 1;
        }
        const KmParams &P = Ps[lo];
        const int64_t k = e - start[lo];
        float *mu = const_cast<float *>(P.mu);
        if (mode == 0) {
            P.S[k] = 0.0;
            P.cnt[k] = 0;
            if (k < P.K) P.nk[k] = 0;
        } else {
            const int32_t c = P.cnt[k];
            if (c > 0) mu[k] = (float)(P.S[k] / (double)c);
        }
        if (P.mu_t) {
            // the transposed copy follows mu (and zero in the padding centre)
            const int kk = (int)(k / P.pt), j = (int)(k - (int64_t)kk * P.pt);
            P.mu_t[(int64_t)j * P.Kpad + kk] = mu[k];
            if (mode == 0 && kk == P.K - 1)
                for (int q = P.K; q < P.Kpad; ++q) P.mu_t[(int64_t)j * P.Kpad + q] = 0.f;
        }
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

// ---- one lane per row part, all K centres per lane (K <= 32)
//
// A half-warp holds NP = ceil(K/2) rows and C = 16 / NP lanes per row (one
// per "copy").  Lane (c, ph) owns row ph of its half-warp and the entries
// t = c, c + C, ... of that row, and accumulates the restricted distances to
// all K centres (NP packed pairs) for them; the C partial sums of a row are
// added with shuffles at the end.  Coordinate j owns one 32-word line of
// shared memory with C copies of its Kpad = 2 NP centre values, copy c at
// pair positions c NP .. c NP + NP - 1.  At unrolled step q, lane (c, ph)
// reads pair (q + ph) mod NP of copy c: the 16 lanes of a half-warp then hit
// 16 distinct bank pairs whatever their rows' coordinates, so each centre
// load is one wavefront per half-warp and carries 8 bytes for every lane.
// The rotation makes accumulator slot q of lane (c, ph) hold centre pair
// (q + ph) mod NP; all lanes of a row share ph, so their slots line up.
// The rows are staged per warp as (idx, val) pairs at a row stride S >= m
// chosen so that a half-warp's stage read touches distinct bank pairs too
// ((ph S + c) mod 16 distinct over its lanes; S = C (mod 16) always works).
struct RcParams {
    const int32_t *idx;
    const float *val;
    int64_t n;
    int m, pt, K, S;
    uint32_t minv;  // floor(2^32 / m) + 1 (m >= 2): e / m = umulhi(e, minv) for e m < 2^32
    const float *mu;
    int32_t *labels;
    float *dist;
    double *Ssum;
    int32_t *cnt;
    int64_t *nk;
    unsigned long long *changed;  // rows whose label changed (may be NULL)
    int do_update;                // 0 none, 2 incremental (changed rows only)
    // Adaptive passes: the kernel runs only if *mode == expect.  The kernel
    // instance with AUTO = true instead chooses the kind of pass itself: mode
    // then points at the caller's int64[3] state and expect is kAutoFirst or
    // kAutoLater (the fields are reused: a larger parameter block made the
    // compiler spill in the assignment loop).  A full rebuild if this is the
    // first pass or state[0] (the previous pass's count of changed rows) >
    // n / 12; a full pass zeroes S, cnt and nk and assigns only
    // (kmeans_sums_kernel, launched next, adds the sums from the labels),
    // otherwise the pass is incremental.  Block 0 records the choice in
    // state[1] (1 full, 2 incremental); changed points at state[2], zero on
    // entry.
    const int64_t *mode;
    int expect;
};

constexpr int kAutoFirst = -2, kAutoLater = -1;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Asks L2 to fetch the 16-byte blocks that lie wholly inside [a0, a1) (a
// hint: no data comes back to the thread, and nothing outside the range is
// touched).
__device__ __forceinline__ void prefetch_l2_inside(const char *a0, const char *a1) {
    const uintptr_t lo = (reinterpret_cast<uintptr_t>(a0) + 15) & ~(uintptr_t)15;
    const uintptr_t hi = reinterpret_cast<uintptr_t>(a1) & ~(uintptr_t)15;
    if (hi > lo)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;"
                     :
                     : "l"(lo), "r"((uint32_t)(hi - lo))
                     : "memory");
}

// groups ahead whose rows the rotated-copies pass prefetches into L2
// (measured at n = 10^6, p = 1024, K = 10: one ahead 0.152 ms per pass, two
// 0.135, three 0.136, four 0.150, none 0.167)
constexpr int kL2Ahead = 2;

__device__ __forceinline__ uint64_t lds64(uint32_t addr) {
    uint64_t v;
    asm volatile("ld.shared.b64 %0, [%1];" : "=l"(v) : "r"(addr));
    return v;
}

// Threads per CTA of the rotated-copies pass: up to 32 warps while a lane's
// NP accumulator pairs and offsets fit 64 registers, then 24, 20 and 16 warps
// as NP grows (no register spills).
// (A row whose distances are all NaN keeps the label 0x7fffffff, which every
// update skips.)
template <int NP>
constexpr int rc_max_threads() { return NP <= 6 ? 1024 : NP <= 9 ? 768 : NP <= 12 ? 640 : 512; }

// The adaptive pass's choice (see RcParams), made by every CTA alike; a full
// pass's zeroing of the sums is spread over the grid.  (Measured at n = 10^6,
// p = 1024, K = 10: an incremental adaptive pass 0.140 ms against 0.147 for
// the earlier four launches, a one-CTA choice kernel and both kinds of
// assignment; the 20-pass loop 3.19 against 3.23 ms.)
__device__ __forceinline__ void rc_auto_choose(const RcParams &P, int *s_update) {
    int64_t *state = const_cast<int64_t *>(P.mode);
    const bool full = P.expect == kAutoFirst || state[0] > P.n / 12;
    if (threadIdx.x == 0) *s_update = full ? 0 : 2;
    if (full) {
        const int64_t KP = (int64_t)P.K * P.pt;
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < KP;
             e += (int64_t)gridDim.x * blockDim.x) {
            P.Ssum[e] = 0.0;
            P.cnt[e] = 0;
        }
        if (blockIdx.x == 0 && (int)threadIdx.x < P.K) P.nk[threadIdx.x] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) state[1] = full ? 1 : 2;
}

template <int NP, bool AUTO>
__global__ void __launch_bounds__(rc_max_threads<NP>()) kmeans_rc_kernel(RcParams P) {
    constexpr int C = 16 / NP;  // lanes per row
    constexpr int RW = 2 * NP;  // rows per warp
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // the kind of update an adaptive pass makes (kept in shared memory: read
    // once per row group, it holds no register through the loop)
    __shared__ int s_update;
    if constexpr (AUTO) {
        rc_auto_choose(P, &s_update);
    } else {
        if (P.mode && *P.mode != P.expect) return;  // the other kind of pass runs
    }
    float *tab = reinterpret_cast<float *>(smem_raw);
    int2 *stage_all = reinterpret_cast<int2 *>(smem_raw + (size_t)P.pt * 128);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    {
        // word w of line j: copy w / (2 NP), centre 2 ((w / 2) mod NP) + (w & 1);
        // eight loads in flight per thread before their stores
        constexpr int kU = 8;
        for (int e0 = tid; e0 < P.pt * 32; e0 += kU * blockDim.x) {
            float x[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int e = e0 + u * blockDim.x;
                const int j = e >> 5, w = e & 31, b = w >> 1;
                x[u] = 0.f;
                if (e < P.pt * 32 && b < C * NP) {
                    const int cc = b / NP;
                    const int k = 2 * (b - cc * NP) + (w & 1);
                    if (k < P.K) x[u] = __ldg(P.mu + (int64_t)k * P.pt + j);
                }
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int e = e0 + u * blockDim.x;
                if (e < P.pt * 32) tab[e] = x[u];
            }
        }
    }
    __syncthreads();

    const int h = lane >> 4, sl = lane & 15;
    const bool used = sl < C * NP;
    const int c = used ? sl / NP : 0;
    const int ph = used ? sl - c * NP : 0;
    const int rw = h * NP + ph;          // row of this lane within the warp's group
    const int lead = h * 16 + ph;        // lane c = 0 of this row
    uint32_t off[NP];                    // byte offsets of the lane's NP pairs in a line
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        int pi = q + ph;
        if (pi >= NP) pi -= NP;
        off[q] = smem_u32(tab) + 8u * (uint32_t)(c * NP + pi);
    }
    const int m = P.m, S = P.S;
    int2 *stage = stage_all + (size_t)warp * RW * S;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + tid) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const bool track_old = P.do_update == 2 || P.changed != nullptr;  // adaptive: changed is set

    // The group's rows are contiguous in the ELL arrays and are read with
    // coalesced loads, eight per lane in flight before their stores.  Two of
    // the warp's lanes ask L2 for the idx and val ranges of the group two
    // steps ahead (a bulk prefetch), so that the loads find their lines in L2
    // rather than in DRAM.
    const int64_t step = nwarps * RW;
    // stage position of entry e of the group: row r = e / m, column e - r m
    auto spos = [&](int e) {
        if (S == m) return e;
        const int r = m == 1 ? e : (int)__umulhi((uint32_t)e, P.minv);
        return r * S + (e - r * m);
    };

    for (int64_t base = gwarp * RW; base < P.n; base += step) {
        const int rows_here = (int)((P.n - base) < RW ? (P.n - base) : RW);
        {
            constexpr int kU = 8;
            const int total = rows_here * m;
            const int32_t *gi = P.idx + base * m;
            const float *gv = P.val + base * m;
            for (int e0 = lane; e0 < total; e0 += 32 * kU) {
                int2 x[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int e = e0 + 32 * u;
                    if (e < total) x[u] = make_int2(__ldg(gi + e), __float_as_int(__ldg(gv + e)));
                }
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int e = e0 + 32 * u;
                    if (e < total) stage[spos(e)] = x[u];
                }
            }
        }
        __syncwarp();
        // (issued after this group's loads: issued before them, the pass
        // measured 0.158 ms instead of 0.135)
        if (lane < 2) {
            const int64_t nb = base + kL2Ahead * step;
            if (nb < P.n) {
                const int rows_b = (int)((P.n - nb) < RW ? (P.n - nb) : RW);
                const char *a0 = lane == 0 ? reinterpret_cast<const char *>(P.idx + nb * m)
                                           : reinterpret_cast<const char *>(P.val + nb * m);
                prefetch_l2_inside(a0, a0 + (size_t)rows_b * m * 4);
            }
        }
        const int64_t i = base + rw;
        const bool row_ok = used && rw < rows_here;
        int old = -1;
        if (track_old && row_ok && c == 0) old = P.labels[i];
        uint64_t acc[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) acc[q] = 0ull;
        const int2 *rs = stage + rw * S;
        if (row_ok) {
#pragma unroll 2
            for (int t = c; t < m; t += C) {
                const int2 iv = rs[t];
                const uint32_t jb = (uint32_t)clamp_index(iv.x, P.pt) << 7;
                const float v = __int_as_float(iv.y);
                const uint64_t vv = pack2(v, v);
#pragma unroll
                for (int q = 0; q < NP; ++q) acc[q] = sqacc2(sub2(vv, lds64(off[q] + jb)), acc[q]);
            }
        }
        // the C partial sums of a row, into its lane c = 0 (the row's lanes
        // are NP apart inside the half-warp)
#pragma unroll
        for (int cc = 1; cc < C; ++cc) {
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const uint64_t o = __shfl_down_sync(kFull, acc[q], cc * NP);
                if (c == 0) {
                    uint64_t a;
                    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(a) : "l"(acc[q]), "l"(o));
                    acc[q] = a;
                }
            }
        }
        // argmin over the K centres (ties to the smaller k); slot q holds pair
        // (q + ph) mod NP
        float bd = INFINITY;
        int bk = 0x7fffffff;
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            int pi = q + ph;
            if (pi >= NP) pi -= NP;
            const int k0 = 2 * pi;
            const float d0 = __uint_as_float((uint32_t)acc[q]);
            const float d1 = __uint_as_float((uint32_t)(acc[q] >> 32));
            if (k0 < P.K && (d0 < bd || (d0 == bd && k0 < bk))) {
                bd = d0;
                bk = k0;
            }
            if (k0 + 1 < P.K && (d1 < bd || (d1 == bd && k0 + 1 < bk))) {
                bd = d1;
                bk = k0 + 1;
            }
        }
        const int label = __shfl_sync(kFull, bk, lead);
        old = __shfl_sync(kFull, old, lead);
        if (row_ok && c == 0) {
            P.labels[i] = label;
            if (P.dist) P.dist[i] = bd;
        }
        const bool moved = row_ok && old != label && (unsigned)label < (unsigned)P.K;
        if (P.changed) {
            const unsigned mv = __ballot_sync(kFull, moved && c == 0);
            if (lane == 0 && mv) atomicAdd(P.changed, (unsigned long long)__popc(mv));
        }
        if ((AUTO ? s_update == 2 : P.do_update == 2) && moved) {
            // incremental sums: the row leaves cluster old and joins label
            // (its C lanes move their own entries)
            for (int t = c; t < m; t += C) {
                const int2 iv = rs[t];
                const int j = clamp_index(iv.x, P.pt);
                const double v = (double)__int_as_float(iv.y);
                atomicAdd(P.Ssum + (int64_t)label * P.pt + j, v);
                atomicAdd(P.cnt + (int64_t)label * P.pt + j, 1);
                if ((unsigned)old < (unsigned)P.K) {
                    atomicAdd(P.Ssum + (int64_t)old * P.pt + j, -v);
                    atomicAdd(P.cnt + (int64_t)old * P.pt + j, -1);
                }
            }
            if (c == 0) {
                atomicAdd(reinterpret_cast<unsigned long long *>(P.nk + label), 1ull);
                if ((unsigned)old < (unsigned)P.K)
                    atomicAdd(reinterpret_cast<unsigned long long *>(P.nk + old),
                              (unsigned long long)(-1LL));
            }
        }
        __syncwarp();  // the stage is rewritten by the next group
    }
}

template <int NP>
cudaError_t launch_rc_np(const RcParams &P, int warps, size_t smem, cudaStream_t s) {
    auto kern = P.expect < 0 ? kmeans_rc_kernel<NP, true> : kmeans_rc_kernel<NP, false>;
    if (warps > rc_max_threads<NP>() / 32) {
        warps = rc_max_threads<NP>() / 32;
        smem = (size_t)P.pt * 128 + (size_t)warps * 2 * NP * P.S * 8;
    }
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t groups = (P.n + 2 * NP - 1) / (2 * NP);
    int64_t blocks = (groups + warps - 1) / warps;
    if (blocks > sms) blocks = sms;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, warps * 32, smem, s>>>(P);
    return cudaGetLastError();
}

// ---- the sums of a full rebuild from finished labels (Eq. (mu_update_one))
//
// After the rotated-copies assignment has written every row's label, this
// pass adds each entry to S[label][idx] and cnt[label][idx] and each row to
// nk[label], in CTA-private shared-memory sums (float S, int32 counts)
// flushed to the caller's float64 / int32 / int64 sums with one atomic per
// touched slot.  A warp takes 32 consecutive rows at a time: lane l holds the
// label of row l and the rows' m entries are read flat and coalesced, each
// entry's label passed by a shuffle.
struct SumParams {
    const int32_t *idx;
    const float *val;
    const int32_t *labels;
    int64_t n;
    int m, pt, K;
    uint32_t minv;  // floor(2^32 / m) + 1 (m >= 2)
    double *Ssum;
    int32_t *cnt;
    int64_t *nk;
    const int64_t *mode;  // adaptive passes: run only if *mode == expect
    int expect;
    // adaptive passes: block 0 moves this pass's count of changed rows
    // (carry[2]) to carry[0] for the next pass and zeroes carry[2] (NULL:
    // nothing); it runs whichever kind of pass ran
    int64_t *carry = nullptr;
};

__global__ void __launch_bounds__(kThreads) kmeans_sums_kernel(SumParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (P.carry && blockIdx.x == 0 && threadIdx.x == 0) {
        P.carry[0] = P.carry[2];
        P.carry[2] = 0;
    }
    if (P.mode && *P.mode != P.expect) return;
    const int KP = P.K * P.pt;
    float *sS = reinterpret_cast<float *>(smem_raw);
    int32_t *sC = reinterpret_cast<int32_t *>(smem_raw + (size_t)KP * 4);
    int32_t *snk = reinterpret_cast<int32_t *>(smem_raw + (size_t)KP * 8);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int e = tid; e < KP; e += blockDim.x) {
        sS[e] = 0.f;
        sC[e] = 0;
    }
    for (int e = tid; e < P.K; e += blockDim.x) snk[e] = 0;
    __syncthreads();
    const int m = P.m;
    const int wpb = blockDim.x >> 5;
    const int64_t nchunks = (P.n + 31) / 32;
    for (int64_t ch = (int64_t)blockIdx.x * wpb + warp; ch < nchunks;
         ch += (int64_t)gridDim.x * wpb) {
        const int64_t r0 = ch * 32;
        const int rows = (int)((P.n - r0) < 32 ? (P.n - r0) : 32);
        const int lab = lane < rows ? __ldg(P.labels + r0 + lane) : -1;
        const bool lab_ok = (unsigned)lab < (unsigned)P.K;
        {
            // rows of one cluster within the 32: one atomic per cluster
            const unsigned grp = __match_any_sync(kFull, lab);
            if (lab_ok && (grp & lanemask_lt()) == 0) atomicAdd(snk + lab, __popc(grp));
        }
        const int total = rows * m;
        const int32_t *gi = P.idx + r0 * m;
        const float *gv = P.val + r0 * m;
        constexpr int kU = 4;
        for (int e0 = lane; e0 - lane < total; e0 += 32 * kU) {
            int jx[kU];
            float vx[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int e = e0 + 32 * u;
                jx[u] = 0;
                vx[u] = 0.f;
                if (e < total) {
                    jx[u] = __ldg(gi + e);
                    vx[u] = __ldg(gv + e);
                }
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int e = e0 + 32 * u;
                const int r = e < total ? (m == 1 ? e : (int)__umulhi((uint32_t)e, P.minv)) : 0;
                const int le = __shfl_sync(kFull, lab, r);
                if (e < total && (unsigned)le < (unsigned)P.K) {
                    const int slot = le * P.pt + clamp_index(jx[u], P.pt);
                    atomicAdd(sS + slot, vx[u]);
                    atomicAdd(sC + slot, 1);
                }
            }
        }
    }
    __syncthreads();
    for (int e = tid; e < KP; e += blockDim.x) {
        const int c = sC[e];
        const float x = sS[e];
        if (x != 0.f) atomicAdd(P.Ssum + e, (double)x);
        if (c) atomicAdd(P.cnt + e, c);
    }
    for (int e = tid; e < P.K; e += blockDim.x)
        if (snk[e]) atomicAdd(reinterpret_cast<unsigned long long *>(P.nk + e),
                              (unsigned long long)(long long)snk[e]);
}

// Launches kmeans_sums_kernel if its shared-memory sums fit; *used tells
// whether it did.
cudaError_t launch_sums(const KmParams &Q, cudaStream_t s, bool *used) {
    *used = false;
    int dev = 0, smem_max = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = (size_t)Q.K * Q.pt * 8 + (((size_t)Q.K * 4 + 15) & ~(size_t)15);
    if (smem > (size_t)smem_max) return cudaSuccess;
    SumParams P;
    P.idx = Q.idx;
    P.val = Q.val;
    P.labels = Q.labels;
    P.n = Q.n;
    P.m = Q.m;
    P.pt = Q.pt;
    P.K = Q.K;
    P.minv = Q.m >= 2 ? (uint32_t)(0x100000000ull / (uint64_t)Q.m + 1) : 0u;
    P.Ssum = Q.S;
    P.cnt = Q.cnt;
    P.nk = Q.nk;
    P.mode = Q.mode;
    P.expect = Q.expect;
    P.carry = Q.auto_state;
    cudaError_t e = cudaFuncSetAttribute(kmeans_sums_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kmeans_sums_kernel, kThreads, smem);
    if (per_sm < 1) per_sm = 1;
    const int64_t chunks = (Q.n + 31) / 32;
    int64_t blocks = (chunks + kWarpsK - 1) / kWarpsK;
    if (blocks > (int64_t)sms * per_sm) blocks = (int64_t)sms * per_sm;
    if (blocks < 1) blocks = 1;
    *used = true;
    kmeans_sums_kernel<<<(unsigned)blocks, kThreads, smem, s>>>(P);
    return cudaGetLastError();
}

// Launches the rotated-copies pass if it applies (K <= 32, no full-rebuild
// sums, the table and at least eight warps' staging fit shared memory);
// *used tells whether it did.
cudaError_t launch_rc(const KmParams &Q, cudaStream_t s, bool *used) {
    *used = false;
    if (!Q.do_assign || Q.K > 32) return cudaSuccess;
    const int NP = (Q.K + 1) / 2;
    const int C = 16 / NP;
    int dev = 0, smem_max = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // stage row stride: the smallest S >= m for which the bank pairs
    // (ph S + c) mod 16 of a half-warp's lanes (ph < NP, c < C) are distinct
    int S = Q.m;
    for (;; ++S) {
        unsigned seen = 0;
        bool ok = true;
        for (int ph = 0; ph < NP && ok; ++ph)
            for (int c = 0; c < C && ok; ++c) {
                const unsigned bit = 1u << ((ph * S + c) & 15);
                ok = !(seen & bit);
                seen |= bit;
            }
        if (ok) break;
    }
    const size_t table = (size_t)Q.pt * 128;
    const size_t per_warp = (size_t)2 * NP * S * 8;
    if (table + 8 * per_warp > (size_t)smem_max) return cudaSuccess;
    int warps = (int)(((size_t)smem_max - table) / per_warp);
    if (warps > kWarpsK) warps = kWarpsK;
    RcParams P;
    P.idx = Q.idx;
    P.val = Q.val;
    P.n = Q.n;
    P.m = Q.m;
    P.pt = Q.pt;
    P.K = Q.K;
    P.S = S;
    P.minv = Q.m >= 2 ? (uint32_t)(0x100000000ull / (uint64_t)Q.m + 1) : 0u;
    P.mu = Q.mu;
    P.labels = Q.labels;
    P.dist = Q.dist;
    P.Ssum = Q.S;
    P.cnt = Q.cnt;
    P.nk = Q.nk;
    P.changed = Q.changed;
    P.do_update = Q.do_update == 2 ? 2 : 0;
    P.mode = Q.auto_state ? Q.auto_state : Q.mode;
    P.expect = Q.auto_state ? (Q.auto_first ? kAutoFirst : kAutoLater) : Q.expect;
    const size_t smem = table + (size_t)warps * per_warp;
    if (Q.do_update == 1) {
        // a full rebuild: this assignment, then the sums from its labels
        const size_t sums_b = (size_t)Q.K * Q.pt * 8 + (((size_t)Q.K * 4 + 15) & ~(size_t)15);
        if (sums_b > (size_t)smem_max) return cudaSuccess;
    }
    *used = true;
    cudaError_t e = cudaSuccess;
    switch (NP) {
        case 1: e = launch_rc_np<1>(P, warps, smem, s); break;
        case 2: e = launch_rc_np<2>(P, warps, smem, s); break;
        case 3: e = launch_rc_np<3>(P, warps, smem, s); break;
        case 4: e = launch_rc_np<4>(P, warps, smem, s); break;
        case 5: e = launch_rc_np<5>(P, warps, smem, s); break;
        case 6: e = launch_rc_np<6>(P, warps, smem, s); break;
        case 7: e = launch_rc_np<7>(P, warps, smem, s); break;
        case 8: e = launch_rc_np<8>(P, warps, smem, s); break;
        case 9: e = launch_rc_np<9>(P, warps, smem, s); break;
        case 10: e = launch_rc_np<10>(P, warps, smem, s); break;
        case 11: e = launch_rc_np<11>(P, warps, smem, s); break;
        case 12: e = launch_rc_np<12>(P, warps, smem, s); break;
        case 13: e = launch_rc_np<13>(P, warps, smem, s); break;
        case 14: e = launch_rc_np<14>(P, warps, smem, s); break;
        case 15: e = launch_rc_np<15>(P, warps, smem, s); break;
        default: e = launch_rc_np<16>(P, warps, smem, s); break;
    }
    if (e != cudaSuccess || Q.do_update != 1) return e;
    bool sums_used = false;
    return launch_sums(Q, s, &sums_used);
}

}  // namespace

static cudaError_t launch_kmeans_mode(const sk_ctx &c, const int32_t *idx, const float *val,
                                      int64_t n, const float *mu, int K, int32_t *labels,
                                      float *dist, double *S, int32_t *cnt, int64_t *nk,
                                      bool do_assign, int do_update, int64_t *changed,
                                      const int64_t *mode, int expect, cudaStream_t s);

cudaError_t launch_kmeans(const sk_ctx &c, const int32_t *idx, const float *val,
                          int64_t n, const float *mu, int K, int32_t *labels, float *dist,
                          double *S, int32_t *cnt, int64_t *nk, bool do_assign,
                          int do_update, int64_t *changed, cudaStream_t s) {
    return launch_kmeans_mode(c, idx, val, n, mu, K, labels, dist, S, cnt, nk, do_assign,
                              do_update, changed, nullptr, 0, s);
}

cudaError_t launch_kmeans_auto(const sk_ctx &c, const int32_t *idx, const float *val,
                               int64_t n, const float *mu, int K, int32_t *labels, float *dist,
                               double *S, int32_t *cnt, int64_t *nk, int64_t *state, int first,
                               cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int64_t thr = n / 12;
    // state[2] counts this pass's changed rows; every pass leaves it at zero
    if (first) {
        const cudaError_t e = cudaMemsetAsync(state + 2, 0, sizeof(int64_t), s);
        if (e != cudaSuccess) return e;
    }
    {
        // two launches: the rotated-copies assignment chooses the kind of
        // pass itself (and zeroes the sums for a full one), then the sums
        // pass (which returns at once after an incremental pass) carries the
        // count of changed rows to state[0]
        KmParams Q;
        Q.idx = idx;
        Q.val = val;
        Q.n = n;
        Q.m = (int)c.m;
        Q.pt = (int)c.pt;
        Q.K = K;
        Q.mu = mu;
        Q.labels = labels;
        Q.dist = dist;
        Q.S = S;
        Q.cnt = cnt;
        Q.nk = nk;
        Q.changed = reinterpret_cast<unsigned long long *>(state + 2);
        Q.do_assign = 1;
        Q.do_update = 1;
        Q.mode = state + 1;
        Q.expect = 1;
        Q.auto_state = state;
        Q.auto_first = first;  // the kernel's threshold is n / 12 too
        bool used = false;
        const cudaError_t e = launch_rc(Q, s, &used);
        if (used || e != cudaSuccess) return e;
    }
    // other K, pt: a one-CTA choice, both kinds of pass (the one not chosen
    // returns at once), then the carry
    kmeans_auto_decide_kernel<<<1, 1024, 0, s>>>(state, thr, first, (int64_t)K * c.pt, K, S,
                                                 cnt, nk);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_kmeans_mode(c, idx, val, n, mu, K, labels, dist, S, cnt, nk, true, 1, state + 2,
                           state + 1, 1, s);
    if (e != cudaSuccess) return e;
    e = launch_kmeans_mode(c, idx, val, n, mu, K, labels, dist, S, cnt, nk, true, 2, state + 2,
                           state + 1, 2, s);
    if (e != cudaSuccess) return e;
    kmeans_auto_carry_kernel<<<1, 32, 0, s>>>(state);
    return cudaGetLastError();
}

static cudaError_t launch_kmeans_mode(const sk_ctx &c, const int32_t *idx, const float *val,
                                      int64_t n, const float *mu, int K, int32_t *labels,
                                      float *dist, double *S, int32_t *cnt, int64_t *nk,
                                      bool do_assign, int do_update, int64_t *changed,
                                      const int64_t *mode, int expect, cudaStream_t s) {
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
    P.mode = mode;
    P.expect = expect;
    bool used = false;
    const cudaError_t e = launch_rc(P, s, &used);
    if (used || e != cudaSuccess) return e;
    if (K <= 64) return launch_kpl<2>(P, s);
    if (K <= 128) return launch_kpl<4>(P, s);
    return launch_kpl<8>(P, s);
}

static size_t km_al256(size_t x) { return (x + 255) & ~(size_t)255; }

cudaError_t kmeans_batch_build(const sk_ctx *ctxs, const BatchKmeans *it, int nd,
                               std::vector<unsigned char> &table, KmeansBatchInfo &info) {
    int dev = 0, smem_max = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    std::vector<KmParams> Ps((size_t)nd);
    std::vector<int64_t> start((size_t)nd + 1);
    // centre-table region: the largest table that fits 70% of shared memory
    size_t mu_cap = 0;
    for (int d = 0; d < nd; ++d) {
        const int LPR = (it[d].K + 1) / 2;
        const size_t mu_b = (size_t)ctxs[d].pt * (2 * LPR) * 4;
        if (mu_b <= (size_t)smem_max * 7 / 10 && mu_b > mu_cap) mu_cap = mu_b;
    }
    mu_cap = (mu_cap + 15) & ~(size_t)15;
    const size_t stage_region = (size_t)smem_max - mu_cap;
    std::vector<KmTask> tasks;
    int64_t total = 0;
    size_t stage_used = 0, stage_used_g = 0;  // all data sets / global-table ones
    for (int d = 0; d < nd; ++d) {
        const sk_ctx &c = ctxs[d];
        KmParams &P = Ps[d];
        std::memset(&P, 0, sizeof(P));
        if (it[d].K < 1 || it[d].K > 64) return cudaErrorInvalidValue;
        P.idx = it[d].idx;
        P.val = it[d].val;
        P.n = it[d].n;
        P.m = (int)c.m;
        P.pt = (int)c.pt;
        P.K = it[d].K;
        P.LPR = (P.K + 1) / 2;
        P.Kpad = 2 * P.LPR;
        P.G = P.LPR <= 16 ? 16 / P.LPR : 0;
        P.RW = P.G ? 2 * P.G : 32 / P.LPR;
        P.mu = it[d].mu;
        P.mu_t = it[d].mu_t;
        P.labels = it[d].labels;
        P.dist = nullptr;
        P.S = it[d].S;
        P.cnt = it[d].cnt;
        P.nk = it[d].nk;
        P.changed = reinterpret_cast<unsigned long long *>(it[d].changed);
        start[d] = total;
        total += (int64_t)P.K * P.pt;
        const bool mu_smem = (size_t)P.pt * P.Kpad * 4 <= mu_cap;
        const size_t st_b = (size_t)kWarpsK * P.RW * P.m * 8;
        const bool staged = st_b <= stage_region;
        P.stage_cap = staged ? P.RW * P.m : 0;
        if (staged && st_b > stage_used) stage_used = st_b;
        if (staged && !mu_smem && P.mu_t && st_b > stage_used_g) stage_used_g = st_b;
        const int variant = (mu_smem ? 1 : (P.mu_t ? 4 : 0)) | (staged ? 2 : 0);
        const int64_t per = (int64_t)kWarpsK * P.RW * 16;  // 16 passes per warp
        for (int64_t r = 0; r < P.n; r += per) {
            KmTask T;
            T.d = d;
            T.variant = variant;
            T.r_begin = r;
            T.r_end = (r + per < P.n) ? r + per : P.n;
            tasks.push_back(T);
        }
    }
    start[nd] = total;
    // tasks whose centre table stays in shared memory (or is not needed)
    // first, then those reading it from global memory; within each group
    // the costliest rows (m K) first
    std::stable_sort(tasks.begin(), tasks.end(), [&](const KmTask &a, const KmTask &b) {
        const int ga = (a.variant & 4) ? 1 : 0, gb = (b.variant & 4) ? 1 : 0;
        if (ga != gb) return ga < gb;
        return (int64_t)Ps[a.d].m * Ps[a.d].K > (int64_t)Ps[b.d].m * Ps[b.d].K;
    });
    info.nd = nd;
    info.ntasks = (int)tasks.size();
    info.ntasks_smem = 0;
    while (info.ntasks_smem < info.ntasks && !(tasks[info.ntasks_smem].variant & 4))
        ++info.ntasks_smem;
    info.total = total;
    info.mu_cap = (int)mu_cap;
    info.smem = mu_cap + stage_used;
    info.params_off = km_al256(table.size());
    info.tasks_off = km_al256(info.params_off + Ps.size() * sizeof(KmParams));
    info.start_off = km_al256(info.tasks_off + tasks.size() * sizeof(KmTask));
    info.ticket_off = km_al256(info.start_off + start.size() * sizeof(int64_t));
    table.resize(info.ticket_off + 256, 0);  // two tickets: one per launch
    std::memcpy(table.data() + info.params_off, Ps.data(), Ps.size() * sizeof(KmParams));
    if (!tasks.empty())
        std::memcpy(table.data() + info.tasks_off, tasks.data(), tasks.size() * sizeof(KmTask));
    std::memcpy(table.data() + info.start_off, start.data(), start.size() * sizeof(int64_t));
    cudaError_t e = cudaFuncSetAttribute(kmeans_batch_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)info.smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kmeans_batch_kernel, kThreads,
                                                  info.smem);
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)sms * per_sm;
    const int na = info.ntasks_smem, ng = info.ntasks - info.ntasks_smem;
    if (grid > na) grid = na > 0 ? na : 1;
    info.grid = (int)grid;
    // the global-table launch: its data sets' staging only (the rest of the
    // SM's memory goes to L1, which holds the tables' hot lines)
    info.smem_g = stage_used_g;
    per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kmeans_batch_kernel, kThreads,
                                                  info.smem_g);
    if (per_sm < 1) per_sm = 1;
    int64_t grid_g = (int64_t)sms * per_sm;
    if (grid_g > ng) grid_g = ng > 0 ? ng : 1;
    info.grid_g = (int)grid_g;
    return cudaSuccess;
}

cudaError_t kmeans_batch_launch(const KmeansBatchInfo &info, unsigned char *dev_table, int op,
                                cudaStream_t s) {
    const KmParams *Ps = reinterpret_cast<const KmParams *>(dev_table + info.params_off);
    const int64_t *start = reinterpret_cast<const int64_t *>(dev_table + info.start_off);
    if (op == 0 || op == 3) {  // reset / finalize
        if (info.total == 0) return cudaSuccess;
        int64_t blocks = (info.total + 255) / 256;
        if (blocks > 8192) blocks = 8192;
        kmeans_sums_batch_kernel<<<(unsigned)blocks, 256, 0, s>>>(Ps, start, info.nd, info.total,
                                                                 op == 0 ? 0 : 1);
        return cudaGetLastError();
    }
    if (info.ntasks == 0) return cudaSuccess;
    unsigned int *ticket = reinterpret_cast<unsigned int *>(dev_table + info.ticket_off);
    cudaError_t e = cudaMemsetAsync(ticket, 0, 2 * sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    const KmTask *tasks = reinterpret_cast<const KmTask *>(dev_table + info.tasks_off);
    // op 1: full sums (after a reset), op 2: incremental
    if (info.ntasks_smem > 0) {
        kmeans_batch_kernel<<<(unsigned)info.grid, kThreads, info.smem, s>>>(
            Ps, tasks, info.ntasks_smem, ticket, info.mu_cap, op == 1 ? 1 : 2);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (info.ntasks > info.ntasks_smem) {
        kmeans_batch_kernel<<<(unsigned)info.grid_g, kThreads, info.smem_g, s>>>(
            Ps, tasks + info.ntasks_smem, info.ntasks - info.ntasks_smem, ticket + 1, 0,
            op == 1 ? 1 : 2);
        e = cudaGetLastError();
    }
    return e;
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
