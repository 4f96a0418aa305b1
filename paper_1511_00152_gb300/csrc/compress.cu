// compress.cu -- fused one-pass compression (Sec. III Eq. (ROS); Algorithm 1,
// lines "Y <- HDX" and "w_i = R_i R_i^T y_i").
//
// One pass over X: each sample is read once from HBM (coalesced 16-byte
// loads), signed by D, transformed by the orthonormal Sylvester
// Walsh-Hadamard matrix, and the m entries of its mask are gathered into the
// ELL output.  The transform runs on a 1024-element "unit" per warp: phase A
// does the butterflies on element bits {0,1,7,8,9} in registers (the layout a
// float4 load gives), a swizzled shared-memory transpose brings bits {2..6}
// into registers for phase B, and for pt > 1024 a phase C across the warps of
// a row group handles bits 10.. .  Units with pt < 1024 hold 1024/pt rows.
//
// The mask (Sec. I-A, Thm. B1) is the partial Fisher-Yates of the written
// spec.  Its m draws are computed 32 at a time, one per lane: Lemire draws in
// parallel (a rejection, probability < pt/2^32 per draw, shifts the word
// index of the later lanes), then the swaps are resolved in parallel: the
// value a step emits is the value of its target position just before the
// step, which is either an earlier step's displaced value (found with
// __match_any_sync) or the position's state after the earlier chunks (a
// tagged shared-memory array).
#include "sk_internal.cuh"

namespace sk {
namespace {

constexpr int kWarps = 8;
constexpr unsigned kFull = 0xffffffffu;

struct CompressParams {
    const float *X;
    int64_t n, p, ldx, row0;
    int m;
    uint32_t k0, k1;
    int32_t *idx;
    float *val;
    float *Y;
    float scale;
    int vec;
};

// Swizzled shared-memory slot of unit element e: XOR of bits 2..4 with bits
// 7..9 makes both the float4 (phase A) and the stride-4 (phase B) access
// patterns bank-conflict free.
__device__ __forceinline__ int phys(int e) { return e ^ (((e >> 7) & 7) << 2); }

template <int G>
__device__ __forceinline__ void group_sync(int grp) {
    if constexpr (G == 1) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(grp + 1), "r"(G * 32) : "memory");
    }
}

template <int L>
__device__ __forceinline__ int yaddr(int ebase, int c) {
    if constexpr (L <= 10) {
        return phys(ebase + c);
    } else {
        return ((c >> 10) << 10) + phys(c & 1023);
    }
}

__device__ __forceinline__ int readA(const uint32_t *A, uint32_t tag, int j) {
    const uint32_t a = A[j];
    return (a >> 16) == tag ? (int)(a & 0xFFFFu) : j;
}

// Mask of one row and its ELL gather, by one warp.
template <int L>
__device__ __forceinline__ void sample_row(const CompressParams &P, int64_t i,
                                           const float *ybuf, int ebase, uint32_t *A,
                                           uint32_t *hit, uint32_t tag, int lane) {
    constexpr int PT = 1 << L;
    const uint64_t g = (uint64_t)(P.row0 + i);
    const int m = P.m;
    int32_t *oidx = P.idx + i * (int64_t)m;
    float *oval = P.val + i * (int64_t)m;
    const unsigned lt = lanemask_lt();
    const unsigned gt = lanemask_gt();
    uint32_t woff = 0;
    for (int c0 = 0; c0 < m; c0 += 32) {
        const int t = c0 + lane;
        const bool act = t < m;
        const uint32_t s = (uint32_t)(PT - t);
        uint32_t w = (uint32_t)t + woff;
        uint64_t prod = 0;
        for (;;) {
            const uint32_t word = act ? mask_word(P.k0, P.k1, g, w) : 0u;
            prod = (uint64_t)word * (uint64_t)s;
            bool rej = false;
            if (act && (uint32_t)prod < s) rej = (uint32_t)prod < ((0u - s) % s);
            const unsigned bal = __ballot_sync(kFull, rej);
            if (bal == 0u) break;
            const int first = __ffs(bal) - 1;
            if (lane >= first) ++w;
            ++woff;
        }
        const int k = act ? t + (int)(prod >> 32) : -1 - lane;
        const unsigned grpm = __match_any_sync(kFull, k);

        // src: latest earlier lane of this chunk whose target is position t.
        hit[lane] = 0u;
        __syncwarp();
        if (act && k < c0 + 32) atomicOr(&hit[k - c0], 1u << lane);
        __syncwarp();
        const unsigned srcm = act ? (hit[lane] & lt) : 0u;
        const int src = srcm ? 31 - __clz(srcm) : lane;
        const int vbase = act ? readA(A, tag, t) : 0;
        int V = vbase;  // value at position t just before step t
        for (;;) {
            const int from = __shfl_sync(kFull, V, src);
            const int nv = srcm ? from : vbase;
            const bool changed = nv != V;
            V = nv;
            if (!__ballot_sync(kFull, changed)) break;
        }
        const unsigned prevm = grpm & lt;
        const int prev = prevm ? 31 - __clz(prevm) : lane;
        const int vprev = __shfl_sync(kFull, V, prev);
        int omega = 0;
        if (act) omega = prevm ? vprev : readA(A, tag, k);
        __syncwarp();
        if (act && c0 + 32 < m && (grpm & gt) == 0u && k >= c0 + 32)
            A[k] = (tag << 16) | (uint32_t)V;
        if (act) {
            oidx[t] = omega;
            oval[t] = ybuf[yaddr<L>(ebase, omega)] * P.scale;
        }
        __syncwarp();
    }
}

template <int L, bool DENSE>
__global__ void __launch_bounds__(kWarps * 32, 2) compress_kernel(CompressParams P) {
    constexpr int PT = 1 << L;
    constexpr int G = (L > 10) ? (PT >> 10) : 1;  // warps per row group
    constexpr int NG = kWarps / G;                // row groups per CTA
    constexpr int RPU = (L <= 10) ? (1024 >> L) : 1;
    constexpr int BUF = (L <= 10) ? 1024 : PT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = warp / G, wg = warp % G;
    float *ybuf = reinterpret_cast<float *>(smem_raw) + grp * BUF;
    uint32_t *A = reinterpret_cast<uint32_t *>(smem_raw + NG * BUF * 4) + grp * PT;
    uint32_t *hit = reinterpret_cast<uint32_t *>(smem_raw + NG * BUF * 4 + NG * PT * 4) + grp * 32;

    if constexpr (!DENSE) {
        if (wg == 0)
            for (int j = lane; j < PT; j += 32) A[j] = 0u;
    }
    uint32_t tag = 1;

    // Sign bits of the 32 coordinates this thread holds in phase A.
    uint32_t smask = 0;
#pragma unroll 1
    for (int r = 0; r < 32; ++r) {
        const int e = 128 * (r >> 2) + 4 * lane + (r & 3);
        const int c = (L <= 10) ? (e & (PT - 1)) : (1024 * wg + e);
        smask |= sign_bit(P.k0, P.k1, (uint32_t)c) << r;
    }

    const int64_t nunits = (L <= 10) ? (P.n + RPU - 1) / RPU : P.n;
    const int64_t stride = (int64_t)gridDim.x * NG;
    for (int64_t u = (int64_t)blockIdx.x * NG + grp; u < nunits; u += stride) {
        const int64_t r0 = u * RPU;
        float v[32];
        // ---- load (phase A layout): element e = 128*ip + 4*lane + q
#pragma unroll
        for (int ip = 0; ip < 8; ++ip) {
            const int e = 128 * ip + 4 * lane;
            if constexpr (L >= 2) {
                const int b = (L <= 10) ? (e >> L) : 0;
                const int c = (L <= 10) ? (e & (PT - 1)) : (1024 * wg + e);
                const int64_t i = r0 + b;
                float4 x4 = make_float4(0.f, 0.f, 0.f, 0.f);
                if (i < P.n) {
                    const float *src = P.X + i * P.ldx + c;
                    if (P.vec) {
                        if (c < P.p) x4 = __ldcs(reinterpret_cast<const float4 *>(src));
                    } else {
                        if (c + 0 < P.p) x4.x = __ldcs(src + 0);
                        if (c + 1 < P.p) x4.y = __ldcs(src + 1);
                        if (c + 2 < P.p) x4.z = __ldcs(src + 2);
                        if (c + 3 < P.p) x4.w = __ldcs(src + 3);
                    }
                }
                v[4 * ip + 0] = x4.x;
                v[4 * ip + 1] = x4.y;
                v[4 * ip + 2] = x4.z;
                v[4 * ip + 3] = x4.w;
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int eq = e + q;
                    const int64_t i = r0 + (eq >> L);
                    const int c = eq & (PT - 1);
                    v[4 * ip + q] = (i < P.n && c < P.p) ? __ldcs(P.X + i * P.ldx + c) : 0.f;
                }
            }
        }
        // ---- D: flip the sign bit where D_j = -1
#pragma unroll
        for (int r = 0; r < 32; ++r)
            v[r] = __uint_as_float(__float_as_uint(v[r]) ^ (((smask >> r) & 1u) << 31));
        // ---- phase A: register bit rb <-> element bit {0,1,7,8,9}[rb]
#pragma unroll
        for (int rb = 0; rb < 5; ++rb) {
            const int eb = rb < 2 ? rb : rb + 5;
            if (eb < L) {
#pragma unroll
                for (int r = 0; r < 32; ++r) {
                    if (!(r & (1 << rb))) {
                        const float a = v[r], b = v[r | (1 << rb)];
                        v[r] = a + b;
                        v[r | (1 << rb)] = a - b;
                    }
                }
            }
        }
        group_sync<G>(grp);  // previous unit's gathers are done with ybuf
        float *wbuf = ybuf + ((L > 10) ? 1024 * wg : 0);
#pragma unroll
        for (int ip = 0; ip < 8; ++ip) {
            const int e = 128 * ip + 4 * lane;
            *reinterpret_cast<float4 *>(wbuf + phys(e)) =
                make_float4(v[4 * ip], v[4 * ip + 1], v[4 * ip + 2], v[4 * ip + 3]);
        }
        __syncwarp();
        // ---- phase B: lane = (q, i''), register j <-> element bits 2..6
        {
            const int q = lane & 3, ib = lane >> 2;
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = wbuf[phys(128 * ib + 4 * j + q)];
#pragma unroll
            for (int rb = 0; rb < 5; ++rb) {
                if (rb + 2 < L) {
#pragma unroll
                    for (int r = 0; r < 32; ++r) {
                        if (!(r & (1 << rb))) {
                            const float a = v[r], b = v[r | (1 << rb)];
                            v[r] = a + b;
                            v[r | (1 << rb)] = a - b;
                        }
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < 32; ++j) wbuf[phys(128 * ib + 4 * j + q)] = v[j];
        }
        // ---- phase C (pt > 1024): element bits 10.. across the group's warps
        if constexpr (L > 10) {
            constexpr int S = 32 / G;
            group_sync<G>(grp);
            const int tau = wg * 32 + lane;
#pragma unroll
            for (int s = 0; s < S; ++s)
#pragma unroll
                for (int w2 = 0; w2 < G; ++w2)
                    v[s * G + w2] = ybuf[1024 * w2 + phys(tau + 32 * G * s)];
#pragma unroll
            for (int rb = 0; (1 << rb) < G; ++rb) {
#pragma unroll
                for (int r = 0; r < 32; ++r) {
                    if (!(r & (1 << rb))) {
                        const float a = v[r], b = v[r | (1 << rb)];
                        v[r] = a + b;
                        v[r | (1 << rb)] = a - b;
                    }
                }
            }
#pragma unroll
            for (int s = 0; s < S; ++s)
#pragma unroll
                for (int w2 = 0; w2 < G; ++w2)
                    ybuf[1024 * w2 + phys(tau + 32 * G * s)] = v[s * G + w2];
        }
        group_sync<G>(grp);

        if constexpr (DENSE) {
            // y rows out, scaled, coalesced 16-byte stores
#pragma unroll
            for (int ip = 0; ip < 8; ++ip) {
                const int e = 128 * ip + 4 * lane;
                const float4 y4 = *reinterpret_cast<const float4 *>(wbuf + phys(e));
                const float ys[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int eq = e + q;
                    const int64_t i = (L <= 10) ? r0 + (eq >> L) : r0;
                    const int c = (L <= 10) ? (eq & (PT - 1)) : (1024 * wg + eq);
                    if (i < P.n) P.Y[i * PT + c] = ys[q] * P.scale;
                }
            }
        } else {
            if (L <= 10 || wg == 0) {
#pragma unroll 1
                for (int b = 0; b < RPU; ++b) {
                    const int64_t i = r0 + b;
                    if (i >= P.n) break;
                    sample_row<L>(P, i, ybuf, b * PT, A, hit, tag, lane);
                    if (++tag == 0x10000u) {
                        for (int j = lane; j < PT; j += 32) A[j] = 0u;
                        __syncwarp();
                        tag = 1;
                    }
                }
            }
        }
    }
}

template <int L, bool DENSE>
cudaError_t launch_L(const CompressParams &P, cudaStream_t s) {
    constexpr int PT = 1 << L;
    constexpr int G = (L > 10) ? (PT >> 10) : 1;
    constexpr int NG = kWarps / G;
    constexpr int RPU = (L <= 10) ? (1024 >> L) : 1;
    constexpr int BUF = (L <= 10) ? 1024 : PT;
    const size_t smem = (size_t)NG * BUF * 4 + (DENSE ? 0 : (size_t)NG * PT * 4 + NG * 32 * 4);
    auto kern = compress_kernel<L, DENSE>;
    static bool configured = false;  // per instantiation; attribute is per device context
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWarps * 32, smem);
    if (per_sm < 1) per_sm = 1;
    const int64_t nunits = (L <= 10) ? (P.n + RPU - 1) / RPU : P.n;
    int64_t blocks = (nunits + NG - 1) / NG;
    const int64_t cap = (int64_t)sms * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, kWarps * 32, smem, s>>>(P);
    return cudaGetLastError();
}

template <bool DENSE>
cudaError_t dispatch(int L, const CompressParams &P, cudaStream_t s) {
    switch (L) {
        case 0: return launch_L<0, DENSE>(P, s);
        case 1: return launch_L<1, DENSE>(P, s);
        case 2: return launch_L<2, DENSE>(P, s);
        case 3: return launch_L<3, DENSE>(P, s);
        case 4: return launch_L<4, DENSE>(P, s);
        case 5: return launch_L<5, DENSE>(P, s);
        case 6: return launch_L<6, DENSE>(P, s);
        case 7: return launch_L<7, DENSE>(P, s);
        case 8: return launch_L<8, DENSE>(P, s);
        case 9: return launch_L<9, DENSE>(P, s);
        case 10: return launch_L<10, DENSE>(P, s);
        case 11: return launch_L<11, DENSE>(P, s);
        case 12: return launch_L<12, DENSE>(P, s);
        case 13: return launch_L<13, DENSE>(P, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_compress(const sk_ctx &c, const float *X, int64_t n, int64_t ldx,
                            int64_t row0, int32_t *idx, float *val, float *Y,
                            cudaStream_t s) {
    CompressParams P;
    P.X = X;
    P.n = n;
    P.p = c.p;
    P.ldx = ldx;
    P.row0 = row0;
    P.m = (int)c.m;
    P.k0 = (uint32_t)c.seed;
    P.k1 = (uint32_t)(c.seed >> 32);
    P.idx = idx;
    P.val = val;
    P.Y = Y;
    P.scale = (float)(1.0 / sqrt((double)c.pt));
    P.vec = ((reinterpret_cast<uintptr_t>(X) & 15) == 0) && (c.p % 4 == 0) && (ldx % 4 == 0);
    if (n == 0) return cudaSuccess;
    return Y ? dispatch<true>(c.log2pt, P, s) : dispatch<false>(c.log2pt, P, s);
}

}  // namespace sk
