// gram_tc.cu -- covariance Gram on the 5th-generation tensor cores (tcgen05 +
// TMEM), the one dense contraction of the path (Sec. V: G = sum_i w_i w_i^T).
//
// Work unit = (output tile, row segment).  A tile is 128 x N of the pt x pt
// Gram (N = 256, or pt when pt = 128), upper tiles only.  The contraction
// runs over the segment's rows in K-slabs of 64 rows:
//   * 8 producer warps scatter the slab's ELL entries that fall in the
//     tile's row block (operand A, 128 x 64) and column block (operand B,
//     N x 64) into zeroed shared-memory tiles, BF16, K-major with the
//     128-byte swizzle; for the split mode also the low parts
//     lo = bf16(v - hi) into a second pair of tiles;
//   * one thread issues tcgen05.mma kind::f16 (M = 128, N, K = 16) four times
//     per slab (twelve for the split mode: hi*hi + hi*lo + lo*hi) into an
//     FP32 accumulator in TMEM, and tcgen05.commit frees the stage;
//   * after the segment, the 8 warps read the accumulator with tcgen05.ld
//     and add it into the caller's FP64 Gram with double atomics (the FP64
//     cross-segment reduction).
// A segment is at most 65536 rows, which bounds the length of each FP32
// accumulation chain.  Every mbarrier wait is bounded: on expiry the kernel
// sets the device error word, stops issuing, drains its MMAs (bounded),
// frees TMEM and returns.
#include <cuda_bf16.h>

#include "sk_internal.cuh"

namespace sk {

__device__ unsigned int g_device_error = 0u;

unsigned int *device_error_word() {
    // device address of g_device_error for kernels in other translation units
    // (looked up on every call: cheap, and correct for whichever device is current)
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_device_error) != cudaSuccess) return nullptr;
    return static_cast<unsigned int *>(ptr);
}

cudaError_t take_device_error(unsigned int *flag) {
    unsigned int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(flag, g_device_error, sizeof(*flag));
    if (e != cudaSuccess) return e;
    if (*flag) e = cudaMemcpyToSymbol(g_device_error, &zero, sizeof(zero));
    return e;
}

namespace {

constexpr int kProducerWarps = 8;
constexpr int kProducers = kProducerWarps * 32;
constexpr int kThreads = kProducers + 32;  // + the MMA warp
constexpr int kSlab = 64;                  // rows per K-slab (128 bytes of BF16)
constexpr int kTileM = 128;
constexpr int kSegmentRows = 1 << 18;     // rows per FP32 accumulation chain (then FP64)
constexpr int kChunk = 8;                  // bucketed entries per producer thread per pass
constexpr int kBlk = 128;                  // column block of the bucketing
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

struct TcParams {
    const int32_t *idx;
    const float *val;
    int64_t n;
    int m;
    int pt;
    int N;        // tile width (columns of the Gram)
    int nbi, nbj;  // row / column block counts
    int ntiles;
    int64_t rows_per_split;  // multiple of kSlab, <= kSegmentRows
    int nsplits;
    int hilo;      // 1: split-BF16 (three products)
    int nstages;
    int stage_bytes;
    int nblk;             // pt / 128 column blocks
    const int2 *bkt;      // bucketed entries: (block << 14 | tile byte offset, value bits)
    const int *boff;      // per slab: nblk + 1 bucket starts (relative to the slab)
    double *G;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar)
                 : "memory");
}

// Bounded wait for the phase of the given parity; false on expiry or abort.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long deadline,
                                          volatile int *abort_flag) {
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (*abort_flag) return false;
        if (clock64() > deadline) return false;
    }
}

__device__ __forceinline__ void named_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Shared-memory matrix descriptor: K-major operand with the 128-byte swizzle
// (rows of 128 bytes, 8-row groups 1024 bytes apart).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
    d |= (uint64_t)1 << 16;                    // leading byte offset (unused here)
    d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset: 8 rows
    d |= (uint64_t)1 << 46;                    // descriptor version
    d |= (uint64_t)2 << 61;                    // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

// Byte offset of element (r, k) in a K-major, 128B-swizzled tile of 64-wide rows.
__device__ __forceinline__ uint32_t sw_off(int r, int k) {
    return (uint32_t)(r * 128 + ((((k >> 3) ^ (r & 7))) << 4) + ((k & 7) << 1));
}

// Bucketing pass: the entries of each 64-row slab (a contiguous ELL range) are
// grouped by 128-column block; each entry carries the byte offset of its
// (column-in-block, row-in-slab) element in a K-major, 128B-swizzled operand
// tile, so the Gram producers only copy.  One CTA per slab; the per-block
// counters take warp-aggregated shared-memory atomics.
__global__ void __launch_bounds__(256) bucket_kernel(const int32_t *idx, const float *val,
                                                     int64_t n, int m, int pt, int nblk,
                                                     int2 *bkt, int *boff) {
    __shared__ int hist[64];
    __shared__ int cursor[64];
    const int64_t s = blockIdx.x;
    const int64_t r0 = s * kSlab;
    const int rows = (int)((n - r0) < kSlab ? (n - r0) : kSlab);
    const int total = rows * m;
    const int32_t *gi = idx + r0 * m;
    const float *gv = val + r0 * m;
    int2 *out = bkt + s * (int64_t)kSlab * m;
    const int tid = threadIdx.x, lane = tid & 31;
    const unsigned lt = lanemask_lt();
    for (int c = tid; c < nblk; c += blockDim.x) hist[c] = 0;
    __syncthreads();
    for (int e0 = 0; e0 < total; e0 += blockDim.x) {
        const int e = e0 + tid;
        const int c = e < total ? ((__ldg(gi + e) & (pt - 1)) >> 7) : -1 - lane;
        const unsigned grp = __match_any_sync(0xffffffffu, c);
        if (e < total && (grp & lt) == 0u) atomicAdd(&hist[c], __popc(grp));
    }
    __syncthreads();
    if (tid == 0) {
        int acc = 0;
        for (int c = 0; c < nblk; ++c) {
            boff[s * (nblk + 1) + c] = acc;
            cursor[c] = acc;
            acc += hist[c];
        }
        boff[s * (nblk + 1) + nblk] = acc;
    }
    __syncthreads();
    const float inv_m = 1.0f / (float)m;
    for (int e0 = 0; e0 < total; e0 += blockDim.x) {
        const int e = e0 + tid;
        int j = 0, c = -1 - lane;
        float v = 0.f;
        if (e < total) {
            j = __ldg(gi + e) & (pt - 1);
            v = __ldg(gv + e);
            c = j >> 7;
        }
        const unsigned grp = __match_any_sync(0xffffffffu, c);
        const int leader = __ffs(grp) - 1;
        int base = 0;
        if (e < total && lane == leader) base = atomicAdd(&cursor[c], __popc(grp));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (e < total) {
            // row within the slab: exact (e + 0.5 is >= 0.5 from every multiple of m)
            const int k = (int)(((float)e + 0.5f) * inv_m);
            const int pos = base + __popc(grp & lt);
            out[pos] = make_int2((c << 14) | (int)sw_off(j & (kBlk - 1), k), __float_as_int(v));
        }
    }
}

__device__ __forceinline__ void decode_tile(const TcParams &P, int t, int &bi, int &bj) {
    const int ratio = P.N / kTileM;  // column blocks are ratio row blocks wide
    bi = 0;
    for (;;) {
        const int first = bi / ratio;
        const int cnt = P.nbj - first;
        if (t < cnt) {
            bj = first + t;
            return;
        }
        t -= cnt;
        ++bi;
    }
}

__global__ void __launch_bounds__(kThreads, 1) gram_tc_kernel(TcParams P) {
    extern __shared__ __align__(1024) unsigned char smem_dyn[];
    // 1024-byte alignment of the operand tiles (the swizzle pattern repeats per 1 KB)
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
    unsigned char *tiles = smem;
    uint64_t *bars = reinterpret_cast<uint64_t *>(tiles + (size_t)P.nstages * P.stage_bytes);
    // bars[0..S) full, bars[S..2S) empty, bars[2S] done
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * P.nstages + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int tile = blockIdx.x % P.ntiles;
    const int split = blockIdx.x / P.ntiles;
    int bi, bj;
    decode_tile(P, tile, bi, bj);
    const int I0 = bi * kTileM, J0 = bj * P.N;
    const int64_t r_begin = (int64_t)split * P.rows_per_split;
    int64_t r_end = r_begin + P.rows_per_split;
    if (r_end > P.n) r_end = P.n;
    const int64_t nslabs = r_end > r_begin ? (r_end - r_begin + kSlab - 1) / kSlab : 0;
    const int N = P.N;
    const int S = P.nstages;
    const uint32_t a_bytes = kTileM * 128, b_bytes = (uint32_t)N * 128;

    if (tid == 0) {
        for (int s = 0; s < 2 * S + 1; ++s) mbar_init(smem_u32(bars + s), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kProducerWarps) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(256));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const long long deadline = clock64() + kWaitCycles;
    const uint32_t done_bar = smem_u32(bars + 2 * S);

    if (warp == kProducerWarps) {
        // ---------------- MMA issuer (one thread)
        if (lane == 0) {
            const uint32_t idesc = instr_desc(kTileM, N);
            int64_t issued = 0;
            for (int64_t i = 0; i < nslabs; ++i) {
                const int s = (int)(i % S);
                const uint32_t u = (uint32_t)(i / S);
                if (!mbar_wait(smem_u32(bars + s), u & 1u, deadline, abort_flag)) {
                    *abort_flag = 1;
                    atomicOr(&g_device_error, 1u);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t base = smem_u32(tiles + (size_t)s * P.stage_bytes);
                const uint32_t a_hi = base, b_hi = base + a_bytes;
                const uint32_t a_lo = base + a_bytes + b_bytes, b_lo = a_lo + a_bytes;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint32_t acc = (i > 0 || kk > 0) ? 1u : 0u;
                    mma_bf16(tmem, smem_desc(a_hi + kk * 32), smem_desc(b_hi + kk * 32), idesc, acc);
                    if (P.hilo) {
                        mma_bf16(tmem, smem_desc(a_hi + kk * 32), smem_desc(b_lo + kk * 32), idesc, 1u);
                        mma_bf16(tmem, smem_desc(a_lo + kk * 32), smem_desc(b_hi + kk * 32), idesc, 1u);
                    }
                }
                mma_commit(smem_u32(bars + S + s));
                ++issued;
            }
            // done barrier: completes when every MMA issued above has finished
            mma_commit(done_bar);
            (void)issued;
        }
        __syncwarp();
    } else {
        // ---------------- producers (then epilogue)
        // Slab i of the segment needs bucket bi (operand A) and buckets
        // [bj*R, bj*R + R) (operand B, R = N / 128) of the bucketed slab; both
        // ranges are contiguous.  The ranges of slab i + 1 are known one slab
        // ahead and its entries are loaded into registers while slab i is
        // scattered, so the load latency overlaps the scatter and the waits.
        const int ptid = tid;  // 0 .. kProducers-1
        const int m = P.m;
        const int R = N / kBlk;
        const int nb1 = P.nblk + 1;
        const int64_t slab0 = r_begin / kSlab;  // global slab index of this segment's first slab
        struct Ranges {
            int a0, na, b0, nb;
        };
        auto ranges = [&](int64_t i) -> Ranges {
            const int *o = P.boff + (slab0 + i) * nb1;
            Ranges r;
            r.a0 = __ldg(o + bi);
            r.na = __ldg(o + bi + 1) - r.a0;
            r.b0 = __ldg(o + bj * R);
            r.nb = __ldg(o + bj * R + R) - r.b0;
            return r;
        };
        int ck[kChunk], cv[kChunk], nk[kChunk], nv[kChunk];
        auto load_pass = [&](int64_t i, const Ranges &r, int ps, int *kk, int *vv) {
            const int2 *base = P.bkt + (slab0 + i) * (int64_t)kSlab * m;
#pragma unroll
            for (int q = 0; q < kChunk; ++q) {
                const int e = ps * (kProducers * kChunk) + q * kProducers + ptid;
                int2 x = make_int2(-1, 0);
                if (e < r.na) {
                    x = __ldg(base + r.a0 + e);
                    x.x |= 1 << 30;  // operand A
                } else if (e < r.na + r.nb) {
                    x = __ldg(base + r.b0 + (e - r.na));
                }
                kk[q] = x.x;
                vv[q] = x.y;
            }
        };
        Ranges cur{0, 0, 0, 0}, nxt{0, 0, 0, 0};
        if (nslabs > 0) {
            cur = ranges(0);
            load_pass(0, cur, 0, ck, cv);
        }
        if (nslabs > 1) nxt = ranges(1);
        int64_t slab = 0;
        int pass = 0;
        bool ok = true;
        const int per_pass = kProducers * kChunk;
        while (slab < nslabs && ok) {
            const int s = (int)(slab % S);
            const uint32_t u = (uint32_t)(slab / S);
            const int npass = (cur.na + cur.nb + per_pass - 1) / per_pass;
            unsigned char *st = tiles + (size_t)s * P.stage_bytes;
            if (pass == 0) {
                if (u > 0) {
                    if (!mbar_wait(smem_u32(bars + S + s), (u - 1) & 1u, deadline, abort_flag)) {
                        *abort_flag = 1;
                        atomicOr(&g_device_error, 1u);
                    }
                }
                named_sync(1, kProducers);  // every producer sees the same abort state
                if (*abort_flag) {
                    ok = false;
                    break;
                }
                for (int off = ptid * 16; off < P.stage_bytes; off += kProducers * 16)
                    *reinterpret_cast<uint4 *>(st + off) = make_uint4(0u, 0u, 0u, 0u);
                named_sync(1, kProducers);
            }
            const bool last_pass = pass + 1 >= npass;
            // prefetch: the next pass of this slab, or the first pass of the next slab
            Ranges nr = cur;
            int64_t ns = slab;
            int np = pass + 1;
            if (last_pass) {
                nr = nxt;
                ns = slab + 1;
                np = 0;
            }
            if (ns < nslabs) load_pass(ns, nr, np, nk, nv);
            if (last_pass && slab + 2 < nslabs) nxt = ranges(slab + 2);
            unsigned char *A_hi = st, *B_hi = st + a_bytes;
            unsigned char *A_lo = st + a_bytes + b_bytes, *B_lo = A_lo + a_bytes;
#pragma unroll
            for (int q = 0; q < kChunk; ++q) {
                const int key = ck[q];
                if (key >= 0) {
                    const bool isA = (key >> 30) & 1;
                    const int c = (key >> 14) & 0xFFFF;
                    const uint32_t off = (uint32_t)(key & 16383);
                    const float v = __int_as_float(cv[q]);
                    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
                    const uint32_t boffb = (uint32_t)(c - bj * R) * (kBlk * 128);
                    unsigned char *dh = isA ? A_hi + off : B_hi + boffb + off;
                    *reinterpret_cast<__nv_bfloat16 *>(dh) = hi;
                    if (P.hilo) {
                        const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
                        unsigned char *dl = isA ? A_lo + off : B_lo + boffb + off;
                        *reinterpret_cast<__nv_bfloat16 *>(dl) = lo;
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < kChunk; ++q) {
                ck[q] = nk[q];
                cv[q] = nv[q];
            }
            if (last_pass) {
                // generic-proxy writes -> visible to the tensor core (async proxy)
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                named_sync(1, kProducers);
                if (ptid == 0) mbar_arrive(smem_u32(bars + s));
                ++slab;
                pass = 0;
                cur = nr;
            } else {
                ++pass;
            }
        }
        // ---------------- epilogue: TMEM -> FP64 Gram
        const bool have = nslabs > 0;
        bool drained = false;
        if (have) drained = mbar_wait(done_bar, 0u, deadline + kWaitCycles, abort_flag) || false;
        if (have && !drained) {
            // a stalled pipeline: give the issued MMAs one more bounded wait
            // (without the abort short-cut) so TMEM is idle before it is freed
            const long long d2 = clock64() + kWaitCycles;
            volatile int never = 0;
            drained = mbar_wait(done_bar, 0u, d2, &never);
            if (!*abort_flag) {
                *abort_flag = 1;
                atomicOr(&g_device_error, 1u);
            }
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (have && drained && !*abort_flag) {
            const int q = warp & 3, h = warp >> 2;
            const int row = I0 + q * 32 + lane;
            for (int c0 = h * 128; c0 < N && c0 < h * 128 + 128; c0 += 32) {
                uint32_t r[32];
                const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                    "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                      "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                      "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
                      "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                      "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]),
                      "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                double *g = P.G + (int64_t)row * P.pt + (J0 + c0);
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    const float x = __uint_as_float(r[c]);
                    if (x != 0.f) atomicAdd(g + c, (double)x);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == kProducerWarps) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
    }
}

}  // namespace

int64_t gram_tc_workspace(const sk_ctx &c, int64_t n) {
    if (n <= 0) return 0;
    const int64_t nslab = (n + kSlab - 1) / kSlab;
    const int64_t nblk = c.pt / kBlk;
    const int64_t ent = nslab * kSlab * c.m * (int64_t)sizeof(int2);
    const int64_t offs = nslab * (nblk + 1) * (int64_t)sizeof(int);
    return ((ent + 255) & ~int64_t(255)) + offs + 256;
}

cudaError_t launch_gram_tc(const sk_ctx &c, int mode, const int32_t *idx, const float *val,
                           int64_t n, double *G, void *work, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if (c.pt < kTileM) return cudaErrorInvalidValue;
    TcParams P;
    P.idx = idx;
    P.val = val;
    P.n = n;
    P.m = (int)c.m;
    P.pt = (int)c.pt;
    P.N = c.pt >= 256 ? 256 : (int)c.pt;
    P.nbi = P.pt / kTileM;
    P.nbj = P.pt / P.N;
    const int ratio = P.N / kTileM;
    P.ntiles = 0;
    for (int bi = 0; bi < P.nbi; ++bi) P.ntiles += P.nbj - bi / ratio;
    P.hilo = (mode == SK_GRAM_BF16X3) ? 1 : 0;
    P.stage_bytes = (kTileM + P.N) * 128 * (P.hilo ? 2 : 1);
    P.nstages = P.hilo ? 2 : 4;
    if (P.N == 128 && !P.hilo) P.nstages = 6;
    if (P.N == 128 && P.hilo) P.nstages = 3;
    P.G = G;
    P.nblk = P.pt / kBlk;
    // workspace: bucketed entries (8 bytes each, 64 m per slab), then offsets
    const int64_t nslab = (n + kSlab - 1) / kSlab;
    const int64_t ent = nslab * kSlab * c.m * (int64_t)sizeof(int2);
    unsigned char *w = static_cast<unsigned char *>(work);
    P.bkt = reinterpret_cast<const int2 *>(w);
    P.boff = reinterpret_cast<const int *>(w + ((ent + 255) & ~int64_t(255)));
    bucket_kernel<<<(unsigned)nslab, 256, 0, s>>>(idx, val, n, P.m, P.pt, P.nblk,
                                                  reinterpret_cast<int2 *>(w),
                                                  const_cast<int *>(P.boff));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;

    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // row splits: no segment longer than kSegmentRows; among the counts that
    // allow, take the one whose units fill whole waves of the SMs best
    const int64_t min_splits = (n + kSegmentRows - 1) / kSegmentRows;
    int64_t best = min_splits;
    double best_eff = 0.0;
    for (int64_t sp = min_splits; sp <= min_splits + 64; ++sp) {
        if ((n + sp - 1) / sp < kSlab) break;
        const int64_t units = sp * P.ntiles;
        const int64_t waves = (units + sms - 1) / sms;
        const double eff = (double)units / (double)(waves * sms);
        if (eff > best_eff + 0.02) {
            best_eff = eff;
            best = sp;
        }
        if (eff > 0.95) break;
    }
    int64_t rps = (n + best - 1) / best;
    rps = (rps + kSlab - 1) / kSlab * kSlab;
    P.rows_per_split = rps;
    P.nsplits = (int)((n + rps - 1) / rps);
    const size_t smem = (size_t)P.nstages * P.stage_bytes + 1024 + 256;
    e = cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = (int64_t)P.ntiles * P.nsplits;
    gram_tc_kernel<<<(unsigned)grid, kThreads, smem, s>>>(P);
    return cudaGetLastError();
}

}  // namespace sk
