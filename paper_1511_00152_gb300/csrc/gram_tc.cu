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
//   * every kChunkSlabs slabs the MMAs switch to the other of two TMEM
//     accumulators (512 columns), and the 8 producer warps read the finished
//     one with tcgen05.ld and add it into FP32 registers with round-to-nearest
//     adds: the tensor core's own accumulation is biased toward zero over long
//     chains, so its chains are kept short (as in error-corrected tensor-core
//     GEMM, Ootomo & Yokota 2022);
//   * after the segment the registers are added into the caller's FP64 Gram
//     with double atomics (the FP64 cross-segment reduction).  Every mbarrier wait is bounded: on expiry the kernel
// sets the device error word, stops issuing, drains its MMAs (bounded),
// frees TMEM and returns.
#include <cuda_bf16.h>

#include <cstring>
#include <vector>

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
constexpr int kThreads = kProducers + 64;  // + the MMA warp + the loader warp
constexpr int kMmaWarp = kProducerWarps;
constexpr int kLoaderWarp = kProducerWarps + 1;
constexpr int kRing = 3;                   // bucket ranges staged ahead (slabs)
constexpr int kSlab = 64;                  // rows per K-slab (128 bytes of BF16)
constexpr int kTileM = 128;
constexpr int kSegmentRows = 1 << 18;     // rows per work unit (FP32 registers, then FP64)
constexpr int kChunkSlabs = 8;            // slabs per tensor-core accumulation chain
constexpr int kBlk = 128;                  // column block of the bucketing
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz: default limit, and drains

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
    int slot_bytes;       // ring slot size (entries of one slab's A and B ranges)
    const int2 *bkt;      // bucketed entries: (block << 14 | tile byte offset, value bits)
    const int *boff;      // per slab: nblk + 1 bucket starts (relative to the slab)
    double *G;
    long long wait_cycles;  // limit of the CTA's pipeline waits (SM clock cycles)
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
// The first test does not block, so a phase still pending once the deadline
// has passed counts as a wait that ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long deadline,
                                          volatile int *abort_flag) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    for (;;) {
        if (*abort_flag) return false;
        if (clock64() > deadline) return false;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
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
struct BucketParams {
    const int32_t *idx;
    const float *val;
    int64_t n;
    int m, pt, nblk;
    int2 *bkt;
    int *boff;
};

__device__ __forceinline__ void bucket_body(const int32_t *idx, const float *val, int64_t n, int m,
                                            int pt, int nblk, int2 *bkt, int *boff, int64_t s) {
    __shared__ int hist[64];
    __shared__ int cursor[64];
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
        const int c = e < total ? (clamp_index(__ldg(gi + e), pt) >> 7) : -1 - lane;
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
            j = clamp_index(__ldg(gi + e), pt);
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

__global__ void __launch_bounds__(256) bucket_kernel(const int32_t *idx, const float *val,
                                                     int64_t n, int m, int pt, int nblk,
                                                     int2 *bkt, int *boff) {
    bucket_body(idx, val, n, m, pt, nblk, bkt, boff, blockIdx.x);
}

// Many data sets: CTA b works on slab b - start[d] of the data set d with
// start[d] <= b < start[d + 1].
__global__ void __launch_bounds__(256) bucket_batch_kernel(const BucketParams *Bs, const int *start,
                                                           int nd) {
    int lo = 0, hi = nd - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    const BucketParams B = Bs[lo];
    bucket_body(B.idx, B.val, B.n, B.m, B.pt, B.nblk, B.bkt, B.boff, (int64_t)blockIdx.x - start[lo]);
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

__device__ __forceinline__ void gram_tc_body(const TcParams &P, int bid) {
    extern __shared__ __align__(1024) unsigned char smem_dyn[];
    // 1024-byte alignment of the operand tiles (the swizzle pattern repeats per 1 KB)
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
    unsigned char *tiles = smem;
    unsigned char *ring = tiles + (size_t)P.nstages * P.stage_bytes;
    int *hdr = reinterpret_cast<int *>(ring + (size_t)kRing * P.slot_bytes);  // 8 ints per slot
    uint64_t *bars = reinterpret_cast<uint64_t *>(hdr + 8 * kRing);
    // bars[0..S) full, [S..2S) empty, [2S] done, [2S+1..+kRing) ring full,
    // [2S+1+kRing..+kRing) ring empty
    uint64_t *acc_full = bars + 2 * P.nstages + 1 + 2 * kRing;  // [2]
    uint64_t *acc_empty = acc_full + 2;                          // [2]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_empty + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int tile = bid % P.ntiles;
    const int split = bid / P.ntiles;
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

    uint64_t *ring_full = bars + 2 * S + 1;
    uint64_t *ring_empty = ring_full + kRing;
    if (tid == 0) {
        for (int s = 0; s < 2 * S + 1 + 2 * kRing + 4; ++s) mbar_init(smem_u32(bars + s), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const long long deadline = clock64() + P.wait_cycles;
    const uint32_t done_bar = smem_u32(bars + 2 * S);

    if (warp == kLoaderWarp) {
        // ---------------- loader (one thread): bucket ranges -> shared ring
        if (lane == 0) {
            const int R = N / kBlk;
            const int nb1 = P.nblk + 1;
            const int64_t slab0 = r_begin / kSlab;
            int64_t issued = 0;
            for (int64_t i = 0; i < nslabs; ++i) {
                const int slot = (int)(i % kRing);
                const uint32_t ur = (uint32_t)(i / kRing);
                if (ur > 0 &&
                    !mbar_wait(smem_u32(ring_empty + slot), (ur - 1) & 1u, deadline, abort_flag)) {
                    *abort_flag = 1;
                    atomicOr(&g_device_error, 1u);
                    break;
                }
                const int *o = P.boff + (slab0 + i) * nb1;
                const int a0 = __ldg(o + bi), a1 = __ldg(o + bi + 1);
                const int bhi = bj * R + R < P.nblk ? bj * R + R : P.nblk;  // ragged last tile
                const int b0 = __ldg(o + bj * R), b1 = __ldg(o + bhi);
                const int64_t E0 = (slab0 + i) * (int64_t)kSlab * P.m;  // slab's first entry
                // 16-byte aligned covers of the two ranges (entries are 8 bytes)
                const int64_t sa = (E0 + a0) & ~int64_t(1), ea = (E0 + a1 + 1) & ~int64_t(1);
                const int64_t sb = (E0 + b0) & ~int64_t(1), eb = (E0 + b1 + 1) & ~int64_t(1);
                const uint32_t bytesA = (uint32_t)((a1 > a0 ? ea - sa : 0) * 8);
                const uint32_t bytesB = (uint32_t)((b1 > b0 ? eb - sb : 0) * 8);
                int *h = hdr + 8 * slot;
                unsigned char *dst = ring + (size_t)slot * P.slot_bytes;
                if (bytesA + bytesB > (uint32_t)P.slot_bytes) {
                    // does not fit: producers read this slab from global memory
                    h[0] = a0; h[1] = a1 - a0; h[2] = b0; h[3] = b1 - b0; h[4] = 1;
                    mbar_arrive(smem_u32(ring_full + slot));
                } else {
                    h[0] = (int)(E0 + a0 - sa);
                    h[1] = a1 - a0;
                    h[2] = (int)(bytesA / 8 + (E0 + b0 - sb));
                    h[3] = b1 - b0;
                    h[4] = 0;
                    const uint32_t bar = smem_u32(ring_full + slot);
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                                 "r"(bytesA + bytesB)
                                 : "memory");
                    if (bytesA)
                        asm volatile(
                            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
                            "[%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
                            "l"(P.bkt + sa), "r"(bytesA), "r"(bar)
                            : "memory");
                    if (bytesB)
                        asm volatile(
                            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
                            "[%0], [%1], %2, [%3];" ::"r"(smem_u32(dst + bytesA)),
                            "l"(P.bkt + sb), "r"(bytesB), "r"(bar)
                            : "memory");
                }
                ++issued;
            }
            // Before the CTA may exit, the last copy into each slot must have
            // landed (they all have, unless the producers stopped early).
            volatile int never = 0;
            for (int64_t i = issued - kRing > 0 ? issued - kRing : 0; i < issued; ++i)
                mbar_wait(smem_u32(ring_full + (i % kRing)), (uint32_t)((i / kRing) & 1),
                          clock64() + kWaitCycles, &never);
        }
        __syncwarp();
    } else if (warp == kMmaWarp) {
        // ---------------- MMA issuer (one thread)
        if (lane == 0) {
            const uint32_t idesc = instr_desc(kTileM, N);
            for (int64_t i = 0; i < nslabs; ++i) {
                const int s = (int)(i % S);
                const uint32_t u = (uint32_t)(i / S);
                const int64_t c = i / kChunkSlabs;  // accumulation chunk
                const int b = (int)(c & 1);
                const bool chunk_first = (i % kChunkSlabs) == 0;
                const bool chunk_last = (i % kChunkSlabs) == kChunkSlabs - 1 || i == nslabs - 1;
                if (chunk_first && c >= 2 &&
                    !mbar_wait(smem_u32(acc_empty + b), (uint32_t)(((c >> 1) - 1) & 1), deadline,
                               abort_flag)) {
                    *abort_flag = 1;
                    atomicOr(&g_device_error, 1u);
                    break;
                }
                if (!mbar_wait(smem_u32(bars + s), u & 1u, deadline, abort_flag)) {
                    *abort_flag = 1;
                    atomicOr(&g_device_error, 1u);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t base = smem_u32(tiles + (size_t)s * P.stage_bytes);
                const uint32_t a_hi = base, b_hi = base + a_bytes;
                const uint32_t a_lo = base + a_bytes + b_bytes, b_lo = a_lo + a_bytes;
                const uint32_t dacc = tmem + (uint32_t)(b * 256);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint32_t acc = (!chunk_first || kk > 0) ? 1u : 0u;
                    mma_bf16(dacc, smem_desc(a_hi + kk * 32), smem_desc(b_hi + kk * 32), idesc, acc);
                    if (P.hilo) {
                        mma_bf16(dacc, smem_desc(a_hi + kk * 32), smem_desc(b_lo + kk * 32), idesc, 1u);
                        mma_bf16(dacc, smem_desc(a_lo + kk * 32), smem_desc(b_hi + kk * 32), idesc, 1u);
                    }
                }
                mma_commit(smem_u32(bars + S + s));
                if (chunk_last) mma_commit(smem_u32(acc_full + b));
            }
            // done barrier: completes when every MMA issued above has finished
            mma_commit(done_bar);
        }
        __syncwarp();
    } else {
        // ---------------- producers (then epilogue)
        // Slab i needs bucket bi (operand A) and buckets [bj*R, bj*R + R)
        // (operand B, R = N / 128); the loader has staged both ranges in ring
        // slot i % kRing (or flagged the slab to be read from global memory).
        const int ptid = tid;  // 0 .. kProducers-1
        const int R = N / kBlk;
        const int64_t slab0 = r_begin / kSlab;
        // FP32 round-to-nearest accumulators: warp w holds TMEM lanes
        // 32*(w%4).. (rows of the tile) and columns 128*(w/4) .. +128
        const int q = warp & 3, hcol = warp >> 2;
        const bool has_cols = hcol * 128 < N;
        float acc[128];
#pragma unroll
        for (int j = 0; j < 128; ++j) acc[j] = 0.f;
        const int64_t nchunks = (nslabs + kChunkSlabs - 1) / kChunkSlabs;
        int64_t consumed = 0;  // chunks already added into acc
        auto consume = [&](int64_t c) -> bool {
            const int b = (int)(c & 1);
            if (!mbar_wait(smem_u32(acc_full + b), (uint32_t)((c >> 1) & 1), deadline, abort_flag)) {
                *abort_flag = 1;
                atomicOr(&g_device_error, 1u);
            }
            // every producer passes the barrier, then all take the same decision
            named_sync(1, kProducers);
            if (*abort_flag) return false;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (has_cols) {
#pragma unroll
                for (int part = 0; part < 4; ++part) {
                    uint32_t r[32];
                    const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) +
                                           (uint32_t)(b * 256 + hcol * 128 + part * 32);
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
#pragma unroll
                    for (int j = 0; j < 32; ++j) acc[part * 32 + j] += __uint_as_float(r[j]);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            named_sync(1, kProducers);
            if (ptid == 0) mbar_arrive(smem_u32(acc_empty + b));
            return true;
        };
        bool ok = true;
        for (int64_t i = 0; i < nslabs && ok; ++i) {
            const int s = (int)(i % S);
            const uint32_t u = (uint32_t)(i / S);
            const int slot = (int)(i % kRing);
            const uint32_t ur = (uint32_t)(i / kRing);
            bool good = true;
            if (u > 0) good = mbar_wait(smem_u32(bars + S + s), (u - 1) & 1u, deadline, abort_flag);
            if (good) good = mbar_wait(smem_u32(ring_full + slot), ur & 1u, deadline, abort_flag);
            if (!good) {
                *abort_flag = 1;
                atomicOr(&g_device_error, 1u);
            }
            named_sync(1, kProducers);  // every producer sees the same abort state
            if (*abort_flag) {
                ok = false;
                break;
            }
            unsigned char *st = tiles + (size_t)s * P.stage_bytes;
            for (int off = ptid * 16; off < P.stage_bytes; off += kProducers * 16)
                *reinterpret_cast<uint4 *>(st + off) = make_uint4(0u, 0u, 0u, 0u);
            named_sync(1, kProducers);
            unsigned char *A_hi = st, *B_hi = st + a_bytes;
            unsigned char *A_lo = st + a_bytes + b_bytes, *B_lo = A_lo + a_bytes;
            const int *h = hdr + 8 * slot;
            const int ha = h[0], na = h[1], hb = h[2], nb = h[3], overflow = h[4];
            const int2 *ent = reinterpret_cast<const int2 *>(ring + (size_t)slot * P.slot_bytes);
            const int2 *gent = P.bkt + (slab0 + i) * (int64_t)kSlab * P.m;
            const int total = na + nb;
            for (int e = ptid; e < total; e += kProducers) {
                const bool isA = e < na;
                int2 x;
                if (!overflow) {
                    x = isA ? ent[ha + e] : ent[hb + (e - na)];
                } else {
                    x = isA ? __ldg(gent + ha + e) : __ldg(gent + hb + (e - na));
                }
                const int c = x.x >> 14;
                const uint32_t off = (uint32_t)(x.x & 16383);
                const float v = __int_as_float(x.y);
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
            // generic-proxy writes -> visible to the tensor core (async proxy);
            // the ring slot is free once every producer is past this point
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            named_sync(1, kProducers);
            if (ptid == 0) {
                mbar_arrive(smem_u32(bars + s));
                mbar_arrive(smem_u32(ring_empty + slot));
            }
            // lagging one chunk behind the MMAs: add chunk c-1 into the registers
            // while the tensor core works on chunk c
            if ((i % kChunkSlabs) == kChunkSlabs - 1) {
                const int64_t c = i / kChunkSlabs;
                if (c >= 1 && consumed == c - 1) {
                    if (!consume(c - 1)) {
                        ok = false;
                        break;
                    }
                    consumed = c;
                }
            }
        }
        // the remaining chunks
        while (ok && consumed < nchunks) {
            if (!consume(consumed)) break;
            ++consumed;
        }
        // ---------------- epilogue: TMEM -> FP64 Gram
        const bool have = nslabs > 0;
        bool drained = false;
        if (have) drained = mbar_wait(done_bar, 0u, deadline + P.wait_cycles, abort_flag);
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
        if (have && drained && !*abort_flag && has_cols) {
            const int row = I0 + q * 32 + lane;
            const int col0 = J0 + hcol * 128;
            if (row < P.pt) {
                double *g = P.G + (int64_t)row * P.pt + col0;
#pragma unroll
                for (int j = 0; j < 128; ++j)
                    if (acc[j] != 0.f && col0 + j < P.pt) atomicAdd(g + j, (double)acc[j]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
}

__global__ void __launch_bounds__(kThreads, 1) gram_tc_kernel(TcParams P) {
    gram_tc_body(P, blockIdx.x);
}

// Many data sets in one launch: CTA b runs unit b - start[d] (tile and row
// split) of data set d with start[d] <= b < start[d + 1]; all data sets share
// the tile width, the precision mode and the ring layout.
__global__ void __launch_bounds__(kThreads, 1) gram_tc_batch_kernel(const TcParams *Ps,
                                                                   const int *start, int nd) {
    int lo = 0, hi = nd - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    const TcParams P = Ps[lo];
    gram_tc_body(P, (int)blockIdx.x - start[lo]);
}

}  // namespace

int64_t gram_tc_workspace(const sk_ctx &c, int64_t n) {
    if (n <= 0) return 0;
    const int64_t nslab = (n + kSlab - 1) / kSlab;
    const int64_t nblk = (c.pt + kBlk - 1) / kBlk;
    const int64_t ent = nslab * kSlab * c.m * (int64_t)sizeof(int2);
    const int64_t offs = nslab * (nblk + 1) * (int64_t)sizeof(int);
    return ((ent + 255) & ~int64_t(255)) + offs + 256;
}

// Launch configuration of one data set's Gram (no launch): tile shape,
// precision stages, row splits, ring slot size and the workspace carve.
static cudaError_t tc_plan(const sk_ctx &c, int mode, const int32_t *idx, const float *val,
                           int64_t n, double *G, void *work, TcParams &P, size_t &smem,
                           int64_t &nslab) {
    if (c.pt < kTileM) return cudaErrorInvalidValue;
    P.idx = idx;
    P.val = val;
    P.n = n;
    P.m = (int)c.m;
    P.pt = (int)c.pt;
    // column tiles of 256 (128 below pt = 256 or when autotuned); a pt that is
    // not a multiple of the tile sizes leaves ragged last blocks whose extra
    // rows and columns hold no entries
    P.N = c.pt >= 256 ? 256 : 128;
    if (c.gram_n == 128 && c.pt >= 128) P.N = 128;  // autotuned tile width
    P.nbi = (P.pt + kTileM - 1) / kTileM;
    P.nbj = (P.pt + P.N - 1) / P.N;
    const int ratio = P.N / kTileM;
    P.ntiles = 0;
    for (int bi = 0; bi < P.nbi; ++bi) P.ntiles += P.nbj - bi / ratio;
    P.hilo = (mode == SK_GRAM_BF16X3) ? 1 : 0;
    P.stage_bytes = (kTileM + P.N) * 128 * (P.hilo ? 2 : 1);
    P.nstages = P.hilo ? 2 : 4;
    if (P.N == 128 && !P.hilo) P.nstages = 6;
    if (P.N == 128 && P.hilo) P.nstages = 3;
    P.G = G;
    P.wait_cycles = wait_limit_cycles();
    P.nblk = (P.pt + kBlk - 1) / kBlk;
    // workspace: bucketed entries (8 bytes each, 64 m per slab), then offsets
    nslab = (n + kSlab - 1) / kSlab;
    const int64_t ent = nslab * kSlab * c.m * (int64_t)sizeof(int2);
    unsigned char *w = static_cast<unsigned char *>(work);
    P.bkt = reinterpret_cast<const int2 *>(w);
    P.boff = reinterpret_cast<const int *>(w + ((ent + 255) & ~int64_t(255)));

    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // row splits: no segment longer than kSegmentRows; among the counts that
    // allow, take the one whose units fill whole waves of the SMs best
    // (times the autotuned multiplier)
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
    if (c.split_mult > 1) {
        const int64_t cap = (n + kSlab - 1) / kSlab;
        best = best * c.split_mult < cap ? best * c.split_mult : cap;
    }
    int64_t rps = (n + best - 1) / best;
    rps = (rps + kSlab - 1) / kSlab * kSlab;
    P.rows_per_split = rps;
    P.nsplits = (int)((n + rps - 1) / rps);
    int smem_max = 0;
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // Dense rows (large m / pt) bring many entries per slab: a ring slot must
    // hold one slab's A and B ranges (on average e = 64 m (128 + N) / pt
    // entries of 8 bytes) or the producers fall back to scattered global
    // reads.  Give up operand stages (down to two) until e plus four standard
    // deviations (sqrt(e), the counts being near-binomial) fits a slot.
    const double slab_entries = 64.0 * (double)c.m * (double)(kTileM + P.N) / (double)c.pt;
    const int64_t need = (int64_t)((slab_entries + 4.0 * sqrt(slab_entries)) * 8.0) + 256;
    while (P.nstages > 2 &&
           ((int64_t)smem_max - (int64_t)P.nstages * P.stage_bytes - 1536) / kRing < need)
        --P.nstages;
    const size_t fixed = (size_t)P.nstages * P.stage_bytes + 1024 + 512;
    int64_t slot = ((int64_t)smem_max - (int64_t)fixed) / kRing;
    slot = slot / 16 * 16;
    if (slot > 65536) slot = 65536;
    if (slot < 16) return cudaErrorInvalidConfiguration;
    P.slot_bytes = (int)slot;
    smem = fixed + (size_t)kRing * P.slot_bytes;
    return cudaSuccess;
}

cudaError_t launch_gram_tc(const sk_ctx &c, int mode, const int32_t *idx, const float *val,
                           int64_t n, double *G, void *work, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    TcParams P;
    size_t smem = 0;
    int64_t nslab = 0;
    cudaError_t e = tc_plan(c, mode, idx, val, n, G, work, P, smem, nslab);
    if (e != cudaSuccess) return e;
    bucket_kernel<<<(unsigned)nslab, 256, 0, s>>>(idx, val, n, P.m, P.pt, P.nblk,
                                                  const_cast<int2 *>(P.bkt),
                                                  const_cast<int *>(P.boff));
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = (int64_t)P.ntiles * P.nsplits;
    gram_tc_kernel<<<(unsigned)grid, kThreads, smem, s>>>(P);
    return cudaGetLastError();
}

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

cudaError_t gram_batch_build(const sk_ctx *ctxs, const BatchGram *rows, int nd, int mode,
                             std::vector<unsigned char> &table, GramBatchInfo &info) {
    std::vector<TcParams> Ps((size_t)nd);
    std::vector<BucketParams> Bs((size_t)nd);
    std::vector<int> slab_start((size_t)nd + 1), cta_start((size_t)nd + 1);
    int64_t slabs = 0, ctas = 0;
    size_t smem = 0;
    // Each data set keeps its own plan (tile width, operand stages, ring slot
    // size): a CTA carves its shared memory from its data set's parameters,
    // and the launch provides the largest plan's size.
    for (int d = 0; d < nd; ++d) {
        TcParams &P = Ps[d];
        size_t sm = 0;
        int64_t nslab = 0;
        slab_start[d] = (int)slabs;
        cta_start[d] = (int)ctas;
        if (rows[d].n == 0) {
            std::memset(&P, 0, sizeof(P));
            std::memset(&Bs[d], 0, sizeof(BucketParams));
            continue;
        }
        cudaError_t e = tc_plan(ctxs[d], mode, rows[d].idx, rows[d].val, rows[d].n, rows[d].G,
                                rows[d].work, P, sm, nslab);
        if (e != cudaSuccess) return e;
        if (!smem) info.first = d;
        if (sm > smem) smem = sm;
        Bs[d] = BucketParams{rows[d].idx, rows[d].val, rows[d].n, P.m, P.pt, P.nblk,
                             const_cast<int2 *>(P.bkt), const_cast<int *>(P.boff)};
        slabs += nslab;
        ctas += (int64_t)P.ntiles * P.nsplits;
        if (slabs > 0x7fffffff || ctas > 0x7fffffff) return cudaErrorInvalidValue;
    }
    slab_start[nd] = (int)slabs;
    cta_start[nd] = (int)ctas;
    info.nd = nd;
    info.slabs = slabs;
    info.ctas = ctas;
    info.smem = smem;
    info.tc_off = al256(table.size());
    info.bk_off = al256(info.tc_off + Ps.size() * sizeof(TcParams));
    info.slab_off = al256(info.bk_off + Bs.size() * sizeof(BucketParams));
    info.cta_off = al256(info.slab_off + slab_start.size() * sizeof(int));
    table.resize(al256(info.cta_off + cta_start.size() * sizeof(int)), 0);
    std::memcpy(table.data() + info.tc_off, Ps.data(), Ps.size() * sizeof(TcParams));
    std::memcpy(table.data() + info.bk_off, Bs.data(), Bs.size() * sizeof(BucketParams));
    std::memcpy(table.data() + info.slab_off, slab_start.data(), slab_start.size() * sizeof(int));
    std::memcpy(table.data() + info.cta_off, cta_start.data(), cta_start.size() * sizeof(int));
    if (smem) {
        cudaError_t e = cudaFuncSetAttribute(gram_tc_batch_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t gram_batch_launch(const GramBatchInfo &info, unsigned char *dev_table, cudaStream_t s) {
    if (info.ctas == 0) return cudaSuccess;
    bucket_batch_kernel<<<(unsigned)info.slabs, 256, 0, s>>>(
        reinterpret_cast<const BucketParams *>(dev_table + info.bk_off),
        reinterpret_cast<const int *>(dev_table + info.slab_off), info.nd);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    gram_tc_batch_kernel<<<(unsigned)info.ctas, kThreads, info.smem, s>>>(
        reinterpret_cast<const TcParams *>(dev_table + info.tc_off),
        reinterpret_cast<const int *>(dev_table + info.cta_off), info.nd);
    return cudaGetLastError();
}

}  // namespace sk
