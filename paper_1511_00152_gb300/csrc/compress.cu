// compress.cu -- fused one-pass compression (Sec. III Eq. (ROS); Algorithm 1,
// lines "Y <- HDX" and "w_i = R_i R_i^T y_i").
//
// One pass over X: each sample is read once from HBM (coalesced 16-byte
// loads), signed by D, transformed by the orthonormal Sylvester
// Walsh-Hadamard matrix, and the m entries of its mask are gathered into the
// ELL output.  The transform runs on a 1024-element "unit" per warp: phase A
// does the butterflies on element bits {0,1,7,8,9} in registers (the layout a
// float4 load gives), a padded shared-memory transpose brings bits {2..6}
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
#include <algorithm>
#include <cstring>
#include <vector>

#include <type_traits>

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
    int mix;            // 0: no preconditioning (H = D = I), the ablation of Sec. VII
    unsigned int *err;  // device error word (bounded waits)
    int ctas_per_sm;    // autotuned residency cap (0: as many as fit)
    long long wait_cycles;  // limit of each bounded mbarrier wait (SM clock cycles)
    int mask_pt;        // range of the masks: pt (2^L, or p with the DCT)
};

constexpr int kNB = 2;  // staging buffers per warp (one unit in flight ahead)

// One task of the multi-data-set launch: units [u_begin, u_end) of data set d.
struct CompressTask {
    int32_t d;
    int32_t L;
    int64_t u_begin;
    int64_t u_end;
};
// Default limit of a bounded wait (~2 s at 2 GHz); copies still in flight
// after a wait ran out are always drained with this limit.
constexpr long long kWaitCycles = 4000000000LL;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Waits for the phase of the given parity for at most `limit` cycles.  The
// first test does not block, so a phase still pending when the limit is
// already over is reported as a wait that ran out (false).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, long long limit) {
    const long long deadline = clock64() + limit;
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

// Stage the raw samples of one unit into buf with 1D bulk copies (TMA),
// completing on bar.  Lane 0 sets the expected byte count first.
template <int L>
__device__ __forceinline__ void issue_unit(const CompressParams &P, int64_t u, int wg, float *buf,
                                           uint32_t bar, int lane) {
    constexpr int PT = 1 << L;
    constexpr int RPU = (L <= 10) ? (1024 >> L) : 1;
    int64_t r0 = u * RPU;
    int rows = (int)((P.n - r0) < RPU ? (P.n - r0) : RPU);
    int cols, c0;
    if constexpr (L <= 10) {
        c0 = 0;
        cols = (int)P.p;
    } else {
        c0 = 1024 * wg;
        cols = (int)(P.p - c0 < 1024 ? P.p - c0 : 1024);
        if (cols < 0) cols = 0;
    }
    const uint32_t bytes_row = (uint32_t)cols * 4u;
    const bool contiguous = (L <= 10) && P.ldx == PT && P.p == PT;
    const uint32_t total = (uint32_t)rows * bytes_row;
    if (lane == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(total)
                     : "memory");
    }
    __syncwarp();
    if (total == 0) return;
    if (contiguous) {
        if (lane == 0) {
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_u32(buf)),
                "l"(P.X + r0 * P.ldx), "r"(total), "r"(bar)
                : "memory");
        }
    } else {
        for (int b = lane; b < rows; b += 32) {
            const float *src = P.X + (r0 + b) * P.ldx + c0;
            float *dst = buf + ((L <= 10) ? b * PT : 0);
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_u32(dst)),
                "l"(src), "r"(bytes_row), "r"(bar)
                : "memory");
        }
    }
}

// Shared-memory slot of unit element e: four floats of padding after every
// 128 elements.  The float4 rows of phase A (e = 128 ip + 4 lane) and the
// stride-4 columns of phase B (e = 128 ib + 4 j + q, bank 4 ib + q + 4 j) are
// then bank-conflict free, and each access is a per-lane base plus a
// compile-time offset (no per-access address arithmetic).  A 1024-element
// unit segment takes kSeg floats.
constexpr int kSeg = 1024 + 32;
__device__ __forceinline__ int phys(int e) { return e + ((e >> 7) << 2); }

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
        return (c >> 10) * kSeg + phys(c & 1023);
    }
}

// Packed FP32 pairs (two independent IEEE round-to-nearest operations each).
__device__ __forceinline__ uint64_t pk2(float lo, float hi) {
    return ((uint64_t)__float_as_uint(hi) << 32) | __float_as_uint(lo);
}
__device__ __forceinline__ float lo2(uint64_t a) { return __uint_as_float((uint32_t)a); }
__device__ __forceinline__ float hi2(uint64_t a) { return __uint_as_float((uint32_t)(a >> 32)); }

// Butterfly stage on bit rb of the 32-element register index r (element r is
// component r&1 of pair r>>1): rb = 0 pairs the two halves of one register
// pair, rb >= 1 pairs whole register pairs with packed add/sub.
template <int NPAIR>
__device__ __forceinline__ void wht_stage(uint64_t (&w)[NPAIR], int rb) {
    if (rb == 0) {
#pragma unroll
        for (int P = 0; P < NPAIR; ++P) {
            const float a = lo2(w[P]), b = hi2(w[P]);
            w[P] = pk2(a + b, a - b);
        }
    } else {
        const int pb = 1 << (rb - 1);
#pragma unroll
        for (int P = 0; P < NPAIR; ++P) {
            if (!(P & pb)) {
                uint64_t sm, df;
                asm("add.rn.f32x2 %0, %1, %2;" : "=l"(sm) : "l"(w[P]), "l"(w[P | pb]));
                asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(df) : "l"(w[P]), "l"(w[P | pb]));
                w[P] = sm;
                w[P | pb] = df;
            }
        }
    }
}

// Entries of the virtual Fisher-Yates array: the value a position holds and
// the tag of the row that wrote it; a position whose tag is not the current
// row's still holds its own index.  32-bit entries: 16-bit tag and value.
// 16-bit entries (the masks-alone kernel, L <= 13): an L-bit value and a
// (16 - L)-bit tag, so the array is cleared every kTagMax rows.
template <typename AT, int L>
struct AEnt;
template <int L>
struct AEnt<uint32_t, L> {
    static constexpr uint32_t kTagMax = 0xFFFFu;
    __device__ static int read(const uint32_t *A, uint32_t tag, int j) {
        const uint32_t a = A[j];
        return (a >> 16) == tag ? (int)(a & 0xFFFFu) : j;
    }
    __device__ static void write(uint32_t *A, int k, uint32_t tag, int V) {
        A[k] = (tag << 16) | (uint32_t)V;
    }
};
template <int L>
struct AEnt<uint16_t, L> {
    static_assert(L <= 13, "16-bit entries leave at least three tag bits");
    static constexpr uint32_t kTagMax = (1u << (16 - L)) - 1u;
    __device__ static int read(const uint16_t *A, uint32_t tag, int j) {
        const uint32_t a = A[j];
        return (a >> L) == tag ? (int)(a & ((1u << L) - 1u)) : j;
    }
    __device__ static void write(uint16_t *A, int k, uint32_t tag, int V) {
        A[k] = (uint16_t)((tag << L) | (uint32_t)V);
    }
};

// Window of the row's mask-word stream: two batches of 128 words (one
// Philox block per lane per batch), batch b in slot b & 1.
struct WordWindow {
    uint32_t *words;  // 256 words of shared memory
    int have0, have1; // batch held by slot 0 / slot 1 (-1: none)
};

__device__ __forceinline__ void ensure_batches(WordWindow &ww, const CompressParams &P, uint64_t g,
                                               uint32_t wlo, uint32_t whi, int lane) {
    for (uint32_t b = wlo >> 7; b <= (whi >> 7); ++b) {
        int &have = (b & 1) ? ww.have1 : ww.have0;
        if (have == (int)b) continue;
        const uint4 o = philox4x32_10(
            make_uint4(b * 32u + (uint32_t)lane, (uint32_t)g, (uint32_t)(g >> 32), kTagMask), P.k0,
            P.k1);
        __syncwarp();
        *reinterpret_cast<uint4 *>(ww.words + (b & 1) * 128 + 4 * lane) = o;
        __syncwarp();
        have = (int)b;
    }
}

// Mask of one row and (GATHER) its ELL gather, by one warp.
template <int L, bool GATHER = true, typename AT = uint32_t>
__device__ __forceinline__ void sample_row(const CompressParams &P, int64_t i,
                                           const float *ybuf, int ebase, AT *A,
                                           uint32_t *hit, uint32_t *words, uint32_t tag, int lane) {
    // the range [0, PT) of the draw: 2^L, or (masks alone) p <= 2^L for the DCT
    const int PT = GATHER ? (1 << L) : P.mask_pt;
    const uint64_t g = (uint64_t)(P.row0 + i);
    const int m = P.m;
    int32_t *oidx = P.idx + i * (int64_t)m;
    float *oval = P.val + i * (int64_t)m;
    const unsigned lt = lanemask_lt();
    const unsigned gt = lanemask_gt();
    uint32_t woff = 0;
    WordWindow ww{words, -1, -1};
    for (int c0 = 0; c0 < m; c0 += 32) {
        const int t = c0 + lane;
        const bool act = t < m;
        const uint32_t s = (uint32_t)(PT - t);
        uint32_t w = (uint32_t)t + woff;
        uint64_t prod = 0;
        uint32_t wtop = (uint32_t)c0 + woff + 31;
        ensure_batches(ww, P, g, (uint32_t)c0 + woff, wtop, lane);
        if constexpr (GATHER) {
            for (;;) {
                const uint32_t word = act ? words[((w >> 7) & 1) * 128 + (w & 127)] : 0u;
                prod = (uint64_t)word * (uint64_t)s;
                bool rej = false;
                if (act && (uint32_t)prod < s) rej = (uint32_t)prod < ((0u - s) % s);
                const unsigned bal = __ballot_sync(kFull, rej);
                if (bal == 0u) break;
                const int first = __ffs(bal) - 1;
                if (lane >= first) ++w;
                ++woff;
                ++wtop;
                ensure_batches(ww, P, g, (uint32_t)c0 + woff, wtop, lane);
            }
        } else {
            // masks alone (mask_kernel): a rejection needs (L mod 2^32) < s
            // first, probability below s / 2^32; only if some lane meets it
            // is the exact threshold 2^32 mod s taken (same draws; measured
            // faster in this kernel, slower inside the fused one)
            uint32_t word = act ? words[((w >> 7) & 1) * 128 + (w & 127)] : 0u;
            prod = (uint64_t)word * (uint64_t)s;
            if (__any_sync(kFull, act && (uint32_t)prod < s)) {
                for (;;) {
                    bool rej = false;
                    if (act && (uint32_t)prod < s) rej = (uint32_t)prod < ((0u - s) % s);
                    const unsigned bal = __ballot_sync(kFull, rej);
                    if (bal == 0u) break;
                    const int first = __ffs(bal) - 1;
                    if (lane >= first) ++w;
                    ++woff;
                    ++wtop;
                    ensure_batches(ww, P, g, (uint32_t)c0 + woff, wtop, lane);
                    word = act ? words[((w >> 7) & 1) * 128 + (w & 127)] : 0u;
                    prod = (uint64_t)word * (uint64_t)s;
                }
            }
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
        // a row's first chunk finds every position still holding its own
        // index (the mask kernel skips that look-up)
        const int vbase = act ? ((GATHER || c0) ? AEnt<AT, L>::read(A, tag, t) : t) : 0;
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
        if (act) omega = prevm ? vprev : ((GATHER || c0) ? AEnt<AT, L>::read(A, tag, k) : k);
        __syncwarp();
        if (act && c0 + 32 < m && (grpm & gt) == 0u && k >= c0 + 32)
            AEnt<AT, L>::write(A, k, tag, V);
        if (act) {
            oidx[t] = omega;
            if constexpr (GATHER) oval[t] = ybuf[yaddr<L>(ebase, omega)] * P.scale;
        }
        __syncwarp();
    }
}

// Shared-memory layout: the fixed part first (mbarriers, each warp's
// mask-word window, one abort word per row group), so that the persistent
// multi-dataset kernel can run units of different pt back to back on the
// same barriers; then, per row group, the staging buffers, the virtual
// Fisher-Yates array and the hit table.
constexpr size_t kFixedSmem = (size_t)kWarps * kNB * 8 + (size_t)kWarps * 256 * 4 + (size_t)kWarps * 4;
static_assert(kFixedSmem % 16 == 0, "bulk-copy destinations stay 16-byte aligned");

template <int L, bool TMA, bool SPLIT = false>
constexpr size_t compress_smem_bytes() {
    constexpr int PT = 1 << L;
    constexpr int G = (L > 10) ? (PT >> 10) : 1;
    constexpr int NG = kWarps / G;
    constexpr int BUF = (L <= 10) ? kSeg : (PT >> 10) * kSeg;
    constexpr int NBUF = TMA ? kNB : 1;
    constexpr int NA = SPLIT ? 0 : PT;  // the mask kernel holds the Fisher-Yates arrays
    return kFixedSmem + (size_t)NG * NBUF * BUF * 4 + (size_t)NG * NA * 4 + (size_t)NG * 32 * 4;
}

__device__ __forceinline__ void init_unit_barriers(unsigned char *smem_raw) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem_raw) + warp * kNB;
    if (lane == 0)
        for (int b = 0; b < kNB; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar + b)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncwarp();
}

// One CTA processes units u = u0 + grp + k * stride (u < u_end) of the data
// set described by P: a unit is RPU rows (pt <= 1024, one warp each) or one
// row (pt > 1024, G warps).  kloc counts the units this warp has staged
// through its two TMA buffers (it carries the buffer / barrier-phase
// sequence across calls).  SPLIT (pt > 1024): the masks are already in
// P.idx (mask_kernel) and all G warps of the row share its gather.  Returns
// false if a bounded wait ran out.
template <int L, bool DENSE, bool TMA, bool SPLIT = false>
__device__ __forceinline__ bool compress_units(const CompressParams &P, int64_t u0,
                                               int64_t stride, int64_t u_end,
                                               unsigned char *smem_raw, int64_t &kloc) {
    constexpr int PT = 1 << L;
    constexpr int G = (L > 10) ? (PT >> 10) : 1;  // warps per row group
    constexpr int NG = kWarps / G;                // row groups per CTA
    constexpr int RPU = (L <= 10) ? (1024 >> L) : 1;
    constexpr int BUF = (L <= 10) ? kSeg : (PT >> 10) * kSeg;
    constexpr int NBUF = TMA ? kNB : 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = warp / G, wg = warp % G;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem_raw) + warp * kNB;
    uint32_t *words = reinterpret_cast<uint32_t *>(smem_raw + (size_t)kWarps * kNB * 8) + warp * 256;
    // set by any warp of the row group whose wait ran out: the group's warps
    // share each wait's outcome and leave together (pt > 1024)
    volatile int *abort_word = reinterpret_cast<volatile int *>(
                                   smem_raw + (size_t)kWarps * kNB * 8 + (size_t)kWarps * 256 * 4) +
                               grp;
    unsigned char *var = smem_raw + kFixedSmem;
    float *ybufs = reinterpret_cast<float *>(var) + grp * NBUF * BUF;
    float *ybuf = ybufs;
    unsigned char *after = var + (size_t)NG * NBUF * BUF * 4;
    uint32_t *A = reinterpret_cast<uint32_t *>(after) + grp * PT;
    uint32_t *hit = reinterpret_cast<uint32_t *>(after + (size_t)NG * (SPLIT ? 0 : PT) * 4) + grp * 32;
    static_assert(!SPLIT || (L > 10 && !DENSE), "split masks: pt > 1024, ELL output");

    if constexpr (!DENSE && !SPLIT) {
        if (wg == 0)
            for (int j = lane; j < PT; j += 32) A[j] = 0u;
    }
    uint32_t tag = 1;

    // Sign bits of the 32 coordinates this thread holds in phase A.
    uint32_t smask = 0;
#pragma unroll 1
    for (int r = 0; r < (P.mix ? 32 : 0); ++r) {
        const int e = 128 * (r >> 2) + 4 * lane + (r & 3);
        const int c = (L <= 10) ? (e & (PT - 1)) : (1024 * wg + e);
        smask |= sign_bit(P.k0, P.k1, (uint32_t)c) << r;
    }

    const int64_t nunits = u_end;
    const int64_t u_first = u0 + grp;
    bool ok = true;
    if constexpr (TMA) {
        if (wg == 0 && lane == 0) *abort_word = 0;
        // the buffer may have been read by the previous call's gathers
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        group_sync<G>(grp);
        if (u_first < nunits) {
            const int b0 = (int)(kloc & 1);
            issue_unit<L>(P, u_first, wg, ybufs + b0 * BUF + ((L > 10) ? kSeg * wg : 0),
                          smem_u32(mbar + b0), lane);
        }
    }
    // SPLIT: the first kMI of this lane's sampled coordinates of the row,
    // fetched before its transform so that their latency hides behind it
    constexpr int kMI = SPLIT ? 2 : 1;
    for (int64_t u = u_first; u < nunits; u += stride, ++kloc) {
        const int64_t r0 = u * RPU;
        int jv[kMI];
        if constexpr (SPLIT) {
            if (r0 < P.n) {
                const int32_t *gi = P.idx + r0 * (int64_t)P.m;
#pragma unroll
                for (int q = 0; q < kMI; ++q) {
                    const int t = wg * 32 + lane + q * G * 32;
                    jv[q] = t < P.m ? __ldcg(gi + t) : 0;
                }
            }
        }
        float v[32];
        if constexpr (TMA) {
            const int bsel = (int)(kloc & 1);
            ybuf = ybufs + bsel * BUF;
            // the other buffer's last reader (previous unit's gathers) is done
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            group_sync<G>(grp);
            if (u + stride < nunits)
                issue_unit<L>(P, u + stride, wg, ybufs + (bsel ^ 1) * BUF + ((L > 10) ? kSeg * wg : 0),
                              smem_u32(mbar + (bsel ^ 1)), lane);
            bool landed = mbar_wait_bounded(smem_u32(mbar + bsel), (uint32_t)((kloc >> 1) & 1),
                                            P.wait_cycles);
            if constexpr (G > 1) {
                // one outcome for the whole row group, so that no warp of it
                // waits at a group barrier for a warp that has left
                if (!landed && lane == 0) *abort_word = 1;
                group_sync<G>(grp);
                landed = *abort_word == 0;
            }
            if (!landed) {
                if (lane == 0 && P.err) atomicOr(P.err, 2u);
                // before leaving, wait (bounded, default limit) for this
                // warp's copies still in flight: this unit's and the next one's
                mbar_wait_bounded(smem_u32(mbar + bsel), (uint32_t)((kloc >> 1) & 1), kWaitCycles);
                if (u + stride < nunits)
                    mbar_wait_bounded(smem_u32(mbar + (bsel ^ 1)), (uint32_t)(((kloc + 1) >> 1) & 1),
                                      kWaitCycles);
                ok = false;
                break;
            }
            float *wb = ybuf + ((L > 10) ? kSeg * wg : 0);
            // zero what the copies did not fill: padding columns and rows past n
            const bool ragged = (L <= 10) ? (r0 + RPU > P.n) : false;
            const int cend = (L <= 10) ? (int)P.p : (int)(P.p - 1024 * wg);
            if (ragged || cend < ((L <= 10) ? PT : 1024)) {
                for (int e = lane; e < 1024; e += 32) {
                    const int b = (L <= 10) ? (e >> L) : 0;
                    const int c = (L <= 10) ? (e & (PT - 1)) : e;
                    if (r0 + b >= P.n || c >= cend) wb[e] = 0.f;
                }
                __syncwarp();
            }
#pragma unroll
            for (int ip = 0; ip < 8; ++ip) {
                const float4 x4 = *reinterpret_cast<const float4 *>(wb + 128 * ip + 4 * lane);
                v[4 * ip + 0] = x4.x;
                v[4 * ip + 1] = x4.y;
                v[4 * ip + 2] = x4.z;
                v[4 * ip + 3] = x4.w;
            }
        } else {
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
        }
        // ---- D: flip the sign bit where D_j = -1; pack into register pairs
        uint64_t w2[16];
#pragma unroll
        for (int P2 = 0; P2 < 16; ++P2) {
            const uint32_t a = __float_as_uint(v[2 * P2]) ^ (((smask >> (2 * P2)) & 1u) << 31);
            const uint32_t b = __float_as_uint(v[2 * P2 + 1]) ^ (((smask >> (2 * P2 + 1)) & 1u) << 31);
            w2[P2] = ((uint64_t)b << 32) | a;
        }
        // ---- phase A: register bit rb <-> element bit {0,1,7,8,9}[rb]
        if (P.mix) {
#pragma unroll
            for (int rb = 0; rb < 5; ++rb) {
                const int eb = rb < 2 ? rb : rb + 5;
                if (eb < L) wht_stage<16>(w2, rb);
            }
        }
        // every lane has read its samples (TMA) / previous gathers are done
        group_sync<G>(grp);
        float *wbuf = ybuf + ((L > 10) ? kSeg * wg : 0);
#pragma unroll
        for (int ip = 0; ip < 8; ++ip) {
            const int e = 128 * ip + 4 * lane;
            *reinterpret_cast<float4 *>(wbuf + phys(e)) =
                make_float4(lo2(w2[2 * ip]), hi2(w2[2 * ip]), lo2(w2[2 * ip + 1]), hi2(w2[2 * ip + 1]));
        }
        __syncwarp();
        // ---- phase B: lane = (q, i''), register j <-> element bits 2..6
        if (P.mix) {
            const int q = lane & 3, ib = lane >> 2;
#pragma unroll
            for (int P2 = 0; P2 < 16; ++P2)
                w2[P2] = pk2(wbuf[phys(128 * ib + 4 * (2 * P2) + q)],
                             wbuf[phys(128 * ib + 4 * (2 * P2 + 1) + q)]);
#pragma unroll
            for (int rb = 0; rb < 5; ++rb)
                if (rb + 2 < L) wht_stage<16>(w2, rb);
#pragma unroll
            for (int P2 = 0; P2 < 16; ++P2) {
                wbuf[phys(128 * ib + 4 * (2 * P2) + q)] = lo2(w2[P2]);
                wbuf[phys(128 * ib + 4 * (2 * P2 + 1) + q)] = hi2(w2[P2]);
            }
        }
        // ---- phase C (pt > 1024): element bits 10.. across the group's warps
        if (L > 10 && P.mix) {
            constexpr int S = 32 / G;
            group_sync<G>(grp);
            const int tau = wg * 32 + lane;
#pragma unroll
            for (int s2 = 0; s2 < S; ++s2)
#pragma unroll
                for (int w3 = 0; w3 < G; w3 += 2)
                    w2[(s2 * G + w3) >> 1] = pk2(ybuf[kSeg * w3 + phys(tau + 32 * G * s2)],
                                                 ybuf[kSeg * (w3 + 1) + phys(tau + 32 * G * s2)]);
#pragma unroll
            for (int rb = 0; (1 << rb) < G; ++rb) wht_stage<16>(w2, rb);
#pragma unroll
            for (int s2 = 0; s2 < S; ++s2)
#pragma unroll
                for (int w3 = 0; w3 < G; w3 += 2) {
                    ybuf[kSeg * w3 + phys(tau + 32 * G * s2)] = lo2(w2[(s2 * G + w3) >> 1]);
                    ybuf[kSeg * (w3 + 1) + phys(tau + 32 * G * s2)] = hi2(w2[(s2 * G + w3) >> 1]);
                }
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
        } else if constexpr (SPLIT) {
            // one row: its m entries are shared by the G warps of the group
            if (r0 < P.n) {
                const int m = P.m;
                const int32_t *gi = P.idx + r0 * (int64_t)m;
                float *ov = P.val + r0 * (int64_t)m;
#pragma unroll
                for (int q = 0; q < kMI; ++q) {
                    const int t = wg * 32 + lane + q * G * 32;
                    if (t < m) ov[t] = ybuf[yaddr<L>(0, jv[q] & (PT - 1))] * P.scale;
                }
                for (int t = wg * 32 + lane + kMI * G * 32; t < m; t += G * 32)
                    ov[t] = ybuf[yaddr<L>(0, __ldcg(gi + t) & (PT - 1))] * P.scale;
            }
        } else {
            if (L <= 10 || wg == 0) {
#pragma unroll 1
                for (int b = 0; b < RPU; ++b) {
                    const int64_t i = r0 + b;
                    if (i >= P.n) break;
                    sample_row<L>(P, i, ybuf, b * PT, A, hit, words, tag, lane);
                    if (++tag == 0x10000u) {
                        for (int j = lane; j < PT; j += 32) A[j] = 0u;
                        __syncwarp();
                        tag = 1;
                    }
                }
            }
        }
    }
    return ok;
}

template <int L, bool DENSE, bool TMA, bool SPLIT = false>
__global__ void __launch_bounds__(kWarps * 32, 2) compress_kernel(CompressParams P) {
    constexpr int PT = 1 << L;
    constexpr int G = (L > 10) ? (PT >> 10) : 1;
    constexpr int NG = kWarps / G;
    constexpr int RPU = (L <= 10) ? (1024 >> L) : 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if constexpr (TMA) init_unit_barriers(smem_raw);
    const int64_t nunits = (L <= 10) ? (P.n + RPU - 1) / RPU : P.n;
    int64_t kloc = 0;
    compress_units<L, DENSE, TMA, SPLIT>(P, (int64_t)blockIdx.x * NG, (int64_t)gridDim.x * NG,
                                         nunits, smem_raw, kloc);
}

// Masks only (pt > 1024): every warp draws whole rows on its own (its own
// virtual Fisher-Yates array and word window) and writes idx; the transform
// kernel then gathers val with all the warps of a row group.  At pt > 1024 a
// row's transform takes G = pt / 1024 warps, and drawing its mask on one of
// them left the other G - 1 waiting.
template <int L>
__host__ __device__ constexpr int mask_warps() { return L >= 13 ? 2 : 4; }

// the masks-alone kernel's virtual Fisher-Yates entries: 16 bits while a
// position fits 13 bits (half the shared memory per warp, twice the warps)
template <int L>
using MaskAT = typename std::conditional<(L <= 13), uint16_t, uint32_t>::type;

template <int L>
constexpr size_t mask_smem_bytes() {
    return (size_t)mask_warps<L>() * (256 * 4 + (1 << L) * sizeof(MaskAT<L>) + 32 * 4);
}

template <int L>
__global__ void __launch_bounds__(mask_warps<L>() * 32) mask_kernel(CompressParams P) {
    constexpr int PT = 1 << L;
    constexpr int MW = mask_warps<L>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    using AT = MaskAT<L>;
    uint32_t *words = reinterpret_cast<uint32_t *>(smem_raw) + warp * 256;
    AT *A = reinterpret_cast<AT *>(smem_raw + (size_t)MW * 256 * 4) + warp * PT;
    uint32_t *hit = reinterpret_cast<uint32_t *>(smem_raw + (size_t)MW * (256 * 4 + PT * sizeof(AT))) +
                    warp * 32;
    for (int j = lane; j < PT; j += 32) A[j] = 0;
    __syncwarp();
    uint32_t tag = 1;
    for (int64_t i = (int64_t)blockIdx.x * MW + warp; i < P.n; i += (int64_t)gridDim.x * MW) {
        sample_row<L, false, AT>(P, i, nullptr, 0, A, hit, words, tag, lane);
        if (++tag > AEnt<AT, L>::kTagMax) {
            __syncwarp();
            for (int j = lane; j < PT; j += 32) A[j] = 0;
            __syncwarp();
            tag = 1;
        }
    }
}

template <int L>
cudaError_t launch_masks(const CompressParams &P, cudaStream_t s) {
    const size_t smem = mask_smem_bytes<L>();
    auto kern = mask_kernel<L>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, mask_warps<L>() * 32, smem);
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (P.n + mask_warps<L>() - 1) / mask_warps<L>();
    const int64_t cap = (int64_t)sms * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, mask_warps<L>() * 32, smem, s>>>(P);
    return cudaGetLastError();
}

template <int L, bool DENSE, bool TMA, bool SPLIT = false>
cudaError_t launch_LT(const CompressParams &P, cudaStream_t s) {
    constexpr int PT = 1 << L;
    constexpr int G = (L > 10) ? (PT >> 10) : 1;
    constexpr int NG = kWarps / G;
    constexpr int RPU = (L <= 10) ? (1024 >> L) : 1;
    const size_t smem = compress_smem_bytes<L, TMA, SPLIT>();
    auto kern = compress_kernel<L, DENSE, TMA, SPLIT>;
    cudaError_t e0 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem);
    if (e0 != cudaSuccess) return e0;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWarps * 32, smem);
    if (per_sm < 1) per_sm = 1;
    const int64_t nunits = (L <= 10) ? (P.n + RPU - 1) / RPU : P.n;
    int64_t blocks = (nunits + NG - 1) / NG;
    if (P.ctas_per_sm > 0 && P.ctas_per_sm < per_sm) per_sm = P.ctas_per_sm;
    const int64_t cap = (int64_t)sms * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, kWarps * 32, smem, s>>>(P);
    return cudaGetLastError();
}

template <int L, bool DENSE>
cudaError_t launch_L(const CompressParams &P, cudaStream_t s) {
    // bulk copies need 16-byte aligned rows whose byte length is a multiple of 16
    if constexpr (L >= 2) {
        if (P.vec) {
            if constexpr (L > 10 && !DENSE) {
                cudaError_t e = launch_masks<L>(P, s);
                if (e != cudaSuccess) return e;
                return launch_LT<L, false, true, true>(P, s);
            }
            return launch_LT<L, DENSE, true>(P, s);
        }
    }
    return launch_LT<L, DENSE, false>(P, s);
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

// ---- many data sets in one persistent launch
//
// The work is a list of tasks (data set, unit range) of about the same
// number of bytes; persistent CTAs take tasks in order from a ticket counter
// and run them with the pt-specific unit code (TMA staging only: every data
// set has 16-byte aligned rows).  Between tasks the CTA synchronises, so the
// shared memory of one task's layout is free before the next one's.
__global__ void __launch_bounds__(kWarps * 32, 2) compress_batch_kernel(
    const CompressParams *Ps, const CompressTask *tasks, int ntasks, unsigned int *ticket) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_task;
    init_unit_barriers(smem_raw);
    int64_t kloc = 0;
    for (;;) {
        if (threadIdx.x == 0) s_task = (int)atomicAdd(ticket, 1u);
        __syncthreads();
        const int t = s_task;
        if (t >= ntasks) break;
        const CompressTask T = tasks[t];
        const CompressParams P = Ps[T.d];
        bool ok = true;
        switch (T.L) {
#define SK_BATCH_CASE(LL)                                                                        \
    case LL:                                                                                     \
        ok = compress_units<LL, false, true>(P, T.u_begin, kWarps / ((LL > 10) ? (1 << (LL - 10)) \
                                                                                : 1),            \
                                             T.u_end, smem_raw, kloc);                          \
        break;
            SK_BATCH_CASE(2)
            SK_BATCH_CASE(3)
            SK_BATCH_CASE(4)
            SK_BATCH_CASE(5)
            SK_BATCH_CASE(6)
            SK_BATCH_CASE(7)
            SK_BATCH_CASE(8)
            SK_BATCH_CASE(9)
            SK_BATCH_CASE(10)
            SK_BATCH_CASE(11)
            SK_BATCH_CASE(12)
            SK_BATCH_CASE(13)
#undef SK_BATCH_CASE
            default:
                break;
        }
        // every group is done with this task's shared memory (and has read
        // s_task) before the next task starts
        if (__syncthreads_or(!ok)) break;
    }
}

size_t compress_smem_for(int L) {
    switch (L) {
        case 2: return compress_smem_bytes<2, true>();
        case 3: return compress_smem_bytes<3, true>();
        case 4: return compress_smem_bytes<4, true>();
        case 5: return compress_smem_bytes<5, true>();
        case 6: return compress_smem_bytes<6, true>();
        case 7: return compress_smem_bytes<7, true>();
        case 8: return compress_smem_bytes<8, true>();
        case 9: return compress_smem_bytes<9, true>();
        case 10: return compress_smem_bytes<10, true>();
        case 11: return compress_smem_bytes<11, true>();
        case 12: return compress_smem_bytes<12, true>();
        default: return compress_smem_bytes<13, true>();
    }
}

}  // namespace

static CompressParams make_params(const sk_ctx &c, const float *X, int64_t n, int64_t ldx,
                                  int64_t row0, int32_t *idx, float *val, float *Y) {
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
    P.mix = (c.flags & SK_FLAG_NO_PRECONDITION) ? 0 : 1;
    P.scale = P.mix ? (float)(1.0 / sqrt((double)c.pt)) : 1.0f;
    P.vec = ((reinterpret_cast<uintptr_t>(X) & 15) == 0) && (c.p % 4 == 0) && (ldx % 4 == 0);
    P.err = device_error_word();
    P.ctas_per_sm = c.compress_ctas;
    P.wait_cycles = wait_limit_cycles();
    P.mask_pt = (int)c.pt;
    return P;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool compress_batchable(const sk_ctx &c, const float *X, int64_t ldx) {
    return c.log2pt >= 2 && ((reinterpret_cast<uintptr_t>(X) & 15) == 0) && (c.p % 4 == 0) &&
           (ldx % 4 == 0);
}

cudaError_t compress_batch_build(const sk_ctx *ctxs, const BatchRows *rows, int nd,
                                 int units_per_group, std::vector<unsigned char> &table,
                                 CompressBatchInfo &info) {
    std::vector<CompressParams> Ps((size_t)nd);
    std::vector<CompressTask> tasks;
    int Lmax = 2;
    for (int d = 0; d < nd; ++d) {
        const sk_ctx &c = ctxs[d];
        Ps[d] = make_params(c, rows[d].X, rows[d].n, rows[d].ldx, rows[d].row0, rows[d].idx,
                            rows[d].val, nullptr);
        const int L = c.log2pt;
        if (L > Lmax) Lmax = L;
        const int64_t rpu = (L <= 10) ? (1024 >> L) : 1;
        const int64_t ng = kWarps / ((L > 10) ? (1 << (L - 10)) : 1);
        const int64_t nunits = (L <= 10) ? (rows[d].n + rpu - 1) / rpu : rows[d].n;
        const int64_t per = ng * (int64_t)units_per_group;
        for (int64_t u = 0; u < nunits; u += per) {
            CompressTask T;
            T.d = d;
            T.L = L;
            T.u_begin = u;
            T.u_end = (u + per < nunits) ? u + per : nunits;
            tasks.push_back(T);
        }
    }
    // largest tasks (pt) first: the tail of the launch is made of small ones
    std::stable_sort(tasks.begin(), tasks.end(),
                     [](const CompressTask &a, const CompressTask &b) { return a.L > b.L; });
    size_t smem = 0;
    for (int d = 0; d < nd; ++d) {
        const size_t b = compress_smem_for(ctxs[d].log2pt);
        if (b > smem) smem = b;
    }
    info.smem = smem;
    info.ntasks = (int)tasks.size();
    info.params_off = align256(table.size());
    info.tasks_off = align256(info.params_off + Ps.size() * sizeof(CompressParams));
    info.ticket_off = align256(info.tasks_off + tasks.size() * sizeof(CompressTask));
    table.resize(info.ticket_off + 256, 0);
    std::memcpy(table.data() + info.params_off, Ps.data(), Ps.size() * sizeof(CompressParams));
    if (!tasks.empty())
        std::memcpy(table.data() + info.tasks_off, tasks.data(), tasks.size() * sizeof(CompressTask));
    cudaError_t e = cudaFuncSetAttribute(compress_batch_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, compress_batch_kernel, kWarps * 32, smem);
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)sms * per_sm;
    if (grid > info.ntasks) grid = info.ntasks > 0 ? info.ntasks : 1;
    info.grid = (int)grid;
    (void)Lmax;
    return cudaSuccess;
}

cudaError_t compress_batch_launch(const CompressBatchInfo &info, unsigned char *dev_table,
                                  cudaStream_t s) {
    if (info.ntasks == 0) return cudaSuccess;
    unsigned int *ticket = reinterpret_cast<unsigned int *>(dev_table + info.ticket_off);
    cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    compress_batch_kernel<<<(unsigned)info.grid, kWarps * 32, info.smem, s>>>(
        reinterpret_cast<const CompressParams *>(dev_table + info.params_off),
        reinterpret_cast<const CompressTask *>(dev_table + info.tasks_off), info.ntasks, ticket);
    return cudaGetLastError();
}

// Masks alone (mask_kernel) for any range pt <= 2^L.
static cudaError_t launch_masks_any(int L, const CompressParams &P, cudaStream_t s) {
    switch (L) {
        case 0: return launch_masks<0>(P, s);
        case 1: return launch_masks<1>(P, s);
        case 2: return launch_masks<2>(P, s);
        case 3: return launch_masks<3>(P, s);
        case 4: return launch_masks<4>(P, s);
        case 5: return launch_masks<5>(P, s);
        case 6: return launch_masks<6>(P, s);
        case 7: return launch_masks<7>(P, s);
        case 8: return launch_masks<8>(P, s);
        case 9: return launch_masks<9>(P, s);
        case 10: return launch_masks<10>(P, s);
        case 11: return launch_masks<11>(P, s);
        case 12: return launch_masks<12>(P, s);
        case 13: return launch_masks<13>(P, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_compress(const sk_ctx &c, const float *X, int64_t n, int64_t ldx,
                            int64_t row0, int32_t *idx, float *val, float *Y,
                            cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const CompressParams P = make_params(c, X, n, ldx, row0, idx, val, Y);
    if (c.flags & SK_FLAG_DCT) {
        // the DCT preconditioner (no padding): masks over [0, p) first, then
        // each row's transform and its gather (or the dense rows)
        if (!Y) {
            const cudaError_t e = launch_masks_any(c.log2pt, P, s);
            if (e != cudaSuccess) return e;
        }
        return launch_dct_forward(c, X, n, ldx, idx, val, Y, s);
    }
    return Y ? dispatch<true>(c.log2pt, P, s) : dispatch<false>(c.log2pt, P, s);
}

}  // namespace sk
