// kmeanspp.cu -- K-means++ seeding on the sparsified rows (Algorithm 1, "find
// initial cluster centers via K-means++"; D. Arthur and S. Vassilvitskii,
// "k-means++: the advantages of careful seeding", SODA 2007), and the
// objective J' of a finished run (Sec. VI-A) for choosing the best restart.
//
// The centres are rows of the data: centre k is the pt-vector of the chosen
// row's ELL entries (zero elsewhere), and D2_i is row i's restricted squared
// distance to its nearest chosen centre.  The choice of a row is an integer
// decision, taken exactly as the library's written spec (include/sk.h):
// D2 in float32 (t ascending), integer weights q_i = floor(D2_i 2^(B - e)),
// exact uint64 prefix sums, and a 64-bit Lemire draw from the KMPP Philox
// stream of (seed, step, restart).  One step is four launches:
//   pick   -- one CTA: the draw, then the block and the row it falls in;
//   centre -- one CTA: the chosen row's scatter (zero, then t ascending);
//   dist   -- D2 = min(D2, distance to the new centre) for every row, rows
//             staged through shared memory in t-chunks, and the global max
//             (as float bits, which order like the non-negative floats);
//   sums   -- per 256-row block, the sum of the integer weights.
#include "sk_internal.cuh"

namespace sk {
namespace {

constexpr uint32_t kTagKmpp = 0x4B4D5050u;  // "KMPP"
constexpr int kRows = 256;                   // rows per block (one thread each)
constexpr int kChunk = 32;                   // staged entries per row per round
constexpr int kPickThreads = 1024;

// Workspace carve (bytes): D2 n floats | block sums nblk uint64 | gmax bits,
// chosen row (int64), B and e.
struct KppWs {
    float *D2;
    unsigned long long *bsum;
    unsigned int *gmax;
    long long *chosen;
};
__host__ __device__ int64_t nblocks(int64_t n) { return (n + kRows - 1) / kRows; }
KppWs carve_kpp(void *work, int64_t n) {
    unsigned char *w = static_cast<unsigned char *>(work);
    KppWs s;
    s.D2 = reinterpret_cast<float *>(w);
    size_t off = ((size_t)n * 4 + 255) & ~(size_t)255;
    s.bsum = reinterpret_cast<unsigned long long *>(w + off);
    off += ((size_t)nblocks(n) * 8 + 255) & ~(size_t)255;
    s.gmax = reinterpret_cast<unsigned int *>(w + off);
    s.chosen = reinterpret_cast<long long *>(w + off + 8);
    return s;
}

// Draw of step k, restart r, uniform over [0, W) (W >= 1): 64-bit Lemire
// multiply-shift with rejection (each attempt is rejected with probability
// below 1/2; after 64 rejections, probability < 2^-64, 0 is returned).
__device__ unsigned long long kpp_draw(uint32_t k0, uint32_t k1, uint32_t k, uint32_t r,
                                       unsigned long long W) {
    const unsigned long long threshold = (0ull - W) % W;
    for (uint32_t a = 0; a < 64; ++a) {
        const uint4 o = philox4x32_10(make_uint4(k, r, a / 2, kTagKmpp), k0, k1);
        const unsigned long long x = (a & 1) ? (((unsigned long long)o.w << 32) | o.z)
                                             : (((unsigned long long)o.y << 32) | o.x);
        if (x * W < threshold) continue;
        return __umul64hi(x, W);
    }
    return 0ull;
}

// Integer weight of a squared distance: floor(d 2^(B - e)) (exact: a float
// times a power of two, truncated).
__device__ __forceinline__ unsigned long long kpp_weight(float d, int shift) {
    return (unsigned long long)((double)d * pow2(shift));
}

// Binary exponent e of a positive float x = f 2^e, 0.5 <= f < 1.
__device__ __forceinline__ int frexp_exponent(float x) {
    const long long bits = __double_as_longlong((double)x);
    return (int)((bits >> 52) & 0x7ff) - 1022;
}

__global__ void __launch_bounds__(kPickThreads) kpp_pick_kernel(KppWs ws, int64_t n, int k,
                                                               uint32_t restart, uint32_t k0,
                                                               uint32_t k1, int B,
                                                               long long *rows_out) {
    __shared__ unsigned long long part[kPickThreads];
    __shared__ unsigned long long s_u, s_before;
    __shared__ long long s_block;
    __shared__ int s_count;
    const int tid = threadIdx.x;
    const int64_t nb = nblocks(n);
    long long chosen = 0;
    bool fallback = (k == 0);
    unsigned long long W = 0;
    if (!fallback) {
        // W = sum of the block sums; each thread a contiguous segment
        const int64_t seg = (nb + kPickThreads - 1) / kPickThreads;
        const int64_t b0 = (int64_t)tid * seg;
        unsigned long long mine = 0;
        for (int64_t b = b0; b < b0 + seg && b < nb; ++b) mine += ws.bsum[b];
        part[tid] = mine;
        __syncthreads();
        // inclusive scan of the segment sums (Hillis-Steele)
        for (int off = 1; off < kPickThreads; off <<= 1) {
            const unsigned long long add = tid >= off ? part[tid - off] : 0ull;
            __syncthreads();
            part[tid] += add;
            __syncthreads();
        }
        W = part[kPickThreads - 1];
        fallback = (W == 0ull);
        if (!fallback) {
            if (tid == 0) s_u = kpp_draw(k0, k1, (uint32_t)k, restart, W);
            __syncthreads();
            const unsigned long long u = s_u;
            const unsigned long long before_seg = tid ? part[tid - 1] : 0ull;
            // the segment holding u: before_seg <= u < part[tid]
            if (before_seg <= u && u < part[tid]) {
                unsigned long long acc = before_seg;
                for (int64_t b = b0; b < b0 + seg && b < nb; ++b) {
                    if (u < acc + ws.bsum[b]) {
                        s_block = b;
                        s_before = acc;
                        break;
                    }
                    acc += ws.bsum[b];
                }
            }
            if (tid == 0) s_count = 0;
            __syncthreads();
            // within the block: the first row whose inclusive prefix exceeds u
            const long long blk = s_block;
            const int shift = B - frexp_exponent(__uint_as_float(*ws.gmax));
            const int64_t i = blk * kRows + tid;
            unsigned long long q = 0;
            if (tid < kRows && i < n) q = kpp_weight(ws.D2[i], shift);
            part[tid] = q;
            __syncthreads();
            for (int off = 1; off < kRows; off <<= 1) {
                const unsigned long long add = (tid < kRows && tid >= off) ? part[tid - off] : 0ull;
                __syncthreads();
                if (tid < kRows) part[tid] += add;
                __syncthreads();
            }
            if (tid < kRows && i < n && s_before + part[tid] <= u) atomicAdd(&s_count, 1);
            __syncthreads();
            chosen = blk * kRows + s_count;
        }
    }
    if (fallback && tid == 0) chosen = (long long)kpp_draw(k0, k1, (uint32_t)k, restart, (unsigned long long)n);
    if (tid == 0) {
        rows_out[k] = chosen;
        *ws.chosen = chosen;
        *ws.gmax = 0u;  // reset for the coming distance pass
    }
}

// Centre k: zero, then the chosen row's entries t ascending (a repeated
// index keeps its last value).
__global__ void kpp_centre_kernel(KppWs ws, const int32_t *idx, const float *val, int m, int pt,
                                  float *cen) {
    const long long c = *ws.chosen;
    for (int j = threadIdx.x; j < pt; j += blockDim.x) cen[j] = 0.f;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int t = 0; t < m; ++t) cen[clamp_index(idx[c * m + t], pt)] = val[c * m + t];
}

__global__ void __launch_bounds__(kRows) kpp_dist_kernel(KppWs ws, const int32_t *idx,
                                                        const float *val, int64_t n, int m,
                                                        int pt, const float *cen, int first) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *cs = reinterpret_cast<float *>(smem_raw);          // pt
    int2 *st = reinterpret_cast<int2 *>(smem_raw + (size_t)pt * 4);  // kRows x (kChunk + 1)
    __shared__ float red[kRows / 32];
    const int tid = threadIdx.x;
    for (int j = tid; j < pt; j += kRows) cs[j] = cen[j];
    const int64_t r0 = (int64_t)blockIdx.x * kRows;
    const int rows = (int)((n - r0) < kRows ? (n - r0) : kRows);
    float d = 0.f;
    for (int t0 = 0; t0 < m; t0 += kChunk) {
        const int cw = (m - t0) < kChunk ? (m - t0) : kChunk;
        __syncthreads();
        // stage entries [t0, t0 + cw) of the block's rows (rows are contiguous)
        for (int e = tid; e < rows * cw; e += kRows) {
            const int r = e / cw, t = e - r * cw;
            const int64_t g = (r0 + r) * m + t0 + t;
            st[r * (kChunk + 1) + t] = make_int2(__ldg(idx + g), __float_as_int(__ldg(val + g)));
        }
        __syncthreads();
        if (tid < rows) {
            for (int t = 0; t < cw; ++t) {
                const int2 e = st[tid * (kChunk + 1) + t];
                const float diff = __int_as_float(e.y) - cs[clamp_index(e.x, pt)];
                d = fmaf(diff, diff, d);
            }
        }
    }
    float dn = 0.f;
    if (tid < rows) {
        const int64_t i = r0 + tid;
        dn = first ? d : fminf(ws.D2[i], d);
        ws.D2[i] = dn;
    }
    // block max, then the global max as float bits
    for (int o = 16; o > 0; o >>= 1) dn = fmaxf(dn, __shfl_xor_sync(0xffffffffu, dn, o));
    if ((tid & 31) == 0) red[tid >> 5] = dn;
    __syncthreads();
    if (tid == 0) {
        float mx = red[0];
        for (int w = 1; w < kRows / 32; ++w) mx = fmaxf(mx, red[w]);
        atomicMax(ws.gmax, __float_as_uint(mx));
    }
}

__global__ void __launch_bounds__(kRows) kpp_sums_kernel(KppWs ws, int64_t n, int B) {
    __shared__ unsigned long long red[kRows / 32];
    const float mx = __uint_as_float(*ws.gmax);
    const int tid = threadIdx.x;
    const int64_t i = (int64_t)blockIdx.x * kRows + tid;
    unsigned long long q = 0;
    if (mx > 0.f && i < n) q = kpp_weight(ws.D2[i], B - frexp_exponent(mx));
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    if ((tid & 31) == 0) red[tid >> 5] = q;
    __syncthreads();
    if (tid == 0) {
        unsigned long long s = 0;
        for (int w = 0; w < kRows / 32; ++w) s += red[w];
        ws.bsum[blockIdx.x] = s;
    }
}

// J' = sum of the winning restricted distances (float64 sum of float32 terms).
__global__ void objective_kernel(const float *dist, int64_t n, double *J) {
    __shared__ double red[256];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        s += (double)dist[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(J, red[0]);
}

}  // namespace

int64_t kmeanspp_workspace(int64_t n) {
    return (int64_t)((((size_t)n * 4 + 255) & ~(size_t)255) +
                     (((size_t)nblocks(n) * 8 + 255) & ~(size_t)255) + 256);
}

cudaError_t launch_kmeanspp(const sk_ctx &c, const int32_t *idx, const float *val, int64_t n,
                            int K, uint32_t restart, float *mu, int64_t *rows, void *work,
                            cudaStream_t s) {
    const KppWs ws = carve_kpp(work, n);
    int B = 62;
    while ((1ull << (62 - B)) < (unsigned long long)(n + 1)) --B;  // 62 - ceil(log2(n + 1))
    const uint32_t k0 = (uint32_t)c.seed, k1 = (uint32_t)(c.seed >> 32);
    const int pt = (int)c.pt, m = (int)c.m;
    const int64_t nb = nblocks(n);
    const size_t dsm = (size_t)pt * 4 + (size_t)kRows * (kChunk + 1) * 8;
    cudaError_t e = cudaFuncSetAttribute(kpp_dist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)dsm);
    if (e != cudaSuccess) return e;
    for (int k = 0; k < K; ++k) {
        kpp_pick_kernel<<<1, kPickThreads, 0, s>>>(ws, n, k, restart, k0, k1, B,
                                                   reinterpret_cast<long long *>(rows));
        float *cen = mu + (int64_t)k * pt;
        kpp_centre_kernel<<<1, 256, 0, s>>>(ws, idx, val, m, pt, cen);
        if (k + 1 == K) break;
        kpp_dist_kernel<<<(unsigned)nb, kRows, dsm, s>>>(ws, idx, val, n, m, pt, cen, k == 0);
        kpp_sums_kernel<<<(unsigned)nb, kRows, 0, s>>>(ws, n, B);
    }
    return cudaGetLastError();
}

cudaError_t launch_objective(const float *dist, int64_t n, double *J, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(J, 0, sizeof(double), s);
    if (e != cudaSuccess) return e;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    if (blocks < 1) blocks = 1;
    objective_kernel<<<(unsigned)blocks, 256, 0, s>>>(dist, n, J);
    return cudaGetLastError();
}

}  // namespace sk
