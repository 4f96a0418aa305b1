// gram_fp32.cu -- the plain FP32 form of the covariance accumulation (Sec. V)
// and the covariance finalize.
//
// G += sum_i w_i w_i^T as a scatter of the m^2 products of each ELL row.  The
// pt x pt output is cut into T x T tiles (T = 128, or pt if smaller); a CTA
// owns one upper tile (bi <= bj) for a slice of the rows and accumulates it in
// shared memory with float atomics.  Per row, a warp compacts the row's
// entries that fall in the tile's row block I and column block J (ballot +
// popc), then spreads the |I| x |J| products over its lanes.  The tile is
// flushed to the caller's float64 G with one double atomic per entry.
//
// cov_finalize applies the rescaling and the diagonal correction of C_n
// (Sec. V): off-diagonal P(P-1)/(m(m-1)) G/n, diagonal times (1 - (P-m)/(P-1)).
// The centred form (C_n - xbar xbar^T + B(C_n)/n, with xbar the sample-mean
// estimate of Sec. IV) scales each C_n entry once more, by 1 + (P-m)/(m n) on
// the diagonal and 1 - (P-m)/(m (P-1) n) off it, and subtracts xbar_j xbar_k.
#include "sk_internal.cuh"

namespace sk {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = 512;
constexpr int kWarpsG = kThreads / 32;

struct GramParams {
    const int32_t *idx;
    const float *val;
    int64_t n;
    int m;
    int pt;
    int T, logT, nb;
    int cap;  // list capacity: entries of one row inside one block <= min(m, T)
    int64_t rows_per_split;
    double *G;
};

__global__ void __launch_bounds__(kThreads) gram_fp32_kernel(GramParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int T = P.T;
    float *tile = reinterpret_cast<float *>(smem_raw);
    // per-warp compaction lists: (local coord, value) for I then J, capacity m each
    int *lists = reinterpret_cast<int *>(smem_raw + (size_t)T * T * 4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *aI = lists + warp * 4 * P.cap;
    float *vI = reinterpret_cast<float *>(aI + P.cap);
    int *aJ = aI + 2 * P.cap;
    float *vJ = reinterpret_cast<float *>(aI + 3 * P.cap);

    // decode the upper tile (bi <= bj) and the row split of this CTA
    int t = blockIdx.x;
    int bi = 0;
    while (t >= P.nb - bi) {
        t -= P.nb - bi;
        ++bi;
    }
    const int bj = bi + t;
    const int64_t r_begin = (int64_t)blockIdx.y * P.rows_per_split;
    int64_t r_end = r_begin + P.rows_per_split;
    if (r_end > P.n) r_end = P.n;

    for (int e = threadIdx.x; e < T * T; e += blockDim.x) tile[e] = 0.f;
    __syncthreads();

    const unsigned lt = lanemask_lt();
    const int m = P.m;
    for (int64_t i = r_begin + warp; i < r_end; i += kWarpsG) {
        const int32_t *ri = P.idx + i * m;
        const float *rv = P.val + i * m;
        int nI = 0, nJ = 0;
        for (int c0 = 0; c0 < m; c0 += 32) {
            const int tt = c0 + lane;
            int j = -1;
            float v = 0.f;
            if (tt < m) {
                j = __ldg(ri + tt);
                v = __ldg(rv + tt);
            }
            const int blk = j >> P.logT;
            const bool inI = tt < m && blk == bi;
            const bool inJ = tt < m && blk == bj;
            const unsigned bI = __ballot_sync(kFull, inI);
            const unsigned bJ = __ballot_sync(kFull, inJ);
            // a row of sk_compress has distinct indices, so at most cap entries
            // fall in one block; anything beyond (malformed input) is dropped
            if (inI) {
                const int pos = nI + __popc(bI & lt);
                if (pos < P.cap) {
                    aI[pos] = j & (T - 1);
                    vI[pos] = v;
                }
            }
            if (inJ) {
                const int pos = nJ + __popc(bJ & lt);
                if (pos < P.cap) {
                    aJ[pos] = j & (T - 1);
                    vJ[pos] = v;
                }
            }
            nI += __popc(bI);
            nJ += __popc(bJ);
        }
        if (nI > P.cap) nI = P.cap;
        if (nJ > P.cap) nJ = P.cap;
        __syncwarp();
        const int npairs = nI * nJ;
        for (int q = lane; q < npairs; q += 32) {
            const int s = q / nJ;
            const int u = q - s * nJ;
            atomicAdd(tile + aI[s] * T + aJ[u], vI[s] * vJ[u]);
        }
        __syncwarp();
    }
    __syncthreads();
    for (int e = threadIdx.x; e < T * T; e += blockDim.x) {
        const float x = tile[e];
        const int a = e / T, b = e - a * T;
        // the last block of a pt that is not a multiple of T is ragged
        if (x != 0.f && bi * T + a < P.pt && bj * T + b < P.pt) {
            atomicAdd(P.G + (int64_t)(bi * T + a) * P.pt + (bj * T + b), (double)x);
        }
    }
}

__global__ void cov_finalize_kernel(const double *G, int pt, double scale_off,
                                    double scale_diag, double cen_off, double cen_diag,
                                    const double *mean, double *C) {
    const int64_t total = (int64_t)pt * pt;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / pt), k = (int)(e - (int64_t)j * pt);
        const int a = j < k ? j : k, b = j < k ? k : j;
        const double g = G[(int64_t)a * pt + b];
        const double cn = (j == k) ? g * scale_diag : g * scale_off;
        C[e] = mean ? cn * ((j == k) ? cen_diag : cen_off) - mean[j] * mean[k] : cn;
    }
}

}  // namespace

cudaError_t launch_gram_fp32(const sk_ctx &c, const int32_t *idx, const float *val,
                             int64_t n, double *G, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    GramParams P;
    P.idx = idx;
    P.val = val;
    P.n = n;
    P.m = (int)c.m;
    P.pt = (int)c.pt;
    // tiles of T x T with T a power of two (the smallest >= pt below 128);
    // the last block is ragged when pt is not a multiple of T
    P.T = 128;
    while (P.T > 1 && P.T / 2 >= c.pt) P.T /= 2;
    P.logT = 0;
    while ((1 << P.logT) < P.T) ++P.logT;
    P.nb = (int)((c.pt + P.T - 1) / P.T);
    P.cap = P.m < P.T ? P.m : P.T;
    P.G = G;
    const int ntiles = P.nb * (P.nb + 1) / 2;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // enough row splits to give every SM a few CTAs, but >= 4 warps' rows each
    int64_t splits = (4LL * sms + ntiles - 1) / ntiles;
    const int64_t max_splits = (n + 4 * kWarpsG - 1) / (4 * kWarpsG);
    if (splits > max_splits) splits = max_splits;
    if (splits < 1) splits = 1;
    if (splits > 65535) splits = 65535;
    P.rows_per_split = (n + splits - 1) / splits;
    const size_t smem = (size_t)P.T * P.T * 4 + (size_t)kWarpsG * 4 * P.cap * 4;
    cudaError_t e = cudaFuncSetAttribute(gram_fp32_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)ntiles, (unsigned)splits);
    gram_fp32_kernel<<<grid, kThreads, smem, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_cov_finalize(const sk_ctx &c, const double *G, int64_t n_total,
                                const double *mean, double *C, cudaStream_t s) {
    const double P = (double)c.pt, M = (double)c.m, N = (double)n_total;
    const double off = P * (P - 1.0) / (M * (M - 1.0)) / N;
    const double diag = off * (1.0 - (P - M) / (P - 1.0));
    const double cen_diag = 1.0 + (P - M) / M / N;
    const double cen_off = 1.0 - (P - M) / (M * (P - 1.0)) / N;
    const int64_t total = c.pt * c.pt;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 8192) blocks = 8192;
    cov_finalize_kernel<<<blocks, 256, 0, s>>>(G, (int)c.pt, off, diag, cen_off, cen_diag, mean,
                                               C);
    return cudaGetLastError();
}

}  // namespace sk
