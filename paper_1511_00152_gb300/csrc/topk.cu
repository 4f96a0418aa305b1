// topk.cu -- top-k principal subspace of the symmetric pt x pt estimate C_n
// (Sec. V: PCA recovers the leading eigenvectors of the covariance), in
// float64 on the device.
//
// Block subspace iteration with b = min(pt, 64, max(k + 8, 2k)) columns:
//   W = C V;  V = W R^{-1} with R the Cholesky factor of W^T W (CholQR),
// repeated `iters` times from a seeded start, then one Rayleigh-Ritz step:
// H = V^T C V (b x b), H = Q diag(lambda) Q^T by cyclic Jacobi rotations, and
// U = V Q restricted to the k largest lambda.  Each eigenvector's sign makes
// its largest-magnitude entry positive.  Everything is float64: the panel
// product is a tiled CUDA-core kernel, the small b x b factorisations run in
// one CTA.
#include <mutex>

#include "sk_internal.cuh"

namespace sk {
namespace {

constexpr int kMaxB = 64;
constexpr uint32_t kTagTopk = 0x544F504Bu;  // "TOPK"

int block_cols(int64_t pt, int k) {
    int b = 2 * k > k + 8 ? 2 * k : k + 8;
    if (b > kMaxB) b = kMaxB;
    if (b > pt) b = (int)pt;
    if (b < k) b = k;
    return b;
}

// Workspace layout (doubles): V[b*pt] W[b*pt] Gm[b*b] Rinv[b*b] H[b*b] Q[b*b] lam[b]
struct Ws {
    double *V, *W, *Gm, *Rinv, *H, *Q, *lam;
};
Ws carve(double *work, int64_t pt, int b) {
    Ws w;
    w.V = work;
    w.W = w.V + (int64_t)b * pt;
    w.Gm = w.W + (int64_t)b * pt;
    w.Rinv = w.Gm + b * b;
    w.H = w.Rinv + b * b;
    w.Q = w.H + b * b;
    w.lam = w.Q + b * b;
    return w;
}

__global__ void init_v_kernel(double *V, int64_t pt, int b, uint32_t k0, uint32_t k1) {
    const int64_t total = (int64_t)b * pt;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const uint4 o = philox4x32_10(make_uint4((uint32_t)e, (uint32_t)(e >> 32), 0u, kTagTopk),
                                      k0, k1);
        V[e] = ((double)o.x + 0.5) * (1.0 / 4294967296.0) - 0.5;
    }
}

// W[c*pt + i] += sum_{j in this CTA's range} C[i*pt + j] * V[c*pt + j] for c < b.
// CTA: 64 rows i (blockIdx.x) times one j-range (blockIdx.y); W must be zeroed
// before the launch and receives the partial sums with double atomics.
__global__ void __launch_bounds__(256) panel_kernel(const double *C, const double *V,
                                                    int64_t pt, int b, int64_t jlen, double *W) {
    __shared__ double Cs[64][33];
    __shared__ double Vs[kMaxB][33];
    const int tid = threadIdx.x;
    const int ri = tid & 63, cg = tid >> 6;  // 4 column groups
    const int64_t i0 = (int64_t)blockIdx.x * 64;
    const int64_t jb = (int64_t)blockIdx.y * jlen;
    int64_t je = jb + jlen;
    if (je > pt) je = pt;
    double acc[kMaxB / 4];
#pragma unroll
    for (int q = 0; q < kMaxB / 4; ++q) acc[q] = 0.0;
    for (int64_t j0 = jb; j0 < je; j0 += 32) {
        for (int e = tid; e < 64 * 32; e += 256) {
            const int r = e >> 5, cc = e & 31;
            const int64_t gi = i0 + r, gj = j0 + cc;
            Cs[r][cc] = (gi < pt && gj < je) ? C[gi * pt + gj] : 0.0;
        }
        for (int e = tid; e < b * 32; e += 256) {
            const int c = e >> 5, cc = e & 31;
            const int64_t gj = j0 + cc;
            Vs[c][cc] = (gj < je) ? V[(int64_t)c * pt + gj] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int cc = 0; cc < 32; ++cc) {
            const double cv = Cs[ri][cc];
#pragma unroll
            for (int q = 0; q < kMaxB / 4; ++q) {
                const int c = cg + 4 * q;
                if (c < b) acc[q] = fma(cv, Vs[c][cc], acc[q]);
            }
        }
        __syncthreads();
    }
    const int64_t gi = i0 + ri;
    if (gi < pt) {
#pragma unroll
        for (int q = 0; q < kMaxB / 4; ++q) {
            const int c = cg + 4 * q;
            if (c < b) atomicAdd(W + (int64_t)c * pt + gi, acc[q]);
        }
    }
}

// Gm[c1*b + c2] = A[c1]^T B[c2] over pt (one CTA per (c1, c2)).
__global__ void small_gram_kernel(const double *A, const double *B, int64_t pt, int b,
                                  double *Gm) {
    __shared__ double red[256];
    const int c1 = blockIdx.x / b, c2 = blockIdx.x % b;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < pt; i += blockDim.x)
        s = fma(A[(int64_t)c1 * pt + i], B[(int64_t)c2 * pt + i], s);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) Gm[blockIdx.x] = red[0];
}

// Cholesky Gm = R^T R (upper R) and Rinv = R^{-1}, one CTA, right-looking:
// per column c the pivot, the scaled row c, then the trailing update in
// parallel.  A pivot that is not safely positive (rank-deficient block) is
// replaced by a tiny positive value so the column is kept and re-normalised in
// later iterations.
__global__ void __launch_bounds__(256) chol_inv_kernel(const double *Gm, int b, double *Rinv) {
    __shared__ double A[kMaxB][kMaxB + 1];
    __shared__ double floor_v;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < b * b; e += nt) {
        A[e / b][e % b] = Gm[e];
        Rinv[e] = 0.0;
    }
    __syncthreads();
    if (tid == 0) {
        double tr = 0.0;
        for (int c = 0; c < b; ++c) tr += A[c][c];
        floor_v = 1e-300 + 1e-28 * tr;
    }
    __syncthreads();
    for (int c = 0; c < b; ++c) {
        if (tid == 0) {
            const double d = A[c][c];
            A[c][c] = sqrt(d > floor_v ? d : floor_v);
        }
        __syncthreads();
        const double inv = 1.0 / A[c][c];
        for (int j = c + 1 + tid; j < b; j += nt) A[c][j] *= inv;
        __syncthreads();
        const int rem = b - c - 1;
        for (int w = tid; w < rem * rem; w += nt) {
            const int i = c + 1 + w / rem, j = c + 1 + w % rem;
            if (j >= i) A[i][j] -= A[c][i] * A[c][j];
        }
        __syncthreads();
    }
    // inverse of upper-triangular R by back substitution, a thread per column
    // (each thread reads and writes only its own column of Rinv)
    for (int j = tid; j < b; j += nt) {
        for (int i = j; i >= 0; --i) {
            double sacc = (i == j) ? 1.0 : 0.0;
            for (int q = i + 1; q <= j; ++q) sacc -= A[i][q] * Rinv[q * b + j];
            Rinv[i * b + j] = sacc / A[i][i];
        }
    }
}

// V[c*pt + i] = sum_{q <= c} W[q*pt + i] * Rinv[q*b + c], a thread per (i, c).
__global__ void apply_rinv_kernel(const double *W, const double *Rinv, int64_t pt, int b,
                                  double *V) {
    __shared__ double Rs[kMaxB * kMaxB];
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) Rs[e] = Rinv[e];
    __syncthreads();
    const int64_t total = (int64_t)b * pt;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / pt);
        const int64_t i = e - (int64_t)c * pt;
        double sacc = 0.0;
        for (int q = 0; q <= c; ++q) sacc = fma(W[(int64_t)q * pt + i], Rs[q * b + c], sacc);
        V[e] = sacc;
    }
}

// Jacobi eigen-decomposition of the symmetric b x b H (one CTA):
// H = Q diag(lam) Q^T.  Parallel (round-robin) ordering: each step applies
// bp/2 disjoint plane rotations at once (bp = b rounded up to even, the extra
// index is a decoupled zero row/column), bp - 1 steps per sweep, sweeps until
// the off-diagonal mass is below 1e-30 of the total.
__global__ void __launch_bounds__(256) jacobi_kernel(const double *Hin, int b, double *Q,
                                                     double *lam) {
    __shared__ double A[kMaxB][kMaxB + 1];
    __shared__ double rc[kMaxB / 2], rs[kMaxB / 2];
    __shared__ int rp[kMaxB / 2], rq[kMaxB / 2];
    __shared__ int done;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int bp = (b + 1) & ~1;
    const int half = bp / 2;
    for (int e = tid; e < bp * bp; e += nt) {
        const int r = e / bp, c = e % bp;
        A[r][c] = (r < b && c < b) ? 0.5 * (Hin[r * b + c] + Hin[c * b + r]) : 0.0;
    }
    // Q (global, b x b) accumulates the rotations
    for (int e = tid; e < b * b; e += nt) Q[e] = (e / b == e % b) ? 1.0 : 0.0;
    __syncthreads();
    for (int sweep = 0; sweep < 60; ++sweep) {
        if (tid == 0) {
            double off = 0.0, tot = 0.0;
            for (int r = 0; r < bp; ++r)
                for (int c = 0; c < bp; ++c) {
                    const double x = A[r][c] * A[r][c];
                    tot += x;
                    if (r != c) off += x;
                }
            done = off <= 1e-30 * tot || tot == 0.0;
        }
        __syncthreads();
        if (done) break;
        for (int step = 0; step < bp - 1; ++step) {
            if (tid < half) {
                // circle method: index 0 fixed, 1..bp-1 rotate
                int p, q;
                if (tid == 0) {
                    p = 0;
                    q = 1 + step % (bp - 1);
                } else {
                    p = 1 + (step + tid) % (bp - 1);
                    q = 1 + (step - tid + (bp - 1)) % (bp - 1);
                }
                const double apq = A[p][q];
                double c = 1.0, sn = 0.0;
                if (apq != 0.0) {
                    const double theta = (A[q][q] - A[p][p]) / (2.0 * apq);
                    const double t = (theta >= 0 ? 1.0 : -1.0) /
                                     (fabs(theta) + sqrt(theta * theta + 1.0));
                    c = 1.0 / sqrt(t * t + 1.0);
                    sn = t * c;
                }
                rp[tid] = p;
                rq[tid] = q;
                rc[tid] = c;
                rs[tid] = sn;
            }
            __syncthreads();
            // columns: A <- A J, Q <- Q J (a pair with the padding index is
            // the identity: its 2x2 block is zero)
            for (int w = tid; w < half * bp; w += nt) {
                const int k = w / bp, r = w % bp;
                const int p = rp[k], q = rq[k];
                if (p >= b || q >= b) continue;
                const double c = rc[k], sn = rs[k];
                const double arp = A[r][p], arq = A[r][q];
                A[r][p] = c * arp - sn * arq;
                A[r][q] = sn * arp + c * arq;
                if (r < b) {
                    const double qrp = Q[r * b + p], qrq = Q[r * b + q];
                    Q[r * b + p] = c * qrp - sn * qrq;
                    Q[r * b + q] = sn * qrp + c * qrq;
                }
            }
            __syncthreads();
            // rows: A <- J^T A
            for (int w = tid; w < half * bp; w += nt) {
                const int k = w / bp, r = w % bp;
                const int p = rp[k], q = rq[k];
                if (p >= b || q >= b) continue;
                const double c = rc[k], sn = rs[k];
                const double apr = A[p][r], aqr = A[q][r];
                A[p][r] = c * apr - sn * aqr;
                A[q][r] = sn * apr + c * aqr;
            }
            __syncthreads();
        }
    }
    for (int r = tid; r < b; r += nt) lam[r] = A[r][r];
}

// U[c*pt + i] = sum_q V[q*pt + i] Q[q*b + order[c]] for the k largest lambda,
// then the sign convention.  One CTA per output column c.
__global__ void ritz_out_kernel(const double *V, const double *Q, const double *lam,
                                int64_t pt, int b, int k, double *U, double *evals) {
    __shared__ int order_c;
    __shared__ double red_v[256];
    __shared__ int64_t red_i[256];
    const int c = blockIdx.x;
    if (threadIdx.x == 0) {
        // c-th largest eigenvalue (ties by lower index)
        bool used[kMaxB];
        for (int q = 0; q < b; ++q) used[q] = false;
        int pick = 0;
        for (int r = 0; r <= c; ++r) {
            pick = -1;
            for (int q = 0; q < b; ++q)
                if (!used[q] && (pick < 0 || lam[q] > lam[pick])) pick = q;
            used[pick] = true;
        }
        order_c = pick;
        evals[c] = lam[pick];
    }
    __syncthreads();
    const int col = order_c;
    double best = -1.0;
    int64_t besti = 0;
    for (int64_t i = threadIdx.x; i < pt; i += blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < b; ++q) s = fma(V[(int64_t)q * pt + i], Q[q * b + col], s);
        U[(int64_t)c * pt + i] = s;
        if (fabs(s) > best) {
            best = fabs(s);
            besti = i;
        }
    }
    red_v[threadIdx.x] = best;
    red_i[threadIdx.x] = besti;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            const double ov = red_v[threadIdx.x + h];
            const int64_t oi = red_i[threadIdx.x + h];
            if (ov > red_v[threadIdx.x] || (ov == red_v[threadIdx.x] && oi < red_i[threadIdx.x])) {
                red_v[threadIdx.x] = ov;
                red_i[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    const bool flip = U[(int64_t)c * pt + red_i[0]] < 0.0;
    __syncthreads();
    if (flip)
        for (int64_t i = threadIdx.x; i < pt; i += blockDim.x) U[(int64_t)c * pt + i] *= -1.0;
}

}  // namespace

// ---- fixed scratch for callers that cannot allocate device memory
//
// One array per device that loads the library, held until the process exits.
// Host code must not pass g_topk_scratch itself to a kernel (on the host the
// name is only a stand-in for the device symbol); its device address is looked
// up once per device with cudaGetSymbolAddress, with that device current.
namespace {
constexpr int64_t kTopkStaticDoubles = 512 * 1024;  // 4 MiB
static __device__ __align__(256) double g_topk_scratch[kTopkStaticDoubles];
std::mutex g_topk_scratch_mu;
double *g_topk_scratch_ptr[128] = {};
}  // namespace

int64_t topk_static_capacity() { return kTopkStaticDoubles; }

cudaError_t topk_static_scratch(double **out) {
    *out = nullptr;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_topk_scratch_mu);
    if (!g_topk_scratch_ptr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_topk_scratch);
        if (e != cudaSuccess) return e;
        g_topk_scratch_ptr[dev] = static_cast<double *>(ptr);
    }
    *out = g_topk_scratch_ptr[dev];
    return cudaSuccess;
}

int64_t topk_workspace(int64_t pt, int k) {
    const int b = block_cols(pt, k);
    return 2 * (int64_t)b * pt + 4 * (int64_t)b * b + b;
}

cudaError_t launch_topk(const sk_ctx &c, const double *C, int k, int iters, double *evals,
                        double *U, double *work, cudaStream_t s) {
    const int64_t pt = c.pt;
    const int b = block_cols(pt, k);
    Ws w = carve(work, pt, b);
    const uint32_t k0 = (uint32_t)c.seed, k1 = (uint32_t)(c.seed >> 32);
    const int pblocks = (int)((pt + 63) / 64);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t jsplit = (2LL * sms + pblocks - 1) / pblocks;
    if (jsplit > (pt + 31) / 32) jsplit = (pt + 31) / 32;
    if (jsplit < 1) jsplit = 1;
    int64_t jlen = (pt + jsplit - 1) / jsplit;
    jlen = (jlen + 31) / 32 * 32;
    jsplit = (pt + jlen - 1) / jlen;
    const dim3 pgrid((unsigned)pblocks, (unsigned)jsplit);
    int eblocks = (int)((b * pt + 255) / 256);
    if (eblocks > 4096) eblocks = 4096;
    int ablocks = (int)((b * pt + 255) / 256);
    if (ablocks > 4096) ablocks = 4096;
    init_v_kernel<<<eblocks, 256, 0, s>>>(w.V, pt, b, k0, k1);
    for (int it = 0; it <= iters; ++it) {
        cudaMemsetAsync(w.W, 0, (size_t)b * pt * sizeof(double), s);
        panel_kernel<<<pgrid, 256, 0, s>>>(C, w.V, pt, b, jlen, w.W);
        if (it == iters) break;
        small_gram_kernel<<<b * b, 256, 0, s>>>(w.W, w.W, pt, b, w.Gm);
        chol_inv_kernel<<<1, 256, 0, s>>>(w.Gm, b, w.Rinv);
        apply_rinv_kernel<<<ablocks, 256, 0, s>>>(w.W, w.Rinv, pt, b, w.V);
    }
    // Rayleigh-Ritz: H = V^T (C V)
    small_gram_kernel<<<b * b, 256, 0, s>>>(w.V, w.W, pt, b, w.H);
    jacobi_kernel<<<1, 256, 0, s>>>(w.H, b, w.Q, w.lam);
    ritz_out_kernel<<<k, 256, 0, s>>>(w.V, w.Q, w.lam, pt, b, k, U, evals);
    return cudaGetLastError();
}

}  // namespace sk
