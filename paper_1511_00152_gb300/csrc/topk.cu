// topk.cu -- top-k principal subspace of the symmetric pt x pt estimate C_n
// (Sec. V: PCA recovers the leading eigenvectors of the covariance), in
// float64 on the device.
//
// Block subspace iteration with b = min(pt, 64, max(k + 8, 2k)) columns:
//   W = C V;  V = W R^{-1} with R the Cholesky factor of W^T W (CholQR),
// repeated `iters` times (at least once) from a seeded start, the last
// CholQR in float64 and the earlier ones from a float32 factor (see
// chol32_kernel), then one Rayleigh-Ritz step:
// H = V^T C V (b x b), H = Q diag(lambda) Q^T, and U = V Q restricted to the
// k largest lambda.  Each eigenvector's sign makes its largest-magnitude
// entry positive.
//
// Float64 throughput is a small fraction of float32's on this GPU, so the
// kernels are shaped by it: the panel product W = C V spreads its b pt^2
// fused multiply-adds over every SM with all b accumulators of a thread in
// registers; the serial steps of the small factorisations take reciprocals
// and square roots from Newton-Raphson iterations seeded by float32 hardware
// estimates instead of float64 division and square root; and the b x b
// eigenproblem is solved by Jacobi in float32 first, then re-orthonormalised
// and polished by a few float64 Jacobi sweeps (whose rotation angles are
// again float32 estimates; each rotation itself is orthogonal to float64
// rounding, so only the convergence rate of the last sweeps changes).
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

// Workspace layout (doubles): V[b*pt] W[b*pt] Gm[b*b] R[b*b] H[b*b] Q[b*b] lam[b]
// (lam holds the reciprocal Cholesky diagonal during the iterations).
struct Ws {
    double *V, *W, *Gm, *R, *H, *Q, *lam;
};
Ws carve(double *work, int64_t pt, int b) {
    Ws w;
    w.V = work;
    w.W = w.V + (int64_t)b * pt;
    w.Gm = w.W + (int64_t)b * pt;
    w.R = w.Gm + b * b;
    w.H = w.R + b * b;
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

// W[c*pt + i] += sum_{j in this CTA's range} C[j*pt + i] V[c*pt + j], c < b
// (C symmetric: row j read coalesced over i).  CTA = 128 columns i x one
// j-range; a thread owns column i and its BC >= b accumulators; V's slice of
// the j-range is staged in shared memory and read as a broadcast.  W is
// zeroed before the launch and receives the partial sums with double atomics.
constexpr int kPanelThreads = 128;
constexpr int kPanelJ = 32;

template <int BC>
__global__ void __launch_bounds__(kPanelThreads) panel_kernel(const double *C, const double *V,
                                                             int64_t pt, int b, int64_t jlen,
                                                             double *W) {
    __shared__ __align__(16) double Vs[kPanelJ][BC];
    const int tid = threadIdx.x;
    const int64_t i = (int64_t)blockIdx.x * kPanelThreads + tid;
    const int64_t jb = (int64_t)blockIdx.y * jlen;
    const int64_t je = (jb + jlen < pt) ? jb + jlen : pt;
    double acc[BC];
#pragma unroll
    for (int c = 0; c < BC; ++c) acc[c] = 0.0;
    for (int64_t j0 = jb; j0 < je; j0 += kPanelJ) {
        const int jn = (int)((je - j0) < kPanelJ ? (je - j0) : kPanelJ);
        for (int e = tid; e < kPanelJ * BC; e += kPanelThreads) {
            const int jj = e / BC, c = e - jj * BC;
            Vs[jj][c] = (jj < jn && c < b) ? V[(int64_t)c * pt + j0 + jj] : 0.0;
        }
        __syncthreads();
        if (i < pt) {
            for (int jj = 0; jj < jn; ++jj) {
                const double cv = C[(j0 + jj) * pt + i];
#pragma unroll
                for (int c = 0; c < BC; ++c) acc[c] = fma(cv, Vs[jj][c], acc[c]);
            }
        }
        __syncthreads();
    }
    if (i < pt) {
#pragma unroll
        for (int c = 0; c < BC; ++c)
            if (c < b) atomicAdd(W + (int64_t)c * pt + i, acc[c]);
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

// In-place upper Cholesky G = R^T R of the SPD b x b matrix in shared memory
// (right-looking, one CTA), with invd[c] = 1 / R[c][c].  A pivot that is not
// safely positive (rank-deficient block) is replaced by a tiny positive value
// so the column is kept and re-normalised in later iterations.
template <int LD>
__device__ void chol_dev(double (*A)[LD], int b, double *invd, double *floor_v) {
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) {
        double tr = 0.0;
        for (int c = 0; c < b; ++c) tr += A[c][c];
        *floor_v = 1e-300 + 1e-28 * (tr > 0.0 ? tr : 0.0);
    }
    __syncthreads();
    for (int c = 0; c < b; ++c) {
        if (tid == 0) {
            double d = A[c][c];
            d = d > *floor_v ? d : *floor_v;
            const double inv = rsqrt_nr(d);
            A[c][c] = d * inv;  // sqrt(d)
            invd[c] = inv;
        }
        __syncthreads();
        const double inv = invd[c];
        for (int j = c + 1 + tid; j < b; j += nt) A[c][j] *= inv;
        __syncthreads();
        const int rem = b - c - 1;
        for (int w = tid; w < rem * rem; w += nt) {
            const int i = c + 1 + w / rem, j = c + 1 + w % rem;
            if (j >= i) A[i][j] -= A[c][i] * A[c][j];
        }
        __syncthreads();
    }
}

// CholQR factor of the iteration: R (upper, b x b) and 1/diag(R) of Gm.
__global__ void __launch_bounds__(256) chol_kernel(const double *Gm, int b, double *R,
                                                   double *invd_out) {
    __shared__ double A[kMaxB][kMaxB + 1];
    __shared__ double invd[kMaxB];
    __shared__ double floor_v;
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) A[e / b][e % b] = Gm[e];
    __syncthreads();
    chol_dev<kMaxB + 1>(A, b, invd, &floor_v);
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
        const int r = e / b, c = e % b;
        R[e] = (c >= r) ? A[r][c] : 0.0;
    }
    for (int c = threadIdx.x; c < b; c += blockDim.x) invd_out[c] = invd[c];
}

// V = W R^{-1}: for each coordinate i, forward substitution over the columns,
// V[c][i] = (W[c][i] - sum_{q<c} V[q][i] R[q][c]) / R[c][c].  Small CTAs so
// the float64 work spreads over many SMs; the solved row lives in shared
// memory (dynamic: b*b + b + 32*b doubles).
constexpr int kApplyThreads = 32;

__global__ void __launch_bounds__(kApplyThreads) apply_solve_kernel(const double *W,
                                                                   const double *R,
                                                                   const double *invd, int64_t pt,
                                                                   int b, double *V) {
    extern __shared__ __align__(16) double sm[];
    double *Rs = sm;
    double *id = Rs + b * b;
    double *xs = id + b;  // [b][kApplyThreads]
    const int tid = threadIdx.x;
    for (int e = tid; e < b * b; e += kApplyThreads) Rs[e] = R[e];
    for (int e = tid; e < b; e += kApplyThreads) id[e] = invd[e];
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * kApplyThreads + tid;
    if (i >= pt) return;
    for (int c = 0; c < b; ++c) {
        double s = W[(int64_t)c * pt + i];
        for (int q = 0; q < c; ++q) s = fma(-xs[q * kApplyThreads + tid], Rs[q * b + c], s);
        s *= id[c];
        xs[c * kApplyThreads + tid] = s;
        V[(int64_t)c * pt + i] = s;
    }
}

// Intermediate CholQR in float32.  In the iterations before the last, V
// only has to be a well-conditioned basis of span(W): V = W M for any
// invertible M keeps the span exactly (the combination is formed in
// float64).  So M = R^{-1} is taken from a float32 Cholesky of the
// diagonally scaled Gram S = D Gm D (D = diag(Gm)^{-1/2}, unit diagonal, so
// float32 range is never an issue), M = D R_S^{-1}; V is then orthonormal
// to float32 accuracy, and the last iteration re-orthonormalises in float64.
__global__ void __launch_bounds__(256) chol32_kernel(const double *Gm, int b, double *Minv) {
    __shared__ float A[kMaxB][kMaxB + 1];
    __shared__ float X[kMaxB][kMaxB + 1];
    __shared__ double d[kMaxB];
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int c = tid; c < b; c += nt) {
        const double g = Gm[c * b + c];
        d[c] = g > 1e-300 ? rsqrt_nr(g) : 1.0;
    }
    __syncthreads();
    for (int e = tid; e < b * b; e += nt) {
        const int r = e / b, c = e % b;
        A[r][c] = (float)(Gm[e] * d[r] * d[c]);
    }
    __syncthreads();
    for (int c = 0; c < b; ++c) {
        if (tid == 0) A[c][c] = sqrtf(fmaxf(A[c][c], 1e-12f));
        __syncthreads();
        const float inv = 1.0f / A[c][c];
        for (int j = c + 1 + tid; j < b; j += nt) A[c][j] *= inv;
        __syncthreads();
        const int rem = b - c - 1;
        for (int w = tid; w < rem * rem; w += nt) {
            const int i = c + 1 + w / rem, j = c + 1 + w % rem;
            if (j >= i) A[i][j] -= A[c][i] * A[c][j];
        }
        __syncthreads();
    }
    // X = R_S^{-1} (upper) by back substitution, a thread per column
    for (int j = tid; j < b; j += nt) {
        for (int i = j; i >= 0; --i) {
            float s = (i == j) ? 1.0f : 0.0f;
            for (int q = i + 1; q <= j; ++q) s -= A[i][q] * X[q][j];
            X[i][j] = s / A[i][i];
        }
    }
    __syncthreads();
    for (int e = tid; e < b * b; e += nt) {
        const int q = e / b, c = e % b;
        Minv[e] = (c >= q) ? d[q] * (double)X[q][c] : 0.0;
    }
}

// V[c*pt + i] = sum_{q <= c} W[q*pt + i] Minv[q*b + c], a thread per (c, i).
__global__ void __launch_bounds__(256) apply_minv_kernel(const double *W, const double *Minv,
                                                        int64_t pt, int b, double *V) {
    __shared__ double Ms[kMaxB * kMaxB];
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) Ms[e] = Minv[e];
    __syncthreads();
    const int64_t total = (int64_t)b * pt;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / pt);
        const int64_t i = e - (int64_t)c * pt;
        double s = 0.0;
        for (int q = 0; q <= c; ++q) s = fma(W[(int64_t)q * pt + i], Ms[q * b + c], s);
        V[e] = s;
    }
}

// ---- cyclic Jacobi on a b x b symmetric matrix in shared memory, one CTA.
// Parallel (round-robin) ordering: each step applies bp/2 disjoint plane
// rotations at once (bp = b rounded up to even; the extra index is a
// decoupled zero row/column), bp - 1 steps per sweep; sweeps until the
// off-diagonal mass is at most tol of the total.  Q accumulates the rotations.
struct JacobiScratch {
    int rp[kMaxB / 2], rq[kMaxB / 2];
    double rc[kMaxB / 2], rs[kMaxB / 2];
    double red[2][256];
    int done;
};

__device__ __forceinline__ void rot_params(float app, float aqq, float apq, double &c,
                                           double &sn) {
    // float32 throughout (the float32 phase)
    if (apq == 0.0f) {
        c = 1.0;
        sn = 0.0;
        return;
    }
    const float th = (aqq - app) / (2.0f * apq);
    const float t = copysignf(1.0f, th) / (fabsf(th) + sqrtf(th * th + 1.0f));
    const float cf = rsqrtf(t * t + 1.0f);
    c = (double)cf;
    sn = (double)(t * cf);
}

__device__ __forceinline__ void rot_params(double app, double aqq, double apq, double &c,
                                           double &sn) {
    // the angle's tangent from a float32 estimate; c and s exact to float64
    // rounding for that tangent, so the rotation stays orthogonal
    if (fabs(apq) <= 1e-290) {
        c = 1.0;
        sn = 0.0;
        return;
    }
    const float th = (float)((aqq - app) * rcp_nr(2.0 * apq));
    const float tf = copysignf(1.0f, th) / (fabsf(th) + sqrtf(th * th + 1.0f));
    const double t = (double)tf;
    c = rsqrt_nr(1.0 + t * t);
    sn = t * c;
}

template <typename T, int LDA, int LDQ>
__device__ void jacobi_dev(T (*A)[LDA], T (*Q)[LDQ], int b, int max_sweeps, double tol,
                           JacobiScratch &js) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int bp = (b + 1) & ~1;
    const int half = bp / 2;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int e = tid; e < b * b; e += nt) {
            const int r = e / b, cc = e - r * b;
            const double x = (double)A[r][cc] * (double)A[r][cc];
            tot += x;
            if (r != cc) off += x;
        }
        js.red[0][tid] = off;
        js.red[1][tid] = tot;
        __syncthreads();
        for (int h = nt / 2; h > 0; h >>= 1) {
            if (tid < h) {
                js.red[0][tid] += js.red[0][tid + h];
                js.red[1][tid] += js.red[1][tid + h];
            }
            __syncthreads();
        }
        if (tid == 0) js.done = js.red[0][0] <= tol * js.red[1][0] || js.red[1][0] == 0.0;
        __syncthreads();
        if (js.done) break;
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
                double c = 1.0, sn = 0.0;
                if (p < b && q < b) rot_params(A[p][p], A[q][q], A[p][q], c, sn);
                js.rp[tid] = p;
                js.rq[tid] = q;
                js.rc[tid] = c;
                js.rs[tid] = sn;
            }
            __syncthreads();
            // columns: A <- A J, Q <- Q J (a pair with the padding index is
            // the identity)
            for (int w = tid; w < half * bp; w += nt) {
                const int k = w / bp, r = w - k * bp;
                const int p = js.rp[k], q = js.rq[k];
                if (p >= b || q >= b) continue;
                const T c = (T)js.rc[k], sn = (T)js.rs[k];
                const T arp = A[r][p], arq = A[r][q];
                A[r][p] = c * arp - sn * arq;
                A[r][q] = sn * arp + c * arq;
                if (r < b) {
                    const T qrp = Q[r][p], qrq = Q[r][q];
                    Q[r][p] = c * qrp - sn * qrq;
                    Q[r][q] = sn * qrp + c * qrq;
                }
            }
            __syncthreads();
            // rows: A <- J^T A
            for (int w = tid; w < half * bp; w += nt) {
                const int k = w / bp, r = w - k * bp;
                const int p = js.rp[k], q = js.rq[k];
                if (p >= b || q >= b) continue;
                const T c = (T)js.rc[k], sn = (T)js.rs[k];
                const T apr = A[p][r], aqr = A[q][r];
                A[p][r] = c * apr - sn * aqr;
                A[q][r] = sn * apr + c * aqr;
            }
            __syncthreads();
        }
    }
}

// Rayleigh-Ritz eigenproblem H = Q diag(lam) Q^T (b x b), one CTA:
//  1. Jacobi in float32 on H rounded to float32 -> Q32 (orthonormal to ~1e-7);
//  2. CholQR of Q32 in float64 -> Qa orthonormal to float64 rounding;
//  3. H' = Qa^T H Qa in float64 (off-diagonal ~1e-7 of the diagonal);
//  4. float64 Jacobi sweeps on H' -> Qb;  Q = Qa Qb, lam = diag.
struct RitzSmem {
    double A64[kMaxB][kMaxB + 1];
    double G[kMaxB][kMaxB + 1];
    double Qa[kMaxB][kMaxB];
    double Qb[kMaxB][kMaxB];
    float A32[kMaxB][kMaxB + 1];
    float Q32[kMaxB][kMaxB];
    double invd[kMaxB];
    double floor_v;
    JacobiScratch js;
};

__global__ void __launch_bounds__(256) ritz_eig_kernel(const double *Hin, int b, int k,
                                                      double *Qout, double *lam, double *ord) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RitzSmem &S = *reinterpret_cast<RitzSmem *>(smem_raw);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int bp = (b + 1) & ~1;
    for (int e = tid; e < bp * bp; e += nt) {
        const int r = e / bp, c = e % bp;
        const double h = (r < b && c < b) ? 0.5 * (Hin[r * b + c] + Hin[c * b + r]) : 0.0;
        S.A64[r][c] = h;
        S.A32[r][c] = (float)h;
        S.Q32[r][c] = (r == c) ? 1.0f : 0.0f;
    }
    __syncthreads();
    // float32 Jacobi stalls near float32 rounding (off-diagonal mass around
    // 1e-13 of the total), so it stops at 1e-10 or after 12 sweeps
    jacobi_dev<float, kMaxB + 1, kMaxB>(S.A32, S.Q32, b, 12, 1e-10, S.js);
    // G = Q32^T Q32 in float64
    for (int e = tid; e < b * b; e += nt) {
        const int i = e / b, j = e % b;
        double g = 0.0;
        for (int r = 0; r < b; ++r) g = fma((double)S.Q32[r][i], (double)S.Q32[r][j], g);
        S.G[i][j] = g;
    }
    __syncthreads();
    chol_dev<kMaxB + 1>(S.G, b, S.invd, &S.floor_v);
    // Qa = Q32 R^{-1}: forward substitution along each row
    for (int r = tid; r < b; r += nt) {
        for (int c = 0; c < b; ++c) {
            double s = (double)S.Q32[r][c];
            for (int q = 0; q < c; ++q) s = fma(-S.Qa[r][q], S.G[q][c], s);
            S.Qa[r][c] = s * S.invd[c];
        }
    }
    __syncthreads();
    // Qb = H Qa, then G = Qa^T Qb, then A64 = sym(G) (padding zero)
    for (int e = tid; e < b * b; e += nt) {
        const int r = e / b, c = e % b;
        double s = 0.0;
        for (int q = 0; q < b; ++q) s = fma(S.A64[r][q], S.Qa[q][c], s);
        S.Qb[r][c] = s;
    }
    __syncthreads();
    for (int e = tid; e < b * b; e += nt) {
        const int i = e / b, j = e % b;
        double s = 0.0;
        for (int r = 0; r < b; ++r) s = fma(S.Qa[r][i], S.Qb[r][j], s);
        S.G[i][j] = s;
    }
    __syncthreads();
    for (int e = tid; e < bp * bp; e += nt) {
        const int r = e / bp, c = e % bp;
        S.A64[r][c] = (r < b && c < b) ? 0.5 * (S.G[r][c] + S.G[c][r]) : 0.0;
        if (r < b && c < b) S.Qb[r][c] = (r == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    // the polish starts from off-diagonal mass ~1e-10..1e-14 of the total;
    // one or two sweeps reach 1e-26 (eigenvector directions to ~1e-13 / gap)
    jacobi_dev<double, kMaxB + 1, kMaxB>(S.A64, S.Qb, b, 30, 1e-26, S.js);
    for (int e = tid; e < b * b; e += nt) {
        const int r = e / b, c = e % b;
        double s = 0.0;
        for (int q = 0; q < b; ++q) s = fma(S.Qa[r][q], S.Qb[q][c], s);
        Qout[e] = s;
    }
    for (int r = tid; r < b; r += nt) lam[r] = S.A64[r][r];
    // indices of the k largest eigenvalues, descending (ties by lower index)
    if (tid == 0) {
        unsigned long long used = 0ull;
        for (int c = 0; c < k; ++c) {
            int pick = -1;
            for (int q = 0; q < b; ++q)
                if (!((used >> q) & 1ull) && (pick < 0 || S.A64[q][q] > S.A64[pick][pick])) pick = q;
            used |= 1ull << pick;
            ord[c] = (double)pick;
        }
    }
}

// U[c*pt + i] = sum_q V[q*pt + i] Q[q*b + ord[c]] and evals[c] = lam[ord[c]],
// a thread per (c, i).
__global__ void __launch_bounds__(256) ritz_u_kernel(const double *V, const double *Q,
                                                    const double *lam, const double *ord,
                                                    int64_t pt, int b, int k, double *U,
                                                    double *evals) {
    __shared__ double Qs[kMaxB * kMaxB];
    __shared__ int os[kMaxB];
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) Qs[e] = Q[e];
    for (int c = threadIdx.x; c < k; c += blockDim.x) os[c] = (int)ord[c];
    __syncthreads();
    if (blockIdx.x == 0)
        for (int c = threadIdx.x; c < k; c += blockDim.x) evals[c] = lam[os[c]];
    const int64_t total = (int64_t)k * pt;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / pt);
        const int64_t i = e - (int64_t)c * pt;
        const int col = os[c];
        double s = 0.0;
        for (int q = 0; q < b; ++q) s = fma(V[(int64_t)q * pt + i], Qs[q * b + col], s);
        U[e] = s;
    }
}

// Sign convention: each eigenvector's largest-magnitude entry (lowest index
// on ties) is made positive.  One CTA per vector.
__global__ void __launch_bounds__(256) sign_fix_kernel(int64_t pt, double *U) {
    __shared__ double red_v[256];
    __shared__ int64_t red_i[256];
    double *u = U + (int64_t)blockIdx.x * pt;
    double best = -1.0;
    int64_t besti = 0;
    for (int64_t i = threadIdx.x; i < pt; i += blockDim.x) {
        const double a = fabs(u[i]);
        if (a > best) {
            best = a;
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
    const bool flip = u[red_i[0]] < 0.0;
    __syncthreads();
    if (flip)
        for (int64_t i = threadIdx.x; i < pt; i += blockDim.x) u[i] = -u[i];
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

template <int BC>
cudaError_t panel_launch(dim3 grid, const double *C, const double *V, int64_t pt, int b,
                         int64_t jlen, double *W, cudaStream_t s) {
    panel_kernel<BC><<<grid, kPanelThreads, 0, s>>>(C, V, pt, b, jlen, W);
    return cudaGetLastError();
}

cudaError_t panel(dim3 grid, const double *C, const double *V, int64_t pt, int b, int64_t jlen,
                  double *W, cudaStream_t s) {
    switch ((b + 7) / 8) {
        case 1: return panel_launch<8>(grid, C, V, pt, b, jlen, W, s);
        case 2: return panel_launch<16>(grid, C, V, pt, b, jlen, W, s);
        case 3: return panel_launch<24>(grid, C, V, pt, b, jlen, W, s);
        case 4: return panel_launch<32>(grid, C, V, pt, b, jlen, W, s);
        case 5: return panel_launch<40>(grid, C, V, pt, b, jlen, W, s);
        case 6: return panel_launch<48>(grid, C, V, pt, b, jlen, W, s);
        case 7: return panel_launch<56>(grid, C, V, pt, b, jlen, W, s);
        default: return panel_launch<64>(grid, C, V, pt, b, jlen, W, s);
    }
}

cudaError_t launch_topk(const sk_ctx &c, const double *C, int k, int iters, double *evals,
                        double *U, double *work, cudaStream_t s) {
    const int64_t pt = c.pt;
    const int b = block_cols(pt, k);
    Ws w = carve(work, pt, b);
    const uint32_t k0 = (uint32_t)c.seed, k1 = (uint32_t)(c.seed >> 32);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // panel grid: 128-column tiles times j-ranges (multiples of 32 rows),
    // about two CTAs per SM
    const int64_t itiles = (pt + kPanelThreads - 1) / kPanelThreads;
    int64_t jsplit = (2LL * sms + itiles - 1) / itiles;
    if (jsplit > (pt + kPanelJ - 1) / kPanelJ) jsplit = (pt + kPanelJ - 1) / kPanelJ;
    if (jsplit < 1) jsplit = 1;
    int64_t jlen = (pt + jsplit - 1) / jsplit;
    jlen = (jlen + kPanelJ - 1) / kPanelJ * kPanelJ;
    jsplit = (pt + jlen - 1) / jlen;
    const dim3 pgrid((unsigned)itiles, (unsigned)jsplit);
    int eblocks = (int)((b * pt + 255) / 256);
    if (eblocks > 4096) eblocks = 4096;
    const unsigned ablocks = (unsigned)((pt + kApplyThreads - 1) / kApplyThreads);
    const size_t apply_smem = (size_t)(b * b + b + kApplyThreads * b) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(apply_solve_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)apply_smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(ritz_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(RitzSmem));
    if (e != cudaSuccess) return e;
    int mblocks = (int)((b * pt + 255) / 256);
    if (mblocks > 4 * sms) mblocks = 4 * sms;
    int ublocks = (int)((k * pt + 255) / 256);
    if (ublocks > 4 * sms) ublocks = 4 * sms;
    // at least one CholQR, the last one in float64
    const int n_it = iters > 0 ? iters : 1;
    init_v_kernel<<<eblocks, 256, 0, s>>>(w.V, pt, b, k0, k1);
    for (int it = 0; it <= n_it; ++it) {
        e = cudaMemsetAsync(w.W, 0, (size_t)b * pt * sizeof(double), s);
        if (e != cudaSuccess) return e;
        e = panel(pgrid, C, w.V, pt, b, jlen, w.W, s);
        if (e != cudaSuccess) return e;
        if (it == n_it) break;
        small_gram_kernel<<<b * b, 256, 0, s>>>(w.W, w.W, pt, b, w.Gm);
        if (it < n_it - 1) {
            chol32_kernel<<<1, 256, 0, s>>>(w.Gm, b, w.R);
            apply_minv_kernel<<<mblocks, 256, 0, s>>>(w.W, w.R, pt, b, w.V);
        } else {
            chol_kernel<<<1, 256, 0, s>>>(w.Gm, b, w.R, w.lam);
            apply_solve_kernel<<<ablocks, kApplyThreads, apply_smem, s>>>(w.W, w.R, w.lam, pt,
                                                                          b, w.V);
        }
    }
    // Rayleigh-Ritz: H = V^T (C V); the order of the k largest goes to Gm
    small_gram_kernel<<<b * b, 256, 0, s>>>(w.V, w.W, pt, b, w.H);
    ritz_eig_kernel<<<1, 256, sizeof(RitzSmem), s>>>(w.H, b, k, w.Q, w.lam, w.Gm);
    ritz_u_kernel<<<ublocks, 256, 0, s>>>(w.V, w.Q, w.lam, w.Gm, pt, b, k, U, evals);
    sign_fix_kernel<<<k, 256, 0, s>>>(pt, U);
    return cudaGetLastError();
}

}  // namespace sk
