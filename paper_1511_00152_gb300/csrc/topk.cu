// topk.cu -- top-k principal subspace of the symmetric pt x pt estimate C_n
// (Sec. V: PCA recovers the leading eigenvectors of the covariance), to
// float64 accuracy on the device.
//
// Block subspace iteration with b = min(pt, 64, max(k + 8, 2k)) columns:
//   W = C V;  V = W R^{-1} with R the Cholesky factor of W^T W (CholQR),
// repeated `iters` times (at least once) from a seeded start, the last
// CholQR in float64 and the earlier ones from a float32 factor (see
// chol32_kernel), the products C V of all but the last two iterations in
// float32 and the last two in double-float (see panel_kernel and DF), then
// one Rayleigh-Ritz step:
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
// j-range; a thread owns column i and its BC >= b accumulators.  The j-range
// goes in chunks of kPanelJ rows: the chunk's tile of C (kPanelJ x 128
// doubles) is copied to shared memory with cp.async one chunk ahead of its
// use (two buffers), and V's slice of the chunk is staged in shared memory
// and read as a broadcast.  W is zeroed before the launch and receives the
// partial sums with double atomics.
// T is the arithmetic: DF (double-float, below) for the products that need
// float64 accuracy, or float for the early iterations (C, scaled by 2^tshift, and V rounded to float as they are
// read, float products and sums; W then holds 2^tshift C V), whose only job
// is to turn V towards the dominant subspace.
constexpr int kPanelThreads = 128;
constexpr int kPanelJ = 16;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// 16-byte global-to-shared copy of the first src_bytes (0..16) bytes of src,
// zero-filling the rest (no byte is read when src_bytes is 0).
__device__ __forceinline__ void cp_async16(void *dst, const void *src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}

// x * 2^t rounded toward zero to float, from the bit pattern of x on the
// integer units (float64-to-float32 conversion instructions run at the low
// float64 rate of this GPU).  Magnitudes below the float normal range
// become zero; a result past the float range keeps the largest exponent.
__device__ __forceinline__ float to_f32_rz(double x, int t) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
    int e = (int)((hi >> 20) & 0x7FFu) - 1023 + 127 + t;
    const uint32_t mant = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    e = e > 254 ? 254 : e;
    const uint32_t bits = (hi & 0x80000000u) | ((uint32_t)e << 23) | mant;
    return e <= 0 ? 0.f : __uint_as_float(bits);
}

// Double-float number h + l (two float32s, |l| below half an ulp of h or
// so): the arithmetic of the panels that need float64 accuracy on this GPU,
// whose float32 FMA rate is about thirty times its float64 rate.  A
// product of two double-float
// numbers is formed with the error-free float32 product (an FMA gives the
// rounding error of h1 h2 exactly) plus the cross terms h1 l2 and l1 h2 (l1
// l2 is dropped), and is added to the accumulator with Knuth's TwoSum;
// about 2^-44 relative per product, twelve float32 operations.
struct DF {
    float h, l;
};

// The part of x that to_f32_rz(x, 0) dropped (the mantissa's low 29 bits,
// rounded to float32), from the bit pattern on the integer units.
__device__ __forceinline__ float f64_tail(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((u >> 52) & 0x7FFu) - 1023 - 52;  // weight of the mantissa's bit 0
    const uint32_t m29 = (uint32_t)(u & 0x1FFFFFFFull);
    if (m29 == 0u || e < -126 || e > 127 - 29) return 0.f;
    const float v = __uint2float_rn(m29) * __int_as_float((e + 127) << 23);
    return (u >> 63) ? -v : v;
}

template <typename T>
__device__ __forceinline__ T panel_in(double x, int t);
template <>
__device__ __forceinline__ float panel_in<float>(double x, int t) { return to_f32_rz(x, t); }
template <>
__device__ __forceinline__ DF panel_in<DF>(double x, int) {
    const float h = to_f32_rz(x, 0);
    return DF{h, h == 0.f ? 0.f : f64_tail(x)};
}

template <typename T>
__device__ __forceinline__ T panel_zero() {
    return T(0);
}
template <>
__device__ __forceinline__ DF panel_zero<DF>() {
    return DF{0.f, 0.f};
}

// acc + a b
template <typename T>
__device__ __forceinline__ T panel_fma(T a, T b, T acc) {
    return fma(a, b, acc);
}
template <>
__device__ __forceinline__ DF panel_fma<DF>(DF a, DF b, DF acc) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    const float t = __fadd_rn(acc.h, p);
    const float z = __fsub_rn(t, acc.h);
    const float err = __fadd_rn(__fsub_rn(acc.h, __fsub_rn(t, z)), __fsub_rn(p, z));
    return DF{t, __fadd_rn(acc.l, __fadd_rn(err, e))};
}

template <typename T>
__device__ __forceinline__ double panel_out(T x) {
    return (double)x;
}
template <>
__device__ __forceinline__ double panel_out<DF>(DF x) {
    return (double)x.h + (double)x.l;
}

// *tshift = -(binary exponent of max_i |C_ii|): the float32 panels read C
// scaled by 2^tshift, which puts the largest diagonal entry near 1 (the
// scale cancels in the float32 CholQR, which normalises by the Gram's
// diagonal).
__global__ void __launch_bounds__(256) diag_shift_kernel(const double *C, int64_t pt,
                                                        int *tshift) {
    __shared__ int red[256];
    int emax = 0;
    for (int64_t i = threadIdx.x; i < pt; i += blockDim.x) {
        const unsigned long long u = (unsigned long long)__double_as_longlong(C[i * pt + i]);
        const int e = (int)((u >> 52) & 0x7FFu);
        emax = e > emax ? e : emax;
    }
    red[threadIdx.x] = emax;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h && red[threadIdx.x + h] > red[threadIdx.x])
            red[threadIdx.x] = red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) *tshift = (red[0] == 0 || red[0] == 0x7FF) ? 0 : 1023 - red[0];
}

template <int BC, typename T>
__global__ void __launch_bounds__(kPanelThreads) panel_kernel(const double *C, const double *V,
                                                             int64_t pt, int b, int64_t jlen,
                                                             const int *tshift, double *W) {
    static_assert(kPanelThreads == 128 && kPanelJ % 2 == 0, "tile shape");
    constexpr int VPT = (kPanelJ * BC + kPanelThreads - 1) / kPanelThreads;  // V loads / thread
    __shared__ __align__(16) double Cs[2][kPanelJ][kPanelThreads];
    __shared__ __align__(16) T Vs[2][kPanelJ][BC];
    const int tid = threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.x * kPanelThreads;
    const int64_t jb = (int64_t)blockIdx.y * jlen;
    const int64_t je = (jb + jlen < pt) ? jb + jlen : pt;
    const int nch = (int)((je - jb + kPanelJ - 1) / kPanelJ);
    const int tC = sizeof(T) == 4 ? *tshift : 0;

    // C tile of chunk q: kPanelJ rows x 64 pieces of 16 bytes (two doubles)
    auto issue_c = [&](int q) {
        const int64_t j0 = jb + (int64_t)q * kPanelJ;
#pragma unroll
        for (int r = 0; r < kPanelJ * 64 / kPanelThreads; ++r) {
            const int e = r * kPanelThreads + tid;
            const int jj = e >> 6, seg = e & 63;
            const int64_t j = j0 + jj, col = i0 + 2 * seg;
            int bytes = 0;
            if (j < je && col < pt) bytes = (pt - col >= 2) ? 16 : 8;
            cp_async16(&Cs[q & 1][jj][2 * seg], bytes ? (const void *)(C + j * pt + col) : C,
                       bytes);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    // V slice of chunk q (consecutive threads: consecutive rows of a column)
    auto load_v = [&](int q, T (&vr)[VPT]) {
        const int64_t j0 = jb + (int64_t)q * kPanelJ;
#pragma unroll
        for (int r = 0; r < VPT; ++r) {
            const int e = r * kPanelThreads + tid;
            const int c = e / kPanelJ, jj = e - c * kPanelJ;
            vr[r] = (e < kPanelJ * BC && c < b && j0 + jj < je)
                        ? panel_in<T>(V[(int64_t)c * pt + j0 + jj], 0)
                        : panel_zero<T>();
        }
    };
    auto store_v = [&](int q, const T (&vr)[VPT]) {
#pragma unroll
        for (int r = 0; r < VPT; ++r) {
            const int e = r * kPanelThreads + tid;
            const int c = e / kPanelJ, jj = e - c * kPanelJ;
            if (e < kPanelJ * BC) Vs[q & 1][jj][c] = vr[r];
        }
    };

    T acc[BC];
#pragma unroll
    for (int c = 0; c < BC; ++c) acc[c] = panel_zero<T>();
    if (nch > 0) {
        T vr[VPT];
        issue_c(0);
        load_v(0, vr);
        store_v(0, vr);
    }
    for (int q = 0; q < nch; ++q) {
        T vr[VPT];
        const bool more = q + 1 < nch;
        if (more) {
            issue_c(q + 1);
            load_v(q + 1, vr);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
#pragma unroll
        for (int jj = 0; jj < kPanelJ; ++jj) {
            const T cv = panel_in<T>(Cs[q & 1][jj][tid], tC);
#pragma unroll
            for (int c = 0; c < BC; ++c) acc[c] = panel_fma<T>(cv, Vs[q & 1][jj][c], acc[c]);
        }
        if (more) store_v(q + 1, vr);
        __syncthreads();
    }
    const int64_t i = i0 + tid;
    if (i < pt) {
#pragma unroll
        for (int c = 0; c < BC; ++c)
            if (c < b) atomicAdd(W + (int64_t)c * pt + i, panel_out<T>(acc[c]));
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

// Gm += W^T W in float32 for the intermediate iterations, whose Gram only
// feeds the float32 Cholesky of chol32_kernel.  A CTA takes a 64-row slice
// of W (each element converted to float once, into shared memory) and adds
// its b x b partial sums to Gm with double atomics; Gm starts at zero
// (chol32_kernel clears it after reading it).
constexpr int kG32Rows = 64;
__global__ void __launch_bounds__(256) gram32_kernel(const double *W, int64_t pt, int b,
                                                    double *Gm) {
    __shared__ float Ws[kG32Rows][kMaxB + 1];
    const int64_t r0 = (int64_t)blockIdx.x * kG32Rows;
    for (int e = threadIdx.x; e < kG32Rows * b; e += blockDim.x) {
        const int c = e / kG32Rows, r = e - c * kG32Rows;
        Ws[r][c] = (r0 + r < pt) ? (float)W[(int64_t)c * pt + r0 + r] : 0.f;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
        const int c1 = e / b, c2 = e - c1 * b;
        if (c2 < c1) continue;
        float s = 0.f;
#pragma unroll 8
        for (int r = 0; r < kG32Rows; ++r) s = fmaf(Ws[r][c1], Ws[r][c2], s);
        atomicAdd(Gm + c1 * b + c2, (double)s);
        if (c2 != c1) atomicAdd(Gm + c2 * b + c1, (double)s);
    }
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
__global__ void __launch_bounds__(256) chol32_kernel(double *Gm, int b, double *Minv) {
    __shared__ float A[kMaxB][kMaxB + 1];  // the scaled Gram, later X = R_S^{-1}
    __shared__ float R[kMaxB][kMaxB + 1];  // R_S, upper
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
    // Gm is read: clear it for the next iteration's gram32_kernel
    for (int e = tid; e < b * b; e += nt) Gm[e] = 0.0;
    // right-looking, one barrier per column: row c of R is written to R while
    // the trailing update reads the unscaled row c of A and scales it itself
    for (int c = 0; c < b; ++c) {
        const float rc = sqrtf(fmaxf(A[c][c], 1e-12f));
        const float inv = 1.0f / rc;
        for (int j = c + tid; j < b; j += nt) R[c][j] = (j == c) ? rc : A[c][j] * inv;
        const int rem = b - c - 1;
        for (int w = tid; w < rem * rem; w += nt) {
            const int i = c + 1 + w / rem, j = c + 1 + w % rem;
            if (j >= i) A[i][j] -= (A[c][i] * inv) * (A[c][j] * inv);
        }
        __syncthreads();
    }
    // X = R_S^{-1} (upper) by back substitution, a thread per column, into A
    float (*X)[kMaxB + 1] = A;
    for (int j = tid; j < b; j += nt) {
        for (int i = j; i >= 0; --i) {
            float s = (i == j) ? 1.0f : 0.0f;
            for (int q = i + 1; q <= j; ++q) s -= R[i][q] * X[q][j];
            X[i][j] = s / R[i][i];
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
    unsigned char pp[kMaxB][kMaxB / 2], pq[kMaxB][kMaxB / 2];  // pair (p, q) of slot k at step s
    double rc[kMaxB / 2], rs[kMaxB / 2];
    float rcf[kMaxB / 2], rsf[kMaxB / 2];
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
    // circle-method pairing of every step: index 0 fixed, 1..bp-1 rotate
    for (int e = tid; e < (bp - 1) * half; e += nt) {
        const int step = e / half, k = e - step * half;
        int p, q;
        if (k == 0) {
            p = 0;
            q = 1 + step % (bp - 1);
        } else {
            p = 1 + (step + k) % (bp - 1);
            q = 1 + (step - k + (bp - 1)) % (bp - 1);
        }
        js.pp[step][k] = (unsigned char)p;
        js.pq[step][k] = (unsigned char)q;
    }
    __syncthreads();
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
                const int p = js.pp[step][tid], q = js.pq[step][tid];
                double c = 1.0, sn = 0.0;
                if (p < b && q < b) rot_params(A[p][p], A[q][q], A[p][q], c, sn);
                js.rc[tid] = c;
                js.rs[tid] = sn;
                js.rcf[tid] = (float)c;
                js.rsf[tid] = (float)sn;
            }
            __syncthreads();
            // A <- J^T A J on the 2 x 2 blocks (pair i rows, pair j columns):
            // the blocks are disjoint, so each is updated on its own, the
            // column rotation first, then the row rotation.  A pair with the
            // padding index is the identity (its entries stay zero).
            for (int w = tid; w < half * half; w += nt) {
                const int ki = w / half, kj = w - ki * half;
                const int p = js.pp[step][ki], q = js.pq[step][ki];
                const int r = js.pp[step][kj], t = js.pq[step][kj];
                T ci, si, cj, sj;
                if constexpr (sizeof(T) == 4) {
                    ci = js.rcf[ki]; si = js.rsf[ki]; cj = js.rcf[kj]; sj = js.rsf[kj];
                } else {
                    ci = js.rc[ki]; si = js.rs[ki]; cj = js.rc[kj]; sj = js.rs[kj];
                }
                const T apr = A[p][r], apt = A[p][t], aqr = A[q][r], aqt = A[q][t];
                const T bpr = cj * apr - sj * apt, bpt = sj * apr + cj * apt;
                const T bqr = cj * aqr - sj * aqt, bqt = sj * aqr + cj * aqt;
                A[p][r] = ci * bpr - si * bqr;
                A[q][r] = si * bpr + ci * bqr;
                A[p][t] = ci * bpt - si * bqt;
                A[q][t] = si * bpt + ci * bqt;
            }
            // Q <- Q J
            for (int w = tid; w < b * half; w += nt) {
                const int row = w / half, k = w - row * half;
                const int p = js.pp[step][k], q = js.pq[step][k];
                if (p >= b || q >= b) continue;
                T c, sn;
                if constexpr (sizeof(T) == 4) {
                    c = js.rcf[k]; sn = js.rsf[k];
                } else {
                    c = js.rc[k]; sn = js.rs[k];
                }
                const T qrp = Q[row][p], qrq = Q[row][q];
                Q[row][p] = c * qrp - sn * qrq;
                Q[row][q] = sn * qrp + c * qrq;
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
    // 1e-13 of the total), so it stops at 1e-12 or after 15 sweeps; its
    // sweeps cost a small fraction of a float64 sweep's
    jacobi_dev<float, kMaxB + 1, kMaxB>(S.A32, S.Q32, b, 15, 1e-12, S.js);
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
    // the polish starts from off-diagonal mass ~1e-12..1e-14 of the total;
    // a sweep with float32-estimated angles shrinks it by ~1e-13 or more, so
    // one sweep normally reaches 1e-20 (off-diagonal norm 1e-10 of the
    // total: eigenvalues to ~1e-20 relative, eigenvector directions to
    // ~1e-10 / relative gap)
    jacobi_dev<double, kMaxB + 1, kMaxB>(S.A64, S.Qb, b, 30, 1e-20, S.js);
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
// up with cudaGetSymbolAddress on every call, with the caller's device current,
// so that no stale address survives a device reset or a new context.
namespace {
constexpr int64_t kTopkStaticDoubles = 512 * 1024;  // 4 MiB
static __device__ __align__(256) double g_topk_scratch[kTopkStaticDoubles];
}  // namespace

int64_t topk_static_capacity() { return kTopkStaticDoubles; }

cudaError_t topk_static_scratch(double **out) {
    *out = nullptr;
    void *ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_topk_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<double *>(ptr);
    return cudaSuccess;
}

int64_t topk_workspace(int64_t pt, int k) {
    const int b = block_cols(pt, k);
    return 2 * (int64_t)b * pt + 4 * (int64_t)b * b + b;
}

template <int BC>
cudaError_t panel_launch(dim3 grid, const double *C, const double *V, int64_t pt, int b,
                         int64_t jlen, const int *tshift, double *W, bool f32, cudaStream_t s) {
    if (f32)
        panel_kernel<BC, float><<<grid, kPanelThreads, 0, s>>>(C, V, pt, b, jlen, tshift, W);
    else
        panel_kernel<BC, DF><<<grid, kPanelThreads, 0, s>>>(C, V, pt, b, jlen, tshift, W);
    return cudaGetLastError();
}

cudaError_t panel(dim3 grid, const double *C, const double *V, int64_t pt, int b, int64_t jlen,
                  const int *tshift, double *W, bool f32, cudaStream_t s) {
    switch ((b + 7) / 8) {
        case 1: return panel_launch<8>(grid, C, V, pt, b, jlen, tshift, W, f32, s);
        case 2: return panel_launch<16>(grid, C, V, pt, b, jlen, tshift, W, f32, s);
        case 3: return panel_launch<24>(grid, C, V, pt, b, jlen, tshift, W, f32, s);
        case 4: return panel_launch<32>(grid, C, V, pt, b, jlen, tshift, W, f32, s);
        case 5: return panel_launch<40>(grid, C, V, pt, b, jlen, tshift, W, f32, s);
        case 6: return panel_launch<48>(grid, C, V, pt, b, jlen, tshift, W, f32, s);
        case 7: return panel_launch<56>(grid, C, V, pt, b, jlen, tshift, W, f32, s);
        default: return panel_launch<64>(grid, C, V, pt, b, jlen, tshift, W, f32, s);
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
    // panel grid: 128-column tiles times j-ranges (multiples of kPanelJ
    // rows, at least four chunks), about four CTAs per SM
    const int64_t itiles = (pt + kPanelThreads - 1) / kPanelThreads;
    int64_t jsplit = (4LL * sms + itiles - 1) / itiles;
    const int64_t jmax = (pt + 4 * kPanelJ - 1) / (4 * kPanelJ);
    if (jsplit > jmax) jsplit = jmax;
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
    // at least one CholQR, the last one in float64; the last three panel
    // products (two power steps and the Rayleigh-Ritz product) in
    // double-float, the earlier ones in float32: each double-float step
    // shrinks the float32 rounding left in span(V) by the gap ratio
    // lambda_{b+1} / lambda_k.
    const int n_it = iters > 0 ? iters : 1;
    const unsigned g32blocks = (unsigned)((pt + kG32Rows - 1) / kG32Rows);
    init_v_kernel<<<eblocks, 256, 0, s>>>(w.V, pt, b, k0, k1);
    e = cudaMemsetAsync(w.Gm, 0, (size_t)b * b * sizeof(double), s);
    if (e != cudaSuccess) return e;
    // H is free until the Rayleigh-Ritz step: it holds the float32 panels' shift
    int *tshift = reinterpret_cast<int *>(w.H);
    if (n_it > 2) diag_shift_kernel<<<1, 256, 0, s>>>(C, pt, tshift);
    for (int it = 0; it <= n_it; ++it) {
        e = cudaMemsetAsync(w.W, 0, (size_t)b * pt * sizeof(double), s);
        if (e != cudaSuccess) return e;
        e = panel(pgrid, C, w.V, pt, b, jlen, tshift, w.W, it < n_it - 2, s);
        if (e != cudaSuccess) return e;
        if (it == n_it) break;
        if (it < n_it - 1) {
            gram32_kernel<<<g32blocks, 256, 0, s>>>(w.W, pt, b, w.Gm);
            chol32_kernel<<<1, 256, 0, s>>>(w.Gm, b, w.R);
            apply_minv_kernel<<<mblocks, 256, 0, s>>>(w.W, w.R, pt, b, w.V);
        } else {
            small_gram_kernel<<<b * b, 256, 0, s>>>(w.W, w.W, pt, b, w.Gm);
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
