// dct.cu -- the DCT preconditioner (Sec. III: y = H D x with H an orthonormal
// DCT matrix; the preconditioner of the paper's big-data runs, Sec. VII) for
// any even p without zero padding, and its transpose for un-mixing.
//
// The orthonormal DCT-II of length N = p is computed from one complex FFT of
// length L = N / 2 (the even/odd reordering of J. Makhoul, "A fast cosine
// transform in one and two dimensions", IEEE TASSP 1980):
//   v_l = u_2l, v_{N-1-l} = u_{2l+1}; z_l = v_2l + i v_{2l+1};  Z = FFT_L(z);
//   V_k = E_k + e^{-2 pi i k / N} O_k,  E_k = (Z_k + conj Z_{L-k}) / 2,
//   O_k = (Z_k - conj Z_{L-k}) / (2i);  W_k = e^{-i pi k / (2N)} V_k;
//   X_k = Re W_k,  X_{N-k} = -Im W_k  (0 < k < L),  y_k = s_k X_k,
// s_0 = sqrt(1/N), s_k = sqrt(2/N).  The inverse (DCT-III, the un-mixing map
// D H^T) runs the same steps backwards with the inverse FFT.
// The FFT is a mixed-radix self-sorting (Stockham) transform in shared memory
// (Govindaraju et al., "High performance discrete Fourier transforms on
// graphics processors", SC'08): each stage of radix R takes the L / R
// butterflies j, multiplies input r by the twiddle exp(-2 pi i k r / (Ns R))
// (k = j mod Ns, Ns the product of the earlier radices), takes the R-point
// DFT and writes output q to (j / Ns) Ns R + k + q Ns.  Supported radices are
// 2, 3, 4, 5, 7, 8, 11, 13 (the factorisation of L is made at sk_init_ex).
//
// Forward rows (compress and precondition) are the hot path: one warp per
// row for p <= 1024 (no block-wide barriers; the CTA's warps share the
// tables), else one CTA per row at a time, persistent over rows, with the
// FFT twiddles and the two post-processing phase tables computed once per CTA
// in float32; the mask of each row has already been drawn (mask_kernel,
// range p) and the row's warp or CTA gathers val = y[idx].  Un-mixing (few rows) computes its twiddles as it goes, in
// float32 or float64.
#include <cstring>

#include <algorithm>

#include "sk_internal.cuh"

namespace sk {
namespace {

template <typename T>
struct Cx;
template <>
struct Cx<float> {
    using type = float2;
};
template <>
struct Cx<double> {
    using type = double2;
};

template <typename C2>
__device__ __forceinline__ C2 cmul(C2 a, C2 b) {
    C2 r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename C2>
__device__ __forceinline__ C2 cadd(C2 a, C2 b) {
    a.x += b.x;
    a.y += b.y;
    return a;
}
template <typename C2>
__device__ __forceinline__ C2 csub(C2 a, C2 b) {
    a.x -= b.x;
    a.y -= b.y;
    return a;
}
template <typename C2>
__device__ __forceinline__ C2 cconj(C2 a) {
    a.y = -a.y;
    return a;
}

// exp(sign * i pi x) in the arithmetic of T.
__device__ __forceinline__ float2 expipi(float x, float sign) {
    float s, c;
    sincospif(x, &s, &c);
    return make_float2(c, sign * s);
}
__device__ __forceinline__ double2 expipi(double x, double sign) {
    double s, c;
    sincospi(x, &s, &c);
    return make_double2(c, sign * s);
}

struct DctParams {
    const void *in;   // forward: X (float, n x ldx); inverse: rows (T, n x N)
    int64_t n, ldx;
    int N, L;         // transform length (= p) and FFT length N / 2
    int nf;
    int fac[16];      // radices of L, in stage order
    uint32_t k0, k1;  // seed (sign spec)
    const int32_t *idx;  // forward gather: masks (n x m)
    float *val;          // forward gather: output (n x m)
    void *out;           // forward dense: Y (float, n x N); inverse: rows (T, n x N)
    int m;
    int vec;             // forward: rows 16-byte aligned with N % 4 == 0 (float4 loads)
};

// Twiddle exp(-2 pi i dir t / L): dir = 1 forward, -1 inverse; from the
// CTA's table (forward only) or computed.
template <typename T, bool TABLE>
struct Twiddle {
    using C2 = typename Cx<T>::type;
    const C2 *tab;
    int L;
    T dir;
    __device__ __forceinline__ C2 operator()(int t) const {
        if constexpr (TABLE) {
            return tab[t];
        } else {
            return expipi((T)(2 * t) / (T)L, -dir);
        }
    }
};

// Radix-4 butterfly on x0..x3 (w_4 = -i dir), outputs in natural order.
template <typename C2, typename R>
__device__ __forceinline__ void dft4(C2 x0, C2 x1, C2 x2, C2 x3, R dir, C2 &y0, C2 &y1, C2 &y2,
                                     C2 &y3) {
    const C2 a = cadd(x0, x2), b = csub(x0, x2);
    const C2 c = cadd(x1, x3), d = csub(x1, x3);
    C2 dm;  // d times -i dir
    dm.x = d.y * dir;
    dm.y = -d.x * dir;
    y0 = cadd(a, c);
    y2 = csub(a, c);
    y1 = cadd(b, dm);
    y3 = csub(b, dm);
}

// One Stockham stage of radix R: in -> out (both L complex in shared memory).
// Radix 2, 4 and 8 are written out; an odd radix uses the symmetric form of
// the R-point DFT: with a_r = x_r + x_{R-r}, b_r = x_r - x_{R-r} (r <= H =
// (R-1)/2), y_q = x_0 + sum_r a_r cos(2 pi r q / R) - i dir sum_r b_r
// sin(2 pi r q / R) and y_{R-q} the same with + i dir, a quarter of the
// multiplications of the direct sum.
template <int R, typename C2, typename TW>
__device__ __forceinline__ void fft_stage(const C2 *in, C2 *out, int L, int Ns, const TW &tw,
                                          int tid, int nthr) {
    using T = decltype(C2().x);
    const int S = L / R;
    const int st = L / (Ns * R);  // twiddle stride: k r st < L
    C2 rt[R];                     // the R-th roots of unity, rt[s] = w_R^s
#pragma unroll
    for (int s = 0; s < R; ++s) rt[s] = tw(s * S);
    for (int j = tid; j < S; j += nthr) {
        const int jq = j / Ns;
        const int k = j - jq * Ns;
        C2 x[R];
#pragma unroll
        for (int r = 0; r < R; ++r) x[r] = in[j + r * S];
        if (Ns > 1) {  // the first stage's twiddles are all 1
#pragma unroll
            for (int r = 1; r < R; ++r) x[r] = cmul(x[r], tw(k * r * st));
        }
        const int base = jq * Ns * R + k;
        if constexpr (R == 2) {
            out[base] = cadd(x[0], x[1]);
            out[base + Ns] = csub(x[0], x[1]);
        } else if constexpr (R == 4) {
            C2 y0, y1, y2, y3;
            dft4(x[0], x[1], x[2], x[3], tw.dir, y0, y1, y2, y3);
            out[base] = y0;
            out[base + Ns] = y1;
            out[base + 2 * Ns] = y2;
            out[base + 3 * Ns] = y3;
        } else if constexpr (R == 8) {
            // two radix-4 DFTs of the even and odd inputs, then w_8^q
            C2 e0, e1, e2, e3, o0, o1, o2, o3;
            dft4(x[0], x[2], x[4], x[6], tw.dir, e0, e1, e2, e3);
            dft4(x[1], x[3], x[5], x[7], tw.dir, o0, o1, o2, o3);
            const T h = (T)0.70710678118654752440;
            C2 t1, t2, t3;  // o1 w_8, o2 w_8^2, o3 w_8^3 with w_8 = h (1 - i dir)
            t1.x = h * (o1.x + tw.dir * o1.y);
            t1.y = h * (o1.y - tw.dir * o1.x);
            t2.x = tw.dir * o2.y;
            t2.y = -tw.dir * o2.x;
            t3.x = h * (-o3.x + tw.dir * o3.y);
            t3.y = h * (-o3.y - tw.dir * o3.x);
            out[base] = cadd(e0, o0);
            out[base + 4 * Ns] = csub(e0, o0);
            out[base + Ns] = cadd(e1, t1);
            out[base + 5 * Ns] = csub(e1, t1);
            out[base + 2 * Ns] = cadd(e2, t2);
            out[base + 6 * Ns] = csub(e2, t2);
            out[base + 3 * Ns] = cadd(e3, t3);
            out[base + 7 * Ns] = csub(e3, t3);
        } else {
            constexpr int H = (R - 1) / 2;
            C2 a[H + 1], b[H + 1];
            C2 y0 = x[0];
#pragma unroll
            for (int r = 1; r <= H; ++r) {
                a[r] = cadd(x[r], x[R - r]);
                b[r] = csub(x[r], x[R - r]);
                y0 = cadd(y0, a[r]);
            }
            out[base] = y0;
#pragma unroll
            for (int q = 1; q <= H; ++q) {
                C2 re = x[0], im;
                im.x = (T)0;
                im.y = (T)0;
#pragma unroll
                for (int r = 1; r <= H; ++r) {
                    const C2 w = rt[(r * q) % R];  // (cos, -dir sin) of 2 pi r q / R
                    re.x += a[r].x * w.x;
                    re.y += a[r].y * w.x;
                    im.x -= b[r].x * w.y;  // b_r dir sin
                    im.y -= b[r].y * w.y;
                }
                // y_q = re - i im, y_{R-q} = re + i im
                C2 yq, yr;
                yq.x = re.x + im.y;
                yq.y = re.y - im.x;
                yr.x = re.x - im.y;
                yr.y = re.y + im.x;
                out[base + q * Ns] = yq;
                out[base + (R - q) * Ns] = yr;
            }
        }
    }
}

// FFT of a (L complex) using b as the other buffer; returns the buffer that
// holds the result.  The CTA's threads take part; syncs between stages.
template <typename C2, typename TW, bool WARP = false>
__device__ C2 *fft(C2 *a, C2 *b, const DctParams &P, const TW &tw, int tid, int nthr) {
    int Ns = 1;
    for (int s = 0; s < P.nf; ++s) {
        const int R = P.fac[s];
        switch (R) {
            case 2: fft_stage<2>(a, b, P.L, Ns, tw, tid, nthr); break;
            case 3: fft_stage<3>(a, b, P.L, Ns, tw, tid, nthr); break;
            case 4: fft_stage<4>(a, b, P.L, Ns, tw, tid, nthr); break;
            case 5: fft_stage<5>(a, b, P.L, Ns, tw, tid, nthr); break;
            case 7: fft_stage<7>(a, b, P.L, Ns, tw, tid, nthr); break;
            case 8: fft_stage<8>(a, b, P.L, Ns, tw, tid, nthr); break;
            case 11: fft_stage<11>(a, b, P.L, Ns, tw, tid, nthr); break;
            default: fft_stage<13>(a, b, P.L, Ns, tw, tid, nthr); break;
        }
        if constexpr (WARP) {
            __syncwarp();
        } else {
            __syncthreads();
        }
        C2 *t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    return a;
}

__device__ __forceinline__ bool sign_neg(const uint32_t *sgn, int l) {
    return (sgn[l >> 5] >> (l & 31)) & 1u;
}

// Forward rows.  DENSE: Y[i] = H D x_i; else val[i, t] = (H D x_i)[idx[i, t]].
template <bool DENSE>
__global__ void __launch_bounds__(512) dct_forward_kernel(DctParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = P.N, L = P.L;
    const int tid = threadIdx.x, nthr = blockDim.x;
    float2 *tw = reinterpret_cast<float2 *>(smem_raw);  // L: exp(-2 pi i t / L)
    float2 *ph = tw + L;                                 // L + 1: exp(-i pi k / (2N))
    float2 *om = ph + (L + 1);                           // L + 1: exp(-2 pi i k / N)
    float2 *b0 = om + (L + 1);                           // L
    float2 *b1 = b0 + L;                                 // L
    uint32_t *sgn = reinterpret_cast<uint32_t *>(b1 + L);  // ceil(N / 32)
    for (int t = tid; t < L; t += nthr) tw[t] = expipi((float)(2 * t) / (float)L, -1.f);
    for (int k = tid; k <= L; k += nthr) {
        ph[k] = expipi((float)k / (float)(2 * N), -1.f);
        om[k] = expipi((float)(2 * k) / (float)N, -1.f);
    }
    for (int w = tid; w < (N + 31) / 32; w += nthr) {
        // sign bits of coordinates 32 w .. 32 w + 31: word w mod 4 of block w / 4
        const uint4 o = philox4x32_10(make_uint4((uint32_t)(w >> 2), 0u, 0u, kTagSign), P.k0, P.k1);
        sgn[w] = pick_word(o, (uint32_t)w & 3u);
    }
    __syncthreads();
    const Twiddle<float, true> twf{tw, L, 1.f};
    const float s0 = sqrtf(1.f / (float)N), s1 = sqrtf(2.f / (float)N);
    const float *X = static_cast<const float *>(P.in);
    // Each thread holds up to kPF float4 (or 4 kPF floats) of a row: every
    // thread's part of a row is loaded at once, and the next row's part is
    // loaded while this row is transformed (N / 4 <= kPF blockDim.x by the
    // launch's choice of blockDim.x).
    constexpr int kPF = 4;
    float4 pre[kPF];
    auto load_row = [&](int64_t i) {
        if (i >= P.n) return;
        const float *xr = X + i * P.ldx;
        if (P.vec) {
#pragma unroll
            for (int u = 0; u < kPF; ++u) {
                const int e = tid + u * nthr;
                if (4 * e < N) pre[u] = __ldcs(reinterpret_cast<const float4 *>(xr) + e);
            }
        } else {
#pragma unroll
            for (int u = 0; u < kPF; ++u) {
                const int l = 4 * (tid + u * nthr);
                pre[u].x = l + 0 < N ? __ldcs(xr + l + 0) : 0.f;
                pre[u].y = l + 1 < N ? __ldcs(xr + l + 1) : 0.f;
                pre[u].z = l + 2 < N ? __ldcs(xr + l + 2) : 0.f;
                pre[u].w = l + 3 < N ? __ldcs(xr + l + 3) : 0.f;
            }
        }
    };
    load_row(blockIdx.x);
    for (int64_t i = blockIdx.x; i < P.n; i += gridDim.x) {
        // u = D x in the reordered sequence v, written as the floats of z
        float *zf = reinterpret_cast<float *>(b0);
#pragma unroll
        for (int u = 0; u < kPF; ++u) {
            const int l0 = 4 * (tid + u * nthr);
            const float xs[4] = {pre[u].x, pre[u].y, pre[u].z, pre[u].w};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int l = l0 + c;
                if (l < N) {
                    const float x = sign_neg(sgn, l) ? -xs[c] : xs[c];
                    zf[(l & 1) ? N - 1 - (l >> 1) : (l >> 1)] = x;
                }
            }
        }
        // the next row's loads fly during this row's transform; this row's
        // masks are fetched early too
        load_row(i + gridDim.x);
        int jm[4];
        if constexpr (!DENSE) {
            const int32_t *gi = P.idx + i * P.m;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int t = tid + u * nthr;
                jm[u] = t < P.m ? __ldcg(gi + t) : 0;
            }
        }
        __syncthreads();
        float2 *Z = fft(b0, b1, P, twf, tid, nthr);
        float *y = reinterpret_cast<float *>(Z == b0 ? b1 : b0);
        for (int k = tid; k <= L; k += nthr) {
            const float2 Zk = Z[k == L ? 0 : k];
            const float2 Zc = cconj(Z[k == 0 ? 0 : L - k]);
            const float2 E = make_float2(0.5f * (Zk.x + Zc.x), 0.5f * (Zk.y + Zc.y));
            // (Zk - Zc) / (2i)
            const float2 O = make_float2(0.5f * (Zk.y - Zc.y), -0.5f * (Zk.x - Zc.x));
            const float2 V = cadd(E, cmul(om[k], O));
            const float2 W = cmul(ph[k], V);
            if (k < N) y[k] = (k == 0 ? s0 : s1) * W.x;
            if (k > 0 && k < L) y[N - k] = s1 * (-W.y);
        }
        __syncthreads();
        if constexpr (DENSE) {
            float *Y = static_cast<float *>(P.out) + i * N;
            for (int k = tid; k < N; k += nthr) Y[k] = y[k];
        } else {
            const int32_t *gi = P.idx + i * P.m;
            float *ov = P.val + i * P.m;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int t = tid + u * nthr;
                if (t < P.m) ov[t] = y[clamp_index(jm[u], N)];
            }
            for (int t = tid + 4 * nthr; t < P.m; t += nthr) ov[t] = y[clamp_index(__ldcg(gi + t), N)];
        }
        __syncthreads();
    }
}

// Forward rows, one warp per row (N <= 1024): the CTA's warps share the
// twiddle and phase tables and each keeps its own two FFT buffers, so a row
// needs no block-wide barrier; a lane holds up to 8 float4 of a row and loads
// the next row's while this one is transformed.
constexpr int kWarpRowsMaxN = 1024;
constexpr int kWarpRowsWarps = 8;

template <bool DENSE>
__global__ void __launch_bounds__(kWarpRowsWarps * 32, 2) dct_forward_warp_kernel(DctParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = P.N, L = P.L;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float2 *tw = reinterpret_cast<float2 *>(smem_raw);  // L
    float2 *ph = tw + L;                                 // L + 1
    float2 *om = ph + (L + 1);                           // L + 1
    uint32_t *sgn = reinterpret_cast<uint32_t *>(om + (L + 1));  // 2 ceil(N / 64) words
    const int sgn_words = 2 * ((N + 63) / 64);
    float2 *b0 = reinterpret_cast<float2 *>(sgn + sgn_words) + (size_t)warp * 2 * L;
    float2 *b1 = b0 + L;
    for (int t = tid; t < L; t += blockDim.x) tw[t] = expipi((float)(2 * t) / (float)L, -1.f);
    for (int k = tid; k <= L; k += blockDim.x) {
        ph[k] = expipi((float)k / (float)(2 * N), -1.f);
        om[k] = expipi((float)(2 * k) / (float)N, -1.f);
    }
    for (int w = tid; w < (N + 31) / 32; w += blockDim.x) {
        const uint4 o = philox4x32_10(make_uint4((uint32_t)(w >> 2), 0u, 0u, kTagSign), P.k0, P.k1);
        sgn[w] = pick_word(o, (uint32_t)w & 3u);
    }
    __syncthreads();
    const Twiddle<float, true> twf{tw, L, 1.f};
    const float s0 = sqrtf(1.f / (float)N), s1 = sqrtf(2.f / (float)N);
    const float *X = static_cast<const float *>(P.in);
    constexpr int kPF = kWarpRowsMaxN / 4 / 32;  // float4 per lane
    float4 pre[kPF];
    auto load_row = [&](int64_t i) {
        if (i >= P.n) return;
        const float *xr = X + i * P.ldx;
#pragma unroll
        for (int u = 0; u < kPF; ++u) {
            const int e = lane + 32 * u;
            if (P.vec) {
                if (4 * e < N) pre[u] = __ldcs(reinterpret_cast<const float4 *>(xr) + e);
            } else {
                const int l = 4 * e;
                pre[u].x = l + 0 < N ? __ldcs(xr + l + 0) : 0.f;
                pre[u].y = l + 1 < N ? __ldcs(xr + l + 1) : 0.f;
                pre[u].z = l + 2 < N ? __ldcs(xr + l + 2) : 0.f;
                pre[u].w = l + 3 < N ? __ldcs(xr + l + 3) : 0.f;
            }
        }
    };
    const int64_t gw = (int64_t)blockIdx.x * kWarpRowsWarps + warp;
    const int64_t nw = (int64_t)gridDim.x * kWarpRowsWarps;
    load_row(gw);
    for (int64_t i = gw; i < P.n; i += nw) {
        float *zf = reinterpret_cast<float *>(b0);
#pragma unroll
        for (int u = 0; u < kPF; ++u) {
            const int l0 = 4 * (lane + 32 * u);
            const float xs[4] = {pre[u].x, pre[u].y, pre[u].z, pre[u].w};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int l = l0 + c;
                if (l < N) {
                    const float x = sign_neg(sgn, l) ? -xs[c] : xs[c];
                    zf[(l & 1) ? N - 1 - (l >> 1) : (l >> 1)] = x;
                }
            }
        }
        // this row's sampled coordinates (the first kMI per lane), fetched
        // before the transform so that their latency hides behind it
        constexpr int kMI = 4;
        int jv[kMI];
        if constexpr (!DENSE) {
            const int32_t *gi = P.idx + i * P.m;
#pragma unroll
            for (int u = 0; u < kMI; ++u) {
                const int t = lane + 32 * u;
                jv[u] = t < P.m ? __ldcg(gi + t) : 0;
            }
        }
        load_row(i + nw);
        __syncwarp();
        float2 *Z = fft<float2, Twiddle<float, true>, true>(b0, b1, P, twf, lane, 32);
        // coefficient k of the post-twiddle gives outputs k (its real part)
        // and N - k (its imaginary part, 0 < k < L)
        auto post = [&](int k) -> float2 {
            const float2 Zk = Z[k == L ? 0 : k];
            const float2 Zc = cconj(Z[k == 0 ? 0 : L - k]);
            const float2 E = make_float2(0.5f * (Zk.x + Zc.x), 0.5f * (Zk.y + Zc.y));
            const float2 O = make_float2(0.5f * (Zk.y - Zc.y), -0.5f * (Zk.x - Zc.x));
            const float2 V = cadd(E, cmul(om[k], O));
            return cmul(ph[k], V);
        };
        if constexpr (DENSE) {
            float *y = reinterpret_cast<float *>(Z == b0 ? b1 : b0);
            for (int k = lane; k <= L; k += 32) {
                const float2 W = post(k);
                if (k < N) y[k] = (k == 0 ? s0 : s1) * W.x;
                if (k > 0 && k < L) y[N - k] = s1 * (-W.y);
            }
            __syncwarp();
            float *Y = static_cast<float *>(P.out) + i * N;
            for (int k = lane; k < N; k += 32) Y[k] = y[k];
        } else {
            // only the m sampled outputs: output j comes from coefficient
            // j (j <= L) or N - j (j > L), the same arithmetic as the dense
            // form
            const int32_t *gi = P.idx + i * P.m;
            float *ov = P.val + i * P.m;
            auto out1 = [&](int t, int jraw) {
                const int j = clamp_index(jraw, N);
                const int k = j <= L ? j : N - j;
                const float2 W = post(k);
                ov[t] = j <= L ? (j == 0 ? s0 : s1) * W.x : s1 * (-W.y);
            };
#pragma unroll
            for (int u = 0; u < kMI; ++u) {
                const int t = lane + 32 * u;
                if (t < P.m) out1(t, jv[u]);
            }
            for (int t = lane + 32 * kMI; t < P.m; t += 32) out1(t, __ldcg(gi + t));
        }
        __syncwarp();
    }
}

// Un-mixing rows: out_i = D H^T in_i (the orthonormal DCT-III, then signs).
template <typename T>
__global__ void __launch_bounds__(512) dct_inverse_kernel(DctParams P) {
    using C2 = typename Cx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = P.N, L = P.L;
    const int tid = threadIdx.x, nthr = blockDim.x;
    C2 *b0 = reinterpret_cast<C2 *>(smem_raw);
    C2 *b1 = b0 + L;
    C2 *V = b1 + L;  // L + 1
    const Twiddle<T, false> twi{nullptr, L, (T)-1};  // inverse FFT: exp(+2 pi i t / L)
    const T s0 = sqrt((T)1 / (T)N), s1 = sqrt((T)2 / (T)N);
    const T *in = static_cast<const T *>(P.in);
    T *out = static_cast<T *>(P.out);
    for (int64_t i = blockIdx.x; i < P.n; i += gridDim.x) {
        const T *yr = in + i * N;
        // X_k = y_k / s_k; W_k = X_k - i X_{N-k} (X_N = 0); V_k = e^{i pi k / (2N)} W_k
        for (int k = tid; k <= L; k += nthr) {
            const T Xk = k < N ? yr[k] / (k == 0 ? s0 : s1) : (T)0;
            const T Xn = (k > 0) ? yr[N - k] / s1 : (T)0;
            C2 W;
            W.x = Xk;
            W.y = -Xn;
            V[k] = cmul(expipi((T)k / (T)(2 * N), (T)1), W);
        }
        __syncthreads();
        // Z_k = E_k + i O_k with E_k = (V_k + conj V_{L-k}) / 2 and
        // O_k = (V_k - conj V_{L-k}) / (2 e^{-2 pi i k / N})
        for (int k = tid; k < L; k += nthr) {
            const C2 Vk = V[k], Vc = cconj(V[L - k]);
            C2 E, D;
            E.x = (T)0.5 * (Vk.x + Vc.x);
            E.y = (T)0.5 * (Vk.y + Vc.y);
            D.x = (T)0.5 * (Vk.x - Vc.x);
            D.y = (T)0.5 * (Vk.y - Vc.y);
            const C2 O = cmul(D, expipi((T)(2 * k) / (T)N, (T)1));  // divide by e^{-2 pi i k / N}
            C2 Zk;
            Zk.x = E.x - O.y;
            Zk.y = E.y + O.x;
            b0[k] = Zk;
        }
        __syncthreads();
        C2 *z = fft(b0, b1, P, twi, tid, nthr);
        // v_q = floats of z / L; x_2l = v_l, x_{2l+1} = v_{N-1-l}; then signs
        const T *zf = reinterpret_cast<const T *>(z);
        T *xo = out + i * N;
        for (int l = tid; l < N; l += nthr) {
            const int q = (l & 1) ? N - 1 - (l >> 1) : (l >> 1);
            T x = zf[q] / (T)L;
            const uint4 o = philox4x32_10(make_uint4((uint32_t)(l >> 7), 0u, 0u, kTagSign), P.k0, P.k1);
            if ((pick_word(o, ((uint32_t)l >> 5) & 3u) >> (l & 31)) & 1u) x = -x;
            xo[l] = x;
        }
        __syncthreads();
    }
}

// Threads per row: about one per 8 of the FFT's L points (whole warps, 64 to
// 512), so that a row's N = 2L floats are at most 4 float4 per thread.
int dct_threads(int L) {
    int t = ((L + 7) / 8 + 31) / 32 * 32;
    if (t < 64) t = 64;
    if (t > 512) t = 512;
    return t;
}

DctParams make_dct(const sk_ctx &c) {
    DctParams P;
    std::memset(&P, 0, sizeof(P));
    P.N = (int)c.p;
    P.L = (int)(c.p / 2);
    P.nf = c.dct_nf;
    for (int s = 0; s < c.dct_nf; ++s) P.fac[s] = c.dct_fac[s];
    P.k0 = (uint32_t)c.seed;
    P.k1 = (uint32_t)(c.seed >> 32);
    P.m = (int)c.m;
    return P;
}

template <typename K>
cudaError_t launch_rows(K kern, const DctParams &P, size_t smem, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int threads = dct_threads(P.L);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (int64_t)sms * per_sm;
    if (blocks > P.n) blocks = P.n;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, threads, smem, s>>>(P);
    return cudaGetLastError();
}

}  // namespace

// The radices of L = p / 2 in stage order (8, 4, 2 first, then odd primes up
// to 13); false if L has a prime factor above 13.
// Shared-memory wavefronts of the warp kernel's FFT stages in the order
// fac[0..nf) (a cost model, no launch): a warp's threads take butterflies
// j = lane, lane + 32, ...; each load in[j + r S], twiddle tw(k r st) and
// store out[(j / Ns) Ns R + k + q Ns] moves 8 bytes a lane, served a
// half-warp at a time, each half-warp taking as many wavefronts as the most
// distinct 4-byte words any one of the 32 banks holds.
static int64_t dct_stage_cost(int64_t L, const int *fac, int nf) {
    auto wavefronts = [](const int64_t *e, int cnt) -> int64_t {
        // e: 8-byte element indices of the active lanes of one half-warp
        if (cnt == 0) return 0;
        int64_t words[32];
        int nw = 0;
        for (int i = 0; i < cnt; ++i)
            for (int h = 0; h < 2; ++h) {
                const int64_t w = 2 * e[i] + h;
                bool seen = false;
                for (int q = 0; q < nw; ++q) seen = seen || words[q] == w;
                if (!seen) words[nw++] = w;
            }
        int per_bank[32] = {0};
        int most = 0;
        for (int q = 0; q < nw; ++q) {
            const int b = (int)(words[q] & 31);
            if (++per_bank[b] > most) most = per_bank[b];
        }
        return most;
    };
    int64_t cost = 0, Ns = 1;
    for (int s = 0; s < nf; ++s) {
        const int64_t R = fac[s], S = L / R, st = L / (Ns * R);
        for (int64_t t0 = 0; t0 < S; t0 += 32)
            for (int64_t r = 0; r < R; ++r)
                for (int kind = 0; kind < 3; ++kind) {
                    if (kind == 2 && (Ns == 1 || r == 0)) continue;  // no twiddle
                    for (int half = 0; half < 2; ++half) {
                        int64_t e[16];
                        int cnt = 0;
                        for (int64_t j = t0 + 16 * half; j < t0 + 16 * half + 16 && j < S; ++j) {
                            const int64_t jq = j / Ns, k = j - jq * Ns;
                            e[cnt++] = kind == 0 ? j + r * S
                                     : kind == 1 ? jq * Ns * R + k + r * Ns
                                                 : (k * r * st) % L;
                        }
                        cost += wavefronts(e, cnt);
                    }
                }
        Ns *= R;
    }
    return cost;
}

bool dct_factor(int64_t L, int *fac, int *nf) {
    int k = 0;
    while (L > 1 && L % 8 == 0 && k < 16) {
        fac[k++] = 8;
        L /= 8;
    }
    while (L > 1 && L % 4 == 0 && k < 16) {
        fac[k++] = 4;
        L /= 4;
    }
    while (L > 1 && L % 2 == 0 && k < 16) {
        fac[k++] = 2;
        L /= 2;
    }
    const int64_t L0 = [&] {
        int64_t v = L;
        for (int q = 0; q < k; ++q) v *= fac[q];
        return v;
    }();
    for (int r : {3, 5, 7, 11, 13})
        while (L > 1 && L % r == 0 && k < 16) {
            fac[k++] = r;
            L /= r;
        }
    *nf = k;
    if (L != 1) return false;
    // Stage order: any order gives the same transform (up to rounding); the
    // one the cost model above rates cheapest is kept (ties: the first
    // met).  Candidates: every distinct order of up to six stages, else the
    // radices-2^k-first order and that order with each distinct radix moved
    // to the front.  (L = 392 = 8 7 7: a first radix-8 stage stores at a
    // stride of 8 elements, 16 lanes into 2 banks; radix 7 first stores at
    // an odd stride, one wavefront per half-warp.)
    int best[16];
    for (int q = 0; q < k; ++q) best[q] = fac[q];
    int64_t best_cost = dct_stage_cost(L0, best, k);
    auto consider = [&](const int *cand) {
        const int64_t c = dct_stage_cost(L0, cand, k);
        if (c < best_cost) {
            best_cost = c;
            for (int q = 0; q < k; ++q) best[q] = cand[q];
        }
    };
    if (k <= 6) {
        int cand[16];
        for (int q = 0; q < k; ++q) cand[q] = fac[q];
        std::sort(cand, cand + k);
        do consider(cand);
        while (std::next_permutation(cand, cand + k));
    } else {
        for (int q = 1; q < k; ++q) {
            if (fac[q] == fac[q - 1]) continue;
            int cand[16];
            cand[0] = fac[q];
            int w = 1;
            for (int u = 0; u < k; ++u)
                if (u != q) cand[w++] = fac[u];
            consider(cand);
        }
    }
    for (int q = 0; q < k; ++q) fac[q] = best[q];
    return true;
}

size_t dct_forward_smem(const sk_ctx &c) {
    const size_t L = (size_t)(c.p / 2);
    return (L + 2 * (L + 1) + 2 * L) * sizeof(float2) + ((size_t)c.p + 31) / 32 * 4;
}

cudaError_t launch_dct_forward(const sk_ctx &c, const float *X, int64_t n, int64_t ldx,
                               const int32_t *idx, float *val, float *Y, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    DctParams P = make_dct(c);
    P.in = X;
    P.n = n;
    P.ldx = ldx;
    P.vec = ((reinterpret_cast<uintptr_t>(X) & 15) == 0) && (c.p % 4 == 0) && (ldx % 4 == 0);
    P.idx = idx;
    P.val = val;
    P.out = Y;
    if (c.p <= kWarpRowsMaxN) {
        // a warp per row: per CTA the shared tables, per warp two buffers
        const size_t L = (size_t)P.L;
        const size_t smem = (3 * L + 2) * sizeof(float2) + 2 * (((size_t)c.p + 63) / 64) * 4 +
                            (size_t)kWarpRowsWarps * 2 * L * sizeof(float2);
        auto kern = Y ? dct_forward_warp_kernel<true> : dct_forward_warp_kernel<false>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWarpRowsWarps * 32, smem);
        if (per_sm < 1) per_sm = 1;
        int64_t blocks = (int64_t)sms * per_sm;
        const int64_t need = (n + kWarpRowsWarps - 1) / kWarpRowsWarps;
        if (blocks > need) blocks = need;
        kern<<<(unsigned)blocks, kWarpRowsWarps * 32, smem, s>>>(P);
        return cudaGetLastError();
    }
    const size_t smem = dct_forward_smem(c);
    return Y ? launch_rows(dct_forward_kernel<true>, P, smem, s)
             : launch_rows(dct_forward_kernel<false>, P, smem, s);
}

cudaError_t launch_dct_inverse(const sk_ctx &c, const void *in, int64_t r, void *out, bool f64,
                               cudaStream_t s) {
    if (r == 0) return cudaSuccess;
    DctParams P = make_dct(c);
    P.in = in;
    P.n = r;
    P.out = out;
    const size_t L = (size_t)P.L;
    const size_t smem = (3 * L + 1) * (f64 ? sizeof(double2) : sizeof(float2));
    return f64 ? launch_rows(dct_inverse_kernel<double>, P, smem, s)
               : launch_rows(dct_inverse_kernel<float>, P, smem, s);
}

}  // namespace sk
