// unmix.cu -- un-mixing mu = (HD)^T mu' = D H mu' (Eq. (mu-mu'); Algorithm 1,
// last line).  Sylvester H is symmetric, so (HD)^T = D H.  One CTA per row:
// the row sits in shared memory, log2(pt) butterfly stages, then the signs and
// the 1/sqrt(pt) scale, truncated to the first p coordinates.  Only K centres
// or k eigenvectors pass through here, so the kernel is kept simple.
#include "sk_internal.cuh"

namespace sk {
namespace {

template <typename T>
__global__ void unmix_kernel(const T *in, int64_t r, int pt, int p, uint32_t k0,
                             uint32_t k1, T scale, int mix, T *out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *y = reinterpret_cast<T *>(smem_raw);
    for (int64_t row = blockIdx.x; row < r; row += gridDim.x) {
        for (int j = threadIdx.x; j < pt; j += blockDim.x) y[j] = in[row * pt + j];
        __syncthreads();
        for (int h = 1; h < (mix ? pt : 1); h <<= 1) {
            for (int q = threadIdx.x; q < pt / 2; q += blockDim.x) {
                const int lo = (q / h) * 2 * h + (q % h);
                const T a = y[lo], b = y[lo + h];
                y[lo] = a + b;
                y[lo + h] = a - b;
            }
            __syncthreads();
        }
        for (int j = threadIdx.x; j < p; j += blockDim.x) {
            const T v = y[j] * scale;
            out[row * p + j] = (mix && sign_bit(k0, k1, (uint32_t)j)) ? -v : v;
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_unmix(const sk_ctx &c, const void *in, int64_t r, void *out, bool f64,
                         cudaStream_t s) {
    if (r == 0) return cudaSuccess;
    // the DCT preconditioner: D H^T with H^T the orthonormal DCT-III (dct.cu)
    if (c.flags & SK_FLAG_DCT) return launch_dct_inverse(c, in, r, out, f64, s);
    const int threads = c.pt >= 512 ? 512 : (c.pt >= 32 ? (int)c.pt : 32);
    int blocks = (int)(r < 1024 ? r : 1024);
    const uint32_t k0 = (uint32_t)c.seed, k1 = (uint32_t)(c.seed >> 32);
    // without preconditioning (H = D = I) un-mixing is the truncation to p
    const int mix = (c.flags & SK_FLAG_NO_PRECONDITION) ? 0 : 1;
    const double sc = mix ? 1.0 / sqrt((double)c.pt) : 1.0;
    if (f64) {
        const size_t smem = (size_t)c.pt * 8;
        cudaError_t e = cudaFuncSetAttribute(unmix_kernel<double>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        unmix_kernel<double><<<blocks, threads, smem, s>>>(
            static_cast<const double *>(in), r, (int)c.pt, (int)c.p, k0, k1, sc, mix,
            static_cast<double *>(out));
    } else {
        const size_t smem = (size_t)c.pt * 4;
        unmix_kernel<float><<<blocks, threads, smem, s>>>(
            static_cast<const float *>(in), r, (int)c.pt, (int)c.p, k0, k1, (float)sc, mix,
            static_cast<float *>(out));
    }
    return cudaGetLastError();
}

}  // namespace sk
