// gram_tc.cu -- tensor-core (tcgen05) Gram for the covariance estimator.
#include "sk_internal.cuh"

namespace sk {

__device__ unsigned int g_device_error = 0u;

cudaError_t take_device_error(unsigned int *flag) {
    unsigned int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(flag, g_device_error, sizeof(*flag));
    if (e != cudaSuccess) return e;
    if (*flag) e = cudaMemcpyToSymbol(g_device_error, &zero, sizeof(zero));
    return e;
}

cudaError_t launch_gram_tc(const sk_ctx &, int, const int32_t *, const float *, int64_t,
                           double *, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace sk
