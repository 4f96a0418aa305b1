// Test fixture (compiled by tests/test_gpu_newton.py): evaluates the
// library's Newton-Raphson float64 reciprocal square root and reciprocal on
// an array of caller-owned device values.
#include "../../paper_1511_00152_gb300/csrc/sk_internal.cuh"

__global__ void newton_eval_kernel(const double *x, int n, double *rs, double *rc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        rc[i] = sk::rcp_nr(x[i]);
        rs[i] = x[i] > 0.0 ? sk::rsqrt_nr(x[i]) : 0.0;
    }
}

extern "C" int newton_eval(const double *x, int n, double *rs, double *rc) {
    if (n <= 0) return 0;
    newton_eval_kernel<<<(n + 255) / 256, 256>>>(x, n, rs, rc);
    return (int)cudaDeviceSynchronize();
}
