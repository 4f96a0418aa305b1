// Test harness (compiled by tests/test_gpu_newton.py): evaluates the
// library's Newton-Raphson float64 reciprocal square root and reciprocal on
// an array of caller-owned device values.
#include "../../paper_1511_00152_gb300/csrc/sk_internal.cuh"

__global__ void nr_probe_kernel(const double *x, int n, double *rs, double *rc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        rc[i] = sk::rcp_nr(x[i]);
        rs[i] = x[i] > 0.0 ? sk::rsqrt_nr(x[i]) : 0.0;
    }
}

extern "C" int nr_probe(const double *x, int n, double *rs, double *rc) {
    if (n <= 0) return 0;
    nr_probe_kernel<<<(n + 255) / 256, 256>>>(x, n, rs, rc);
    return (int)cudaDeviceSynchronize();
}
