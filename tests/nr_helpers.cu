// Test helper: evaluates the library's FP64 Newton-Raphson helpers (rcp_nr,
// rsqrt_nr, sqrt_nr of device_math.cuh) and CUDA's own correctly rounded
// FP64 reciprocal and square root on the same inputs, for
// tests/test_gpu_nr_helpers.py.  Not part of the product.
#include <cstdint>
#include <cuda_runtime.h>

#include "../paper_2206_02937_gb300/csrc/device_math.cuh"

namespace {
__global__ void k_eval(const double* d, int64_t n, double* out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = d[i];
    out[6 * i + 0] = compton::rcp_nr(x);
    out[6 * i + 1] = __drcp_rn(x);
    out[6 * i + 2] = x > 0.0 ? compton::rsqrt_nr(x) : 0.0;
    out[6 * i + 3] = x > 0.0 ? __drcp_rn(__dsqrt_rn(x)) : 0.0;
    out[6 * i + 4] = x >= 0.0 ? compton::sqrt_nr(x) : 0.0;
    out[6 * i + 5] = x >= 0.0 ? __dsqrt_rn(x) : 0.0;
}
}  // namespace

// d: n doubles (host); out: 6n doubles (host).  Returns the CUDA error code.
extern "C" int nr_helpers_eval(const double* d, int64_t n, double* out)
{
    if (n <= 0) return 0;
    double *dd = nullptr, *dout = nullptr;
    cudaError_t e = cudaMalloc(&dd, 8 * n);
    if (e == cudaSuccess) e = cudaMalloc(&dout, 48 * n);
    if (e == cudaSuccess) e = cudaMemcpy(dd, d, 8 * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_eval<<<(unsigned)((n + 255) / 256), 256>>>(dd, n, dout);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, 48 * n, cudaMemcpyDeviceToHost);
    cudaFree(dd);
    cudaFree(dout);
    return (int)e;
}
