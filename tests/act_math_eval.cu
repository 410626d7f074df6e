// Test harness: the surrogate epilogue's SiLU forms (act_math.cuh) and CUDA's
// expf-based SiLU on the same inputs h (z = 2 h), for tests/test_gpu_act_math.py.
#include <cstdint>
#include <cuda_runtime.h>

#include "../paper_2206_02937_gb300/csrc/act_math.cuh"

namespace {
__global__ void k_eval(const float* h, int64_t n, float* out_fma, float* out_mufu, float* out_expf)
{
    using namespace compton::act;
    const int64_t i = 2 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    if (i >= n) return;
    const float h0 = h[i], h1 = i + 1 < n ? h[i + 1] : 0.0f;
    const uint64_t hp = pk2(h0, h1);
    float a0, a1, b0, b1;
    upk2(silu2_fma(hp), a0, a1);
    upk2(silu2_mufu(hp), b0, b1);
    out_fma[i] = a0;
    out_mufu[i] = b0;
    out_expf[i] = 2.0f * h0 / (1.0f + expf(-2.0f * h0));
    if (i + 1 < n) {
        out_fma[i + 1] = a1;
        out_mufu[i + 1] = b1;
        out_expf[i + 1] = 2.0f * h1 / (1.0f + expf(-2.0f * h1));
    }
}
}  // namespace

extern "C" int act_math_eval(const float* h_host, int64_t n, float* fma_host, float* mufu_host, float* expf_host)
{
    float* d = nullptr;
    const size_t b = (size_t)n * sizeof(float);
    if (cudaMalloc(&d, 4 * b) != cudaSuccess) return 1;
    int rc = 0;
    if (cudaMemcpy(d, h_host, b, cudaMemcpyHostToDevice) != cudaSuccess) rc = 2;
    if (!rc && n > 0) {
        const int64_t pairs = (n + 1) / 2;
        k_eval<<<(unsigned)((pairs + 255) / 256), 256>>>(d, n, d + n, d + 2 * n, d + 3 * n);
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) rc = 3;
    }
    if (!rc && (cudaMemcpy(fma_host, d + n, b, cudaMemcpyDeviceToHost) != cudaSuccess ||
                cudaMemcpy(mufu_host, d + 2 * n, b, cudaMemcpyDeviceToHost) != cudaSuccess ||
                cudaMemcpy(expf_host, d + 3 * n, b, cudaMemcpyDeviceToHost) != cudaSuccess))
        rc = 4;
    cudaFree(d);
    return rc;
}
