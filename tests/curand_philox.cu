// Test helper: Philox4x32-10 blocks from cuRAND's device generator
// (curandStatePhilox4_32_10_t), used as a library to pin the oracle's own
// Philox.  Not part of the product; tests/test_gpu_philox.py builds and loads
// it.
//
// Mapping of a block at counter (c0, c1, c2, c3) under key (k0, k1) onto the
// cuRAND device API, as that API documents it: curand_init's seed is the key
// (k0 low word, k1 high word), its subsequence is the counter's high 64 bits
// (c2 low, c3 high), and the position within a subsequence counts 32-bit
// outputs, four per block, so the block with low counter bits c0 | c1 << 32
// starts 4 (c0 | c1 << 32) outputs in.  The skip is taken as four skipahead
// calls of (c0 | c1 << 32) outputs each, which stays within 64 bits for any
// counter.  curand4 then returns the block's four words.
#include <cstdint>
#include <cuda_runtime.h>
#include <curand_kernel.h>

namespace {
__global__ void k_blocks(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long seed = (unsigned long long)key[2 * i] | ((unsigned long long)key[2 * i + 1] << 32);
    unsigned long long sub = (unsigned long long)ctr[4 * i + 2] | ((unsigned long long)ctr[4 * i + 3] << 32);
    unsigned long long lo = (unsigned long long)ctr[4 * i] | ((unsigned long long)ctr[4 * i + 1] << 32);
    curandStatePhilox4_32_10_t st;
    curand_init(seed, sub, 0ull, &st);
    for (int r = 0; r < 4; ++r) skipahead(lo, &st);
    uint4 v = curand4(&st);
    out[4 * i] = v.x;
    out[4 * i + 1] = v.y;
    out[4 * i + 2] = v.z;
    out[4 * i + 3] = v.w;
}
}  // namespace

// ctr: 4n words, key: 2n words, out: 4n words, all host memory.  Returns the
// CUDA error code (0 on success).
extern "C" int curand_philox_blocks(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n)
{
    if (n <= 0) return 0;
    uint32_t *dc = nullptr, *dk = nullptr, *dout = nullptr;
    cudaError_t e = cudaMalloc(&dc, 16ull * n);
    if (e == cudaSuccess) e = cudaMalloc(&dk, 8ull * n);
    if (e == cudaSuccess) e = cudaMalloc(&dout, 16ull * n);
    if (e == cudaSuccess) e = cudaMemcpy(dc, ctr, 16ull * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dk, key, 8ull * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_blocks<<<(n + 127) / 128, 128>>>(dc, dk, dout, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, 16ull * n, cudaMemcpyDeviceToHost);
    cudaFree(dc);
    cudaFree(dk);
    cudaFree(dout);
    return (int)e;
}
