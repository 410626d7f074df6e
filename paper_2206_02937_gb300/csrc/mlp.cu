// mlp.cu -- the surrogate network that replaces the probability calculation
// (arXiv 2206.02937, Sec. 2: a network object loaded once and run on any batch
// of inputs; Sec. 3.2: inputs are the lepton and photon momenta in units of
// m_e c, fully connected layers, sigmoid output y' in [0, 1]).
//
// Network: 6 inputs -> 4 hidden layers of 64 SiLU units -> 1 sigmoid output,
// predicting r = sigma_KN v / (2 sigma_T), the probability normalised by the
// cell maximum P_max = 2 sigma_T c dt max w of Sec. 3.2.  Inputs are
// f = [sgnlog(u/s_u)/n_u, sgnlog(k/s_k)/n_k] with sgnlog(z) = sign(z) ln(1+|z|).
//
// Kernels:
//   k_mlp_pack   FP32 parameter vector -> BF16 weight tiles in the 128-byte
//                swizzled K-major layout the tensor core reads (layer 0's six
//                inputs zero-padded to K = 64), FP8 E4M3 tiles (K padded to 128)
//                with per-tensor scales, transposed FP32 copies for the CUDA
//                core path, biases and the output layer.
//   k_mlp_bf16   tcgen05 forward: 128 samples per tile, one row per thread;
//                per hidden layer four 128x64x16 BF16 MMAs into a 64-column
//                FP32 TMEM accumulator, then bias + SiLU in registers and the
//                BF16 activations written back to shared memory as the next
//                layer's A operand; the 64 -> 1 output layer on the CUDA cores.
//   k_mlp_fp8    the same with E4M3 operands (kind::f8f6f4, K = 32 per MMA)
//                and per-tensor scales, FP32 accumulation.
//   k_mlp_fp32   FP32 forward on the CUDA cores (reference precision).
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "act_math.cuh"
#include "ctx.hpp"
#include "device_math.cuh"
#include "features.cuh"
#include "tc_ptx.cuh"

namespace compton {

namespace {

// Eight row groups (warpgroups) per CTA, one CTA per SM: each group its own
// 128-row tile, A buffer, 64 TMEM columns and mbarrier, all sharing one copy
// of the weights; 32 warps per SM at 64 registers hide the per-layer chain
// (MMA, TMEM read, SiLU, A store, group barrier) best among the measured
// shapes (2 groups x 3 CTAs 1.48 ms, 4 x 2 1.44, 6 x 1 1.34, 8 x 1 1.31 ms
// for 16.8M samples in BF16).
constexpr int kMlpGroups = 8;
constexpr int kMlpMinCtas = 1;  // CTAs per SM the registers are budgeted for
constexpr int kMlpThreads = 128 * kMlpGroups;
constexpr uint32_t kMlpTmemCols = kMlpGroups <= 2 ? 128 : (kMlpGroups <= 4 ? 256 : 512);  // 64 per group, a power of 2
constexpr int kTileM = 128;
// shared-memory layout of the tensor-core kernels (base aligned to 1024 B)
constexpr uint32_t kOffW = 0;                           // 4 weight tiles
constexpr uint32_t kWTileBytes = 8192;                  // 64 rows x 128 B
constexpr uint32_t kOffA = kOffW + 4 * kWTileBytes;     // A tiles (128 x 128 B each, one per group)
constexpr uint32_t kOffRaw = kOffA + 16384 * kMlpGroups;  // next tile's momenta per group, [6][128] floats
constexpr uint32_t kOffBB = kOffRaw + 6 * kTileM * 4 * kMlpGroups;  // BF16: half-bias blocks of layers 1-3
constexpr uint32_t kOffOnes = kOffBB + 3 * 2048;        // BF16: A block of the bias step (1, 1 in K 0, 1)
constexpr uint32_t kOffBias = kOffOnes + 4096;          // 4 x 64 floats (FP8: half biases)
constexpr uint32_t kOffW4 = kOffBias + 1024;            // 64 floats
constexpr uint32_t kOffScale = kOffW4 + 256;            // 8 floats
constexpr uint32_t kOffBar = kOffScale + 32;            // one mbarrier per group
constexpr uint32_t kOffSlot = kOffBar + 8 * kMlpGroups;  // TMEM address
constexpr uint32_t kSmemTc = kOffSlot + 8 + 1024;       // + alignment slack

constexpr uint64_t kWaitNs = 2000000000ull;             // 2 s bound on every wait
// Of each 32 activations of a BF16 layer a thread finishes, the first
// 2 * kSiluFmaPairs take SiLU on the FMA pipe (act::silu2_fma), the others
// tanh on the multi-function unit (act::silu2_mufu), whose instructions share
// the MIO queue with the shared-memory traffic (the kernel's top stall).
// Measured (16.8M samples, BF16): 0, 1, 2 and 4 pairs of 16: 1.217, 1.163,
// 1.170 and 1.265 ms; FP8 was fastest with none.
constexpr int kSiluFmaPairs = 1;
// BF16 on k_mlp_ta (the A operand in tensor memory) instead of k_mlp_tc<false>.
constexpr bool kBf16TmemA = true;

__device__ __forceinline__ float silu_exact(float z) { return z / (1.0f + expf(-z)); }
__device__ __forceinline__ float sigmoid_exact(float z) { return 1.0f / (1.0f + expf(-z)); }

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ uint32_t pack_e4m3x4(float a, float b, float c, float d)
{
    const __nv_fp8x2_storage_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
    const __nv_fp8x2_storage_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
    return (uint32_t)lo | ((uint32_t)hi << 16);
}

// ---------------------------------------------------------------------------
// Packing.  theta layout (float, 12993): W0 (64x6), b0, W1 (64x64), b1, W2, b2,
// W3, b3, W4 (1x64), b4; W stored (out, in) row-major.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float theta_w(const float* th, int l, int n, int k)
{
    if (l == 0) return k < 6 ? th[n * 6 + k] : 0.0f;
    return th[mlp_off_w(l) + n * 64 + k];
}

__global__ void k_mlp_pack(MlpDev m)
{
    const float* th = m.theta;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    // BF16 tiles: 4 x 64 x 64
    if (i < 4 * 64 * 64) {
        const int l = i / 4096, n = (i / 64) % 64, k = i % 64;
        uint8_t* base = reinterpret_cast<uint8_t*>(m.wbf16) + l * kWTileBytes;
        const __nv_bfloat16 v = __float2bfloat16_rn(theta_w(th, l, n, k));
        *reinterpret_cast<__nv_bfloat16*>(base + tc::sw128_offset(n, k >> 3) + (k & 7) * 2) = v;
        // transposed FP32 copy for the CUDA-core path: wt[l][k][n]
        m.wt32[l * 4096 + k * 64 + n] = theta_w(th, l, n, k);
        // inference image: W / 2 (exact), and in layer 0's padding columns
        // 6, 7 the half bias as hi + lo (the A rows carry 1, 1 there)
        uint8_t* hbase = reinterpret_cast<uint8_t*>(m.whalf) + l * kWTileBytes;
        float hv = 0.5f * theta_w(th, l, n, k);
        if (l == 0 && (k == 6 || k == 7)) {
            const float hb = 0.5f * th[mlp_off_b(0) + n];
            const float hi = __bfloat162float(__float2bfloat16_rn(hb));
            hv = k == 6 ? hi : hb - hi;
        }
        *reinterpret_cast<__nv_bfloat16*>(hbase + tc::sw128_offset(n, k >> 3) + (k & 7) * 2) =
            __float2bfloat16_rn(hv);
    }
    // half-bias blocks of layers 1-3: row n, K columns 0 (hi) and 1 (lo), zeros to 15
    if (i < 3 * 64 * 16) {
        const int l = 1 + i / 1024, n = (i / 16) % 64, k = i % 16;
        uint8_t* bb = reinterpret_cast<uint8_t*>(m.whalf) + 4 * kWTileBytes + (l - 1) * 2048;
        const float hb = 0.5f * th[mlp_off_b(l) + n];
        const float hi = __bfloat162float(__float2bfloat16_rn(hb));
        const float v = k == 0 ? hi : (k == 1 ? hb - hi : 0.0f);
        *reinterpret_cast<__nv_bfloat16*>(bb + tc::sw32_offset(n, k >> 3) + (k & 7) * 2) = __float2bfloat16_rn(v);
    }
    // FP8 tiles: 4 x 64 rows x 128 B (K = 64 real + 64 zero)
    if (i < 4 * 64 * 128) {
        const int l = i / 8192, n = (i / 128) % 64, k = i % 128;
        uint8_t* base = reinterpret_cast<uint8_t*>(m.wfp8) + l * kWTileBytes;
        const float w = k < 64 ? theta_w(th, l, n, k) * m.scale_w_inv[l] : 0.0f;
        base[tc::sw128_offset(n, k >> 4) + (k & 15)] = __nv_cvt_float_to_fp8(w, __NV_SATFINITE, __NV_E4M3);
    }
    if (i < 4 * 64) {
        const int l = i / 64, n = i % 64;
        m.bias[i] = th[mlp_off_b(l) + n];
    }
    if (i < 64) m.w4[i] = th[mlp_off_w(4) + i];
    if (i == 0) m.b4[0] = th[mlp_off_b(4)];
}

// Per-tensor amax of each layer's weights (for the FP8 scales): one block per layer.
__global__ void k_mlp_weight_amax(MlpDev m)
{
    __shared__ float red[32];
    const int l = blockIdx.x;
    const int n_el = l == 0 ? 64 * 6 : 64 * 64;
    const float* w = m.theta + mlp_off_w(l);
    float a = 0.0f;
    for (int i = threadIdx.x; i < n_el; i += blockDim.x) a = fmaxf(a, fabsf(w[i]));
    for (int d = 16; d > 0; d >>= 1) a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, d));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = fmaxf(t, red[i]);
        const float s = t > 0.0f ? t / 448.0f : 1.0f;  // 448 = largest finite E4M3
        m.scale_w[l] = s;
        m.scale_w_inv[l] = 1.0f / s;
    }
}

// ---------------------------------------------------------------------------
// Tensor-core forward (BF16 or FP8 operands).  kFp8 selects the operand type.
// ---------------------------------------------------------------------------
struct MlpArgs {
    MlpDev m;
    const float* u[3];
    const float* k[3];
    int64_t n;
    float* r_out;
    DeviceStats* stats;
    // binned input (pairs of a compton_bin_pairs list) when cinfo != nullptr
    const CellInfo* cinfo;
    const int32_t* tile_cell;
    const int64_t* n_pairs;
    // candidate input (rows of the candidate list) when cand != nullptr
    const CandPair* cand;
    const uint32_t* n_cand;
    // decide: P and the Bernoulli trial of every candidate row in the
    // epilogue, accepted pairs appended to the list (r_out unused)
    bool decide;
    MlpDecide dec;
    AcceptedPair* accepted;
    uint32_t* n_accepted;
};

// Probability and decision of candidate row `row` from its network output
// (pre-sigmoid z) and the momenta of its record: P = 1 - exp(-2 n dt r) inside the network's
// training range (compton_mlp_set_range; by default gamma <= 1e3, eps in
// [1e-4, 1]), else the analytic
// probability (counted); accepted rows go to the list with their momenta.
// Called by every thread of a warp.
__device__ __forceinline__ void decide_row(const MlpArgs& a, int64_t row, bool live, float z)
{
    const unsigned lane = threadIdx.x & 31u;
    bool hit = false, fb = false;
    float x = -1.0f;
    CandPair c{};
    if (live) {
        c = a.cand[row];
        const float r = __fdividef(1.0f, 1.0f + __expf(-z));
        const float g2 = fmaf(c.u[0], c.u[0], fmaf(c.u[1], c.u[1], fmaf(c.u[2], c.u[2], 1.0f)));
        const float e2 = fmaf(c.k[0], c.k[0], fmaf(c.k[1], c.k[1], c.k[2] * c.k[2]));
        float P;
        if (mlp_in_range(a.m, g2, e2)) {
            P = one_minus_exp_neg(2.0f * c.dens * a.dec.dt * r);
        } else {
            fb = true;
            P = analytic_prob(c.u[0], c.u[1], c.u[2], c.k[0], c.k[1], c.k[2], c.dens, a.dec.dt, a.dec.gamma64, &x);
        }
        hit = c.u0 < P;
        if (a.dec.prob_out) a.dec.prob_out[c.p] = P;
        if (a.dec.flag_out) a.dec.flag_out[c.p] = hit ? 1 : 0;
    }
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    const unsigned mf = __ballot_sync(0xffffffffu, fb);
    if (m) {
        uint32_t at = 0;
        if (lane == 0) at = atomicAdd(a.n_accepted, (uint32_t)__popc(m));
        at = __shfl_sync(0xffffffffu, at, 0);
        if (hit)
            a.accepted[at + __popc(m & ((1u << lane) - 1u))] =
                AcceptedPair{c.ie, c.ig, x, c.p, {c.u[0], c.u[1], c.u[2]}, {c.k[0], c.k[1], c.k[2]}, {0u, 0u}};
    }
    if (lane == 0) {
        if (m) atomicAdd(&a.stats->scatters, (unsigned long long)__popc(m));
        if (mf) atomicAdd(&a.stats->mlp_fallbacks, (unsigned long long)__popc(mf));
    }
}

// Electron and photon index of pair p of a binned pair list: the cell is
// found by binary search between the cells of p's 1024-pair scatter tile.
__device__ __forceinline__ void binned_pair(const MlpArgs& a, int64_t p, int& ie, int& ig)
{
    const int64_t t = p / kPairsPerTile;
    int lo = a.tile_cell[t], hi = a.tile_cell[t + 1];
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((int64_t)a.cinfo[mid].pair_off <= p) lo = mid; else hi = mid - 1;
    }
    const CellInfo ci = a.cinfo[lo];
    const int j = (int)(p - ci.pair_off);
    ie = ci.e_start + j;
    ig = ci.g_start + j;
}

// Raw momenta of pair `row` (electron u, photon k), zeros past the end.
__device__ __forceinline__ void load_pair_raw(const MlpArgs& a, int64_t row, int64_t n_rows, float* q)
{
    if (row >= n_rows) {
#pragma unroll
        for (int i = 0; i < 6; ++i) q[i] = 0.0f;
        return;
    }
    if (a.cand) {
        const CandPair& c = a.cand[row];
        q[0] = c.u[0];
        q[1] = c.u[1];
        q[2] = c.u[2];
        q[3] = c.k[0];
        q[4] = c.k[1];
        q[5] = c.k[2];
        return;
    }
    int ie = (int)row, ig = (int)row;
    if (a.cinfo) binned_pair(a, row, ie, ig);
    q[0] = a.u[0][ie];
    q[1] = a.u[1][ie];
    q[2] = a.u[2][ie];
    q[3] = a.k[0][ig];
    q[4] = a.k[1][ig];
    q[5] = a.k[2][ig];
}

__device__ __forceinline__ void load_pair_features(const MlpArgs& a, int64_t row, float* f)
{
    float q[6];
    load_pair_raw(a, row, row + 1, q);
    features(a.m, q[0], q[1], q[2], q[3], q[4], q[5], f);
}

// Asynchronous copy of pair `row`'s momenta (electron u, photon k) into the
// staging column st[0], st[128], ..., st[640]; nothing past the end.
__device__ __forceinline__ void stage_pair_raw(const MlpArgs& a, int64_t row, int64_t n_rows, float* st)
{
    if (row >= n_rows) return;
    const float* src[6];
    if (a.cand) {
        const CandPair* c = a.cand + row;
        src[0] = &c->u[0];
        src[1] = &c->u[1];
        src[2] = &c->u[2];
        src[3] = &c->k[0];
        src[4] = &c->k[1];
        src[5] = &c->k[2];
    } else {
        int ie = (int)row, ig = (int)row;
        if (a.cinfo) binned_pair(a, row, ie, ig);
        src[0] = a.u[0] + ie;
        src[1] = a.u[1] + ie;
        src[2] = a.u[2] + ie;
        src[3] = a.k[0] + ig;
        src[4] = a.k[1] + ig;
        src[5] = a.k[2] + ig;
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const uint32_t d = tc::smem_u32(st + i * kTileM);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src[i]) : "memory");
    }
}

// Barrier of the 128 threads of row group g (named barrier 1 + g), and the
// same with an OR over their flags.
__device__ __forceinline__ void group_sync(int g) { asm volatile("bar.sync %0, 128;" ::"r"(1 + g) : "memory"); }
__device__ __forceinline__ bool group_sync_or(int g, bool flag)
{
    uint32_t out;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, %2, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(out)
        : "r"((uint32_t)flag), "r"(1 + g)
        : "memory");
    return out != 0;
}

template <bool kFp8>
__global__ void __launch_bounds__(kMlpThreads, kMlpMinCtas) k_mlp_tc(MlpArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* Wt = sm + kOffW;
    const int tid = threadIdx.x;
    const int g = tid >> 7;     // row group: its own tile, A buffer, TMEM columns and mbarrier
    const int lt = tid & 127;   // row within the group's tile
    uint8_t* Ah = sm + kOffA + g * 16384;
    float* st = reinterpret_cast<float*>(sm + kOffRaw) + g * 6 * kTileM + lt;  // this row's staged momenta
    float* hbias = reinterpret_cast<float*>(sm + kOffBias);  // half the biases
    float* w4 = reinterpret_cast<float*>(sm + kOffW4);
    float* scale = reinterpret_cast<float*>(sm + kOffScale);  // [0..3] w scales, [4..7] 1/activation scales
    uint64_t* bar0 = reinterpret_cast<uint64_t*>(sm + kOffBar);
    uint64_t* bar = bar0 + g;
    uint32_t* slot = reinterpret_cast<uint32_t*>(sm + kOffSlot);

    const int warp = tid >> 5;
    const MlpDev& m = a.m;
    // BF16: the half-weight image with its half-bias blocks (the bias enters
    // the MMA as one more K step against a block of ones, and the
    // accumulator is h = z / 2 directly); FP8: weights, biases in the epilogue
    const uint4* wsrc = reinterpret_cast<const uint4*>(kFp8 ? m.wfp8 : m.whalf);
    for (int i = tid; i < (int)(4 * kWTileBytes / 16); i += kMlpThreads) reinterpret_cast<uint4*>(Wt)[i] = wsrc[i];
    if (!kFp8) {
        for (int i = tid; i < 3 * 2048 / 16; i += kMlpThreads)
            reinterpret_cast<uint4*>(sm + kOffBB)[i] = wsrc[4 * kWTileBytes / 16 + i];
        // rows of the ones block: BF16 1.0 in K columns 0 and 1 (chunk 0 before the swizzle)
        for (int r = tid; r < kTileM; r += kMlpThreads) {
            *reinterpret_cast<uint4*>(sm + kOffOnes + tc::sw32_offset(r, 0)) = make_uint4(0x3F803F80u, 0u, 0u, 0u);
            *reinterpret_cast<uint4*>(sm + kOffOnes + tc::sw32_offset(r, 1)) = make_uint4(0u, 0u, 0u, 0u);
        }
    }
    for (int i = tid; i < kMlpGroups * 16384 / 16; i += kMlpThreads)
        reinterpret_cast<uint4*>(sm + kOffA)[i] = make_uint4(0, 0, 0, 0);
    for (int i = tid; i < 256; i += kMlpThreads) hbias[i] = 0.5f * m.bias[i];  // SiLU takes h = z / 2
    if (tid < 64) w4[tid] = m.w4[tid];
    if (tid < 4) {
        scale[tid] = m.scale_w[tid];
        scale[4 + tid] = m.scale_a_inv[tid];
    }
    const float b4 = m.b4[0];
    if (tid == 0) {
        for (int q = 0; q < kMlpGroups; ++q) tc::mbar_init(bar0 + q, 1);
        tc::fence_barrier_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(slot, kMlpTmemCols);
        tc::tmem_relinquish();
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *slot + 64u * (uint32_t)g;  // the group's 64 columns
    // a warp reads the TMEM lanes of its quarter of the warpgroup
    const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    constexpr uint32_t idesc = kFp8 ? tc::make_idesc(0, 0, 128, 64) : tc::make_idesc(1, 1, 128, 64);
    const uint32_t sW = tc::smem_u32(Wt), sA = tc::smem_u32(Ah);
    uint32_t phase = 0;
    bool failed = false;
    const int64_t n_rows = a.cand ? (int64_t)*a.n_cand : (a.cinfo ? *a.n_pairs : a.n);
    const int64_t n_tiles = (n_rows + kTileM - 1) / kTileM;

    // the next tile's momenta are copied (cp.async, each thread its own row)
    // into the group's staging columns while the current tile runs its layers
    const int64_t tile0 = (int64_t)blockIdx.x * kMlpGroups + g;
    const int64_t tstride = (int64_t)gridDim.x * kMlpGroups;
    if (tile0 < n_tiles) stage_pair_raw(a, tile0 * kTileM + lt, n_rows, st);
    for (int64_t tile = tile0; tile < n_tiles && !failed; tile += tstride) {
        const int64_t row = tile * kTileM + lt;
        float f[6] = {0, 0, 0, 0, 0, 0};
        asm volatile("cp.async.wait_all;" ::: "memory");
        if (row < n_rows)
            features<true>(m, st[0], st[kTileM], st[2 * kTileM], st[3 * kTileM], st[4 * kTileM], st[5 * kTileM], f);
        if (tile + tstride < n_tiles) stage_pair_raw(a, (tile + tstride) * kTileM + lt, n_rows, st);
        // layer-0 input: the 6 features in chunk 0 of the row, chunk 1 zeroed
        // (the single K step of layer 0 reads bytes 0..31 of the row)
        if (kFp8) {
            const float s = scale[4];
            *reinterpret_cast<uint4*>(Ah + tc::sw128_offset(lt, 0)) =
                make_uint4(pack_e4m3x4(f[0] * s, f[1] * s, f[2] * s, f[3] * s), pack_e4m3x4(f[4] * s, f[5] * s, 0, 0),
                           0u, 0u);
        } else {
            // K columns 6, 7 carry 1, 1: layer 0's half bias (hi, lo) sits there in W
            *reinterpret_cast<uint4*>(Ah + tc::sw128_offset(lt, 0)) =
                make_uint4(pack_bf16x2(f[0], f[1]), pack_bf16x2(f[2], f[3]), pack_bf16x2(f[4], f[5]), 0x3F803F80u);
        }
        *reinterpret_cast<uint4*>(Ah + tc::sw128_offset(lt, 1)) = make_uint4(0u, 0u, 0u, 0u);
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        group_sync(g);
        tc::fence_after_sync();

        uint64_t acc2 = act::pk2(0.0f, 0.0f);  // output layer, two partial sums
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            if (lt == 0) {
                const uint64_t ad = tc::sw128_kmajor_desc(sA);
                const uint64_t bd = tc::sw128_kmajor_desc(sW + l * kWTileBytes);
                // K steps of 32 bytes that hold data: layer 0 one (6 features),
                // hidden layers 64 values = 4 steps in BF16, 2 in E4M3
                const int n_ks = l == 0 ? 1 : (kFp8 ? 2 : 4);
                for (int ks = 0; ks < n_ks; ++ks) {
                    // 32-byte K step inside the 128-byte swizzle atom
                    if (kFp8) tc::mma_f8(tmem, ad + 2 * ks, bd + 2 * ks, idesc, ks > 0);
                    else tc::mma_bf16(tmem, ad + 2 * ks, bd + 2 * ks, idesc, ks > 0);
                }
                if (!kFp8 && l > 0)  // the half bias: ones (K 0, 1) against (hi, lo)
                    tc::mma_bf16(tmem, tc::sw32_kmajor_desc(sW + (kOffOnes - kOffW)),
                                 tc::sw32_kmajor_desc(sW + (kOffBB - kOffW) + (l - 1) * 2048), idesc, 1u);
                tc::mma_commit(bar);
            }
            const bool ok = tc::mbar_wait(bar, phase, kWaitNs);
            phase ^= 1u;
            tc::fence_after_sync();
            if (ok) {
                // h = z / 2 = (deq acc + b) / 2, SiLU in pairs of columns; the
                // accumulator is read 16 columns at a time, the next quarter's
                // load in flight while the current one is finished
                const float hq = 0.5f * (kFp8 ? scale[l] / scale[4 + l] : 1.0f);  // w scale x activation scale
                const uint64_t hq2 = act::pk2(hq, hq);
                const float snext = (kFp8 && l < 3) ? scale[4 + l + 1] : 1.0f;
                const float* hb = hbias + l * 64;
                // columns 16 qc .. 16 qc + 15 of the layer, from registers r
                auto quarter = [&](int qc, uint32_t (&r)[16]) {
                    const float4* hb4 = reinterpret_cast<const float4*>(hb + 16 * qc);
                    uint32_t pk[8];
                    float y[16];
#pragma unroll
                    for (int c4 = 0; c4 < 4; ++c4) {
                        const float4 b = kFp8 ? hb4[c4] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            const int c = 4 * c4 + 2 * q;
                            const uint64_t acc = act::pk2(__uint_as_float(r[c]), __uint_as_float(r[c + 1]));
                            // BF16: the accumulator is h already; FP8: h = (deq acc + b) / 2
                            const uint64_t h2 =
                                kFp8 ? act::fma2(acc, hq2, q ? act::pk2(b.z, b.w) : act::pk2(b.x, b.y)) : acc;
                            const uint64_t y2 = (!kFp8 && (8 * qc + c / 2) % 16 < kSiluFmaPairs)
                                                    ? act::silu2_fma(h2)
                                                    : act::silu2_mufu(h2);
                            act::upk2(y2, y[c], y[c + 1]);
                        }
                    }
                    if (l < 3) {
                        if (kFp8) {
                            // 16 values -> 16 bytes = chunk qc of the 64-byte real half of the row
                            *reinterpret_cast<uint4*>(Ah + tc::sw128_offset(lt, qc)) = make_uint4(
                                pack_e4m3x4(y[0] * snext, y[1] * snext, y[2] * snext, y[3] * snext),
                                pack_e4m3x4(y[4] * snext, y[5] * snext, y[6] * snext, y[7] * snext),
                                pack_e4m3x4(y[8] * snext, y[9] * snext, y[10] * snext, y[11] * snext),
                                pack_e4m3x4(y[12] * snext, y[13] * snext, y[14] * snext, y[15] * snext));
                        } else {
#pragma unroll
                            for (int c = 0; c < 8; ++c) pk[c] = pack_bf16x2(y[2 * c], y[2 * c + 1]);
                            // 16 BF16 values = chunks 2 qc, 2 qc + 1 of the row
                            *reinterpret_cast<uint4*>(Ah + tc::sw128_offset(lt, 2 * qc)) =
                                make_uint4(pk[0], pk[1], pk[2], pk[3]);
                            *reinterpret_cast<uint4*>(Ah + tc::sw128_offset(lt, 2 * qc + 1)) =
                                make_uint4(pk[4], pk[5], pk[6], pk[7]);
                        }
                    } else {
                        const float4* w4v = reinterpret_cast<const float4*>(w4 + 16 * qc);
#pragma unroll
                        for (int c4 = 0; c4 < 4; ++c4) {
                            const float4 w = w4v[c4];
                            acc2 = act::fma2(act::pk2(y[4 * c4], y[4 * c4 + 1]), act::pk2(w.x, w.y), acc2);
                            acc2 = act::fma2(act::pk2(y[4 * c4 + 2], y[4 * c4 + 3]), act::pk2(w.z, w.w), acc2);
                        }
                    }
                };
                uint32_t ra[16], rb[16];
                tc::tmem_ld16(trow + 0, ra);
                tc::tmem_wait16(ra);
                tc::tmem_ld16(trow + 16, rb);
                quarter(0, ra);
                tc::tmem_wait16(rb);
                tc::tmem_ld16(trow + 32, ra);
                quarter(1, rb);
                tc::tmem_wait16(ra);
                tc::tmem_ld16(trow + 48, rb);
                quarter(2, ra);
                tc::tmem_wait16(rb);
                quarter(3, rb);
            }
            if (l < 3) tc::fence_proxy_async_smem();
            tc::fence_before_sync();
            const bool bad = group_sync_or(g, !ok);
            tc::fence_after_sync();
            if (bad) {
                failed = true;
                break;
            }
        }
        float acc_lo, acc_hi;
        act::upk2(acc2, acc_lo, acc_hi);
        const float acc_out = acc_lo + acc_hi;
        if (a.decide) decide_row(a, row, !failed && row < n_rows, acc_out + b4);
        else if (!failed && row < n_rows) a.r_out[row] = __fdividef(1.0f, 1.0f + __expf(-(acc_out + b4)));
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (failed && lt == 0) atomicOr(&a.stats->error_flags, (unsigned long long)kErrTimeout);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(*slot, kMlpTmemCols);
}

// ---------------------------------------------------------------------------
// BF16 forward with the A operand in tensor memory.  Each row group keeps its
// accumulator (64 columns) and its next layer's input (32 columns, two BF16
// values per column) in TMEM, so an epilogue writes a row's 64 activations
// with four tcgen05.st instead of shared-memory stores and a proxy fence;
// 96 columns per group fit five groups in the 512 columns.  Otherwise as
// k_mlp_tc<false>: half weights in shared memory, the half bias as one more
// K step against a block of ones, h = z / 2 in the accumulator.
// ---------------------------------------------------------------------------
constexpr int kTaGroups = 5;
constexpr int kTaThreads = 128 * kTaGroups;
constexpr uint32_t kTaOffW = 0;                                     // 4 half-weight tiles
constexpr uint32_t kTaOffRaw = kTaOffW + 4 * kWTileBytes;           // staged momenta per group
constexpr uint32_t kTaOffBB = kTaOffRaw + 6 * kTileM * 4 * kTaGroups;  // half-bias blocks (256-aligned)
constexpr uint32_t kTaOffOnes = kTaOffBB + 3 * 2048;                // ones block of the bias step
constexpr uint32_t kTaOffW4 = kTaOffOnes + 4096;                    // 64 floats
constexpr uint32_t kTaOffBar = kTaOffW4 + 256;                      // one mbarrier per group
constexpr uint32_t kTaOffSlot = kTaOffBar + 8 * 8;                  // TMEM address
constexpr uint32_t kTaSmem = kTaOffSlot + 16 + 1024;                // + alignment slack
// requested at launch: more than half an SM's shared memory, so that one CTA
// (which allocates all 512 TMEM columns) is resident per SM
constexpr uint32_t kTaSmemLaunch = 120 * 1024;
static_assert(kTaSmem <= kTaSmemLaunch, "layout exceeds the launch size");
static_assert(kTaOffBB % 256 == 0 && kTaOffOnes % 256 == 0, "32-byte swizzled blocks need 256-byte alignment");

__global__ void __launch_bounds__(kTaThreads, 1) k_mlp_ta(MlpArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x;
    const int g = tid >> 7;
    const int lt = tid & 127;
    const int warp = tid >> 5;
    float* st = reinterpret_cast<float*>(sm + kTaOffRaw) + g * 6 * kTileM + lt;
    float* w4 = reinterpret_cast<float*>(sm + kTaOffW4);
    uint64_t* bar0 = reinterpret_cast<uint64_t*>(sm + kTaOffBar);
    uint64_t* bar = bar0 + g;
    uint32_t* slot = reinterpret_cast<uint32_t*>(sm + kTaOffSlot);
    const MlpDev& m = a.m;
    const uint4* wsrc = reinterpret_cast<const uint4*>(m.whalf);
    for (int i = tid; i < (int)(4 * kWTileBytes / 16); i += kTaThreads)
        reinterpret_cast<uint4*>(sm + kTaOffW)[i] = wsrc[i];
    for (int i = tid; i < 3 * 2048 / 16; i += kTaThreads)
        reinterpret_cast<uint4*>(sm + kTaOffBB)[i] = wsrc[4 * kWTileBytes / 16 + i];
    for (int r = tid; r < kTileM; r += kTaThreads) {
        *reinterpret_cast<uint4*>(sm + kTaOffOnes + tc::sw32_offset(r, 0)) = make_uint4(0x3F803F80u, 0u, 0u, 0u);
        *reinterpret_cast<uint4*>(sm + kTaOffOnes + tc::sw32_offset(r, 1)) = make_uint4(0u, 0u, 0u, 0u);
    }
    if (tid < 64) w4[tid] = m.w4[tid];
    const float b4 = m.b4[0];
    if (tid == 0) {
        for (int q = 0; q < kTaGroups; ++q) tc::mbar_init(bar0 + q, 1);
        tc::fence_barrier_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(slot, 512);
        tc::tmem_relinquish();
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t dcol = *slot + 96u * (uint32_t)g;  // accumulator: 64 columns
    const uint32_t acol = dcol + 64u;                 // next layer's input: 32 columns
    const uint32_t lanes = (uint32_t)((warp & 3) * 32) << 16;
    const uint32_t trow = dcol + lanes, arow = acol + lanes;
    constexpr uint32_t idesc = tc::make_idesc(1, 1, 128, 64);
    const uint32_t sW = tc::smem_u32(sm + kTaOffW);
    uint32_t phase = 0;
    bool failed = false;
    const int64_t n_rows = a.cand ? (int64_t)*a.n_cand : (a.cinfo ? *a.n_pairs : a.n);
    const int64_t n_tiles = (n_rows + kTileM - 1) / kTileM;
    const int64_t tile0 = (int64_t)blockIdx.x * kTaGroups + g;
    const int64_t tstride = (int64_t)gridDim.x * kTaGroups;
    if (tile0 < n_tiles) stage_pair_raw(a, tile0 * kTileM + lt, n_rows, st);
    for (int64_t tile = tile0; tile < n_tiles && !failed; tile += tstride) {
        const int64_t row = tile * kTileM + lt;
        float f[6] = {0, 0, 0, 0, 0, 0};
        asm volatile("cp.async.wait_all;" ::: "memory");
        if (row < n_rows)
            features<true>(m, st[0], st[kTileM], st[2 * kTileM], st[3 * kTileM], st[4 * kTileM], st[5 * kTileM], f);
        if (tile + tstride < n_tiles) stage_pair_raw(a, (tile + tstride) * kTileM + lt, n_rows, st);
        {
            // layer 0's input: 6 features and 1, 1 (K 6, 7: the half bias' hi, lo rows of W)
            const uint32_t x0[8] = {pack_bf16x2(f[0], f[1]), pack_bf16x2(f[2], f[3]), pack_bf16x2(f[4], f[5]),
                                    0x3F803F80u, 0u, 0u, 0u, 0u};
            tc::tmem_st8(arow, x0);
            tc::tmem_wait_st();
        }
        tc::fence_before_sync();
        group_sync(g);
        tc::fence_after_sync();

        uint64_t acc2 = act::pk2(0.0f, 0.0f);
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            if (lt == 0) {
                const uint64_t bd = tc::sw128_kmajor_desc(sW + l * kWTileBytes);
                const int n_ks = l == 0 ? 1 : 4;
                for (int ks = 0; ks < n_ks; ++ks) tc::mma_bf16_ta(dcol, acol + 8 * ks, bd + 2 * ks, idesc, ks > 0);
                if (l > 0)
                    tc::mma_bf16(dcol, tc::sw32_kmajor_desc(sW + kTaOffOnes),
                                 tc::sw32_kmajor_desc(sW + kTaOffBB + (l - 1) * 2048), idesc, 1u);
                tc::mma_commit(bar);
            }
            const bool ok = tc::mbar_wait(bar, phase, kWaitNs);
            phase ^= 1u;
            tc::fence_after_sync();
            if (ok) {
                auto quarter = [&](int qc, uint32_t (&r)[16]) {
                    uint32_t pk[8];
                    float y[16];
#pragma unroll
                    for (int c = 0; c < 16; c += 2) {
                        const uint64_t h2 = act::pk2(__uint_as_float(r[c]), __uint_as_float(r[c + 1]));
                        const uint64_t y2 =
                            ((8 * qc + c / 2) % 16 < kSiluFmaPairs) ? act::silu2_fma(h2) : act::silu2_mufu(h2);
                        act::upk2(y2, y[c], y[c + 1]);
                    }
                    if (l < 3) {
#pragma unroll
                        for (int c = 0; c < 8; ++c) pk[c] = pack_bf16x2(y[2 * c], y[2 * c + 1]);
                        tc::tmem_st8(arow + 8 * qc, pk);  // K 16 qc .. 16 qc + 15 of the next layer
                    } else {
                        const float4* w4v = reinterpret_cast<const float4*>(w4 + 16 * qc);
#pragma unroll
                        for (int c4 = 0; c4 < 4; ++c4) {
                            const float4 w = w4v[c4];
                            acc2 = act::fma2(act::pk2(y[4 * c4], y[4 * c4 + 1]), act::pk2(w.x, w.y), acc2);
                            acc2 = act::fma2(act::pk2(y[4 * c4 + 2], y[4 * c4 + 3]), act::pk2(w.z, w.w), acc2);
                        }
                    }
                };
                uint32_t ra[16], rb[16];
                tc::tmem_ld16(trow + 0, ra);
                tc::tmem_wait16(ra);
                tc::tmem_ld16(trow + 16, rb);
                quarter(0, ra);
                tc::tmem_wait16(rb);
                tc::tmem_ld16(trow + 32, ra);
                quarter(1, rb);
                tc::tmem_wait16(ra);
                tc::tmem_ld16(trow + 48, rb);
                quarter(2, ra);
                tc::tmem_wait16(rb);
                quarter(3, rb);
                if (l < 3) tc::tmem_wait_st();
            }
            tc::fence_before_sync();
            const bool bad = group_sync_or(g, !ok);
            tc::fence_after_sync();
            if (bad) {
                failed = true;
                break;
            }
        }
        float acc_lo, acc_hi;
        act::upk2(acc2, acc_lo, acc_hi);
        const float acc_out = acc_lo + acc_hi;
        if (a.decide) decide_row(a, row, !failed && row < n_rows, acc_out + b4);
        else if (!failed && row < n_rows) a.r_out[row] = __fdividef(1.0f, 1.0f + __expf(-(acc_out + b4)));
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (failed && lt == 0) atomicOr(&a.stats->error_flags, (unsigned long long)kErrTimeout);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(*slot, 512);
}

// ---------------------------------------------------------------------------
// FP32 forward on the CUDA cores: one sample per thread, activations in shared
// memory laid out [unit][thread] (conflict-free), transposed weights read as
// broadcasts, 64 accumulators in registers.
// ---------------------------------------------------------------------------
constexpr int kF32Threads = 128;

template <bool kCalib>
__global__ void __launch_bounds__(kF32Threads) k_mlp_fp32(MlpArgs a)
{
    extern __shared__ float smf[];
    float* wt = smf;                    // 4 x 64 x 64 (layer 0 uses the first 6 rows)
    float* hs = wt + 4 * 4096;          // 64 x kF32Threads
    float* bias = hs + 64 * kF32Threads;
    float* w4 = bias + 256;
    const int tid = threadIdx.x;
    const MlpDev& m = a.m;
    for (int i = tid; i < 4 * 4096 / 4; i += kF32Threads)
        reinterpret_cast<float4*>(wt)[i] = reinterpret_cast<const float4*>(m.wt32)[i];
    for (int i = tid; i < 256; i += kF32Threads) bias[i] = m.bias[i];
    if (tid < 64) w4[tid] = m.w4[tid];
    const float b4 = m.b4[0];
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * kF32Threads;
    const int64_t n_rows = a.cand ? (int64_t)*a.n_cand : (a.cinfo ? *a.n_pairs : a.n);
    for (int64_t row = (int64_t)blockIdx.x * kF32Threads + tid; row < n_rows; row += stride) {
        float f[6];
        load_pair_features(a, row, f);
        float amax[4] = {0, 0, 0, 0};
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            hs[i * kF32Threads + tid] = f[i];
            if (kCalib) amax[0] = fmaxf(amax[0], fabsf(f[i]));
        }
        float out = b4;
        for (int l = 0; l < 4; ++l) {
            float acc[64];
#pragma unroll
            for (int j = 0; j < 64; ++j) acc[j] = bias[l * 64 + j];
            const int n_in = l == 0 ? 6 : 64;
            for (int i = 0; i < n_in; ++i) {
                const float hi = hs[i * kF32Threads + tid];
                const float4* wr = reinterpret_cast<const float4*>(wt + l * 4096 + i * 64);
#pragma unroll
                for (int j4 = 0; j4 < 16; ++j4) {
                    const float4 w = wr[j4];
                    acc[4 * j4 + 0] = fmaf(w.x, hi, acc[4 * j4 + 0]);
                    acc[4 * j4 + 1] = fmaf(w.y, hi, acc[4 * j4 + 1]);
                    acc[4 * j4 + 2] = fmaf(w.z, hi, acc[4 * j4 + 2]);
                    acc[4 * j4 + 3] = fmaf(w.w, hi, acc[4 * j4 + 3]);
                }
            }
            if (l < 3) {
#pragma unroll
                for (int j = 0; j < 64; ++j) {
                    const float s = silu_exact(acc[j]);
                    hs[j * kF32Threads + tid] = s;
                    if (kCalib) amax[l + 1] = fmaxf(amax[l + 1], fabsf(s));
                }
            } else {
#pragma unroll
                for (int j = 0; j < 64; ++j) out = fmaf(silu_exact(acc[j]), w4[j], out);
            }
        }
        if (kCalib) {
#pragma unroll
            for (int l = 0; l < 4; ++l) atomicMax(reinterpret_cast<int*>(m.amax) + l, __float_as_int(amax[l]));
        } else {
            a.r_out[row] = sigmoid_exact(out);
        }
    }
}

// FP8 activation scales from the calibration maxima: inputs of layer l are
// stored as E4M3(h * 448 / amax_l).
__global__ void k_mlp_set_act_scales(MlpDev m)
{
    const int l = threadIdx.x;
    if (l < 4) {
        const float a = m.amax[l];
        m.scale_a_inv[l] = a > 0.0f ? 448.0f / a : 1.0f;
    }
}

// Persistent grid: as many CTAs as fit on every SM at once, counted from the
// device's shared-memory limits (per SM, and reserved per CTA), the register
// file and the thread limit, capped by the work.
int grid_persistent(const void* kernel, int threads, int smem, int64_t work_items, int per_item)
{
    int dev = 0, n_sm = 1, smem_sm = 0, smem_rsv = 0, regs_sm = 65536, thr_sm = 2048;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    cudaFuncAttributes fa{};
    int regs = 64;
    if (cudaFuncGetAttributes(&fa, kernel) == cudaSuccess) {
        regs = fa.numRegs > 0 ? fa.numRegs : 64;
        smem += (int)fa.sharedSizeBytes;
    }
    cudaGetLastError();
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    cudaGetLastError();
    int per_sm = smem > 0 ? smem_sm / (smem + smem_rsv) : 32;
    const int by_regs = regs_sm / (regs * threads);
    const int by_thr = thr_sm / threads;
    if (by_regs < per_sm) per_sm = by_regs;
    if (by_thr < per_sm) per_sm = by_thr;
    if (n_sm < 1) n_sm = 1;
    if (per_sm < 1) per_sm = 1;
    const int64_t need = (work_items + per_item - 1) / per_item;
    const int64_t full = (int64_t)per_sm * n_sm;
    return (int)(need < 1 ? 1 : (need < full ? need : full));
}

}  // namespace

compton_status mlp_repack(compton_ctx* ctx, cudaStream_t stream)
{
    MlpDev m = ctx->mlp;
    k_mlp_weight_amax<<<4, 256, 0, stream>>>(m);
    COMPTON_LAUNCH_CHECK(ctx, "k_mlp_weight_amax");
    k_mlp_pack<<<(4 * 64 * 128 + 255) / 256, 256, 0, stream>>>(m);
    COMPTON_LAUNCH_CHECK(ctx, "k_mlp_pack");
    return COMPTON_OK;
}

compton_status launch_mlp_infer(compton_ctx* ctx, const float* ux, const float* uy, const float* uz,
                                const float* kx, const float* ky, const float* kz, int64_t n, compton_mode mode,
                                float* r_out, cudaStream_t stream, bool binned, bool candidates,
                                const MlpDecide* decide)
{
    MlpArgs a;
    a.decide = decide != nullptr && mode != COMPTON_MODE_MLP_FP32;
    if (decide) a.dec = *decide;
    a.accepted = ctx->accepted;
    a.n_accepted = ctx->n_accepted;
    a.m = ctx->mlp;
    a.u[0] = ux;
    a.u[1] = uy;
    a.u[2] = uz;
    a.k[0] = kx;
    a.k[1] = ky;
    a.k[2] = kz;
    a.n = n;
    a.r_out = r_out;
    a.stats = ctx->stats;
    a.cinfo = binned ? ctx->cinfo : nullptr;
    a.tile_cell = binned ? ctx->tile_cell : nullptr;
    a.n_pairs = binned ? ctx->n_pairs : nullptr;
    a.cand = candidates ? ctx->cand : nullptr;
    a.n_cand = candidates ? ctx->n_cand : nullptr;
    if (mode == COMPTON_MODE_MLP_FP32) {
        const int smem = (4 * 4096 + 64 * kF32Threads + 256 + 64) * 4;
        COMPTON_CUDA_TRY(ctx, cudaFuncSetAttribute(k_mlp_fp32<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   smem));
        const int grid = grid_persistent((const void*)k_mlp_fp32<false>, kF32Threads, smem, n, kF32Threads);
        {
            TimedScope ts_(ctx, COMPTON_K_MLP, stream);
            k_mlp_fp32<false><<<grid, kF32Threads, smem, stream>>>(a);
        }
        COMPTON_LAUNCH_CHECK(ctx, "k_mlp_fp32");
        return COMPTON_OK;
    }
    const bool fp8 = mode == COMPTON_MODE_MLP_FP8;
    if (!fp8 && kBf16TmemA) {
        const void* kt = (const void*)k_mlp_ta;
        COMPTON_CUDA_TRY(ctx, cudaFuncSetAttribute(kt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTaSmemLaunch));
        const int grid_ta = grid_persistent(kt, kTaThreads, (int)kTaSmemLaunch, n, kTileM * kTaGroups);
        {
            TimedScope ts_(ctx, COMPTON_K_MLP, stream);
            k_mlp_ta<<<grid_ta, kTaThreads, kTaSmemLaunch, stream>>>(a);
        }
        COMPTON_LAUNCH_CHECK(ctx, "k_mlp_ta");
        return COMPTON_OK;
    }
    const void* kern = fp8 ? (const void*)k_mlp_tc<true> : (const void*)k_mlp_tc<false>;
    COMPTON_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemTc));
    const int grid = grid_persistent(kern, kMlpThreads, (int)kSmemTc, n, kTileM * kMlpGroups);
    {
        TimedScope ts_(ctx, COMPTON_K_MLP, stream);
        if (fp8) k_mlp_tc<true><<<grid, kMlpThreads, kSmemTc, stream>>>(a);
        else k_mlp_tc<false><<<grid, kMlpThreads, kSmemTc, stream>>>(a);
    }
    COMPTON_LAUNCH_CHECK(ctx, fp8 ? "k_mlp_tc<fp8>" : "k_mlp_tc<bf16>");
    return COMPTON_OK;
}

namespace {
// The bounded mbarrier wait of the tensor-core kernels, on a barrier that no
// one arrives at: it must give up after timeout_ns and record the timeout.
__global__ void k_selftest_wait(uint64_t timeout_ns, DeviceStats* stats)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        tc::fence_barrier_init();
        if (!tc::mbar_wait(&bar, 0, timeout_ns)) atomicOr(&stats->error_flags, (unsigned long long)kErrTimeout);
    }
}
}  // namespace

compton_status launch_selftest_wait(compton_ctx* ctx, uint64_t timeout_ns, cudaStream_t stream)
{
    k_selftest_wait<<<1, 32, 0, stream>>>(timeout_ns, ctx->stats);
    COMPTON_LAUNCH_CHECK(ctx, "k_selftest_wait");
    return COMPTON_OK;
}

compton_status launch_mlp_calibrate(compton_ctx* ctx, const float* ux, const float* uy, const float* uz,
                                    const float* kx, const float* ky, const float* kz, int64_t n,
                                    cudaStream_t stream)
{
    const bool binned = false;
    MlpArgs a;
    a.m = ctx->mlp;
    a.u[0] = ux;
    a.u[1] = uy;
    a.u[2] = uz;
    a.k[0] = kx;
    a.k[1] = ky;
    a.k[2] = kz;
    a.n = n;
    a.r_out = nullptr;
    a.stats = ctx->stats;
    a.cinfo = binned ? ctx->cinfo : nullptr;
    a.tile_cell = binned ? ctx->tile_cell : nullptr;
    a.n_pairs = binned ? ctx->n_pairs : nullptr;
    a.cand = nullptr;
    a.n_cand = nullptr;
    a.decide = false;
    a.accepted = nullptr;
    a.n_accepted = nullptr;
    const int smem = (4 * 4096 + 64 * kF32Threads + 256 + 64) * 4;
    COMPTON_CUDA_TRY(ctx, cudaMemsetAsync(ctx->mlp.amax, 0, 4 * sizeof(float), stream));
    COMPTON_CUDA_TRY(ctx, cudaFuncSetAttribute(k_mlp_fp32<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const int grid = grid_persistent((const void*)k_mlp_fp32<true>, kF32Threads, smem, n, kF32Threads);
    k_mlp_fp32<true><<<grid, kF32Threads, smem, stream>>>(a);
    COMPTON_LAUNCH_CHECK(ctx, "k_mlp_fp32<calib>");
    k_mlp_set_act_scales<<<1, 32, 0, stream>>>(ctx->mlp);
    COMPTON_LAUNCH_CHECK(ctx, "k_mlp_set_act_scales");
    return COMPTON_OK;
}

}  // namespace compton
