// serve.cu -- continuous-batching serving of pre-paired Compton batches.
//
// The paper's network object is invoked "for any given batch of inputs"
// (Sec. 2); a PIC code produces such batches from many tiles and time steps.
// This engine admits pair lists of uneven sizes as they arrive, runs them
// together on the GPU and returns each result as soon as it is done:
//
//   compton_submit    validates a request and queues it (host, thread-safe).
//   engine thread     loops: admits queued requests while a block of the
//                     budgeted pool fits them (first fit, in arrival order),
//                     stages each admitted request into its block (device to
//                     device copies on the copy stream, then the network pass
//                     for surrogate requests); launches one k_serve over the
//                     pending tiles (1024 pairs each) of every staged request;
//                     when a launch completes, requests whose tiles are all
//                     done are copied back to the caller's output arrays and
//                     their blocks freed.  Up to two launches are in flight.
//   compton_poll      returns ENOTREADY or the request's result.
//
// Every pair of request r uses Philox counter (pair index within r, step_r)
// under key seed_r, so a request's result does not depend on what it shares
// the GPU with.  No kernel waits on another or on the host: all coordination
// is host-side through events.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ctx.hpp"
#include "device_math.cuh"

namespace compton {

constexpr int kServeThreads = 256;
constexpr int kServePairsPerThread = kPairsPerTile / kServeThreads;
constexpr int kServeQueueCap = kPairsPerTile + kServeThreads;
constexpr int kMaxTilesPerLaunch = 32768;  // 33.5M pairs
constexpr int kTileRing = 4;

struct ReqDev {
    float* u[3];
    float* k[3];
    const float* dens;   // per pair, or nullptr
    const float* r_mlp;  // network output per pair (surrogate requests)
    float dens_scalar;
    int mode;
    uint64_t seed, step;
    unsigned long long* scatters;
};

struct TileDev {
    int32_t req;
    int32_t count;
    int64_t first;
};

namespace {

struct SQEntry {
    int32_t req, p;
    float x, F2;
};

__device__ __forceinline__ void serve_resolve(const ReqDev* reqs, const SQEntry& e, float gamma64, float c64sq)
{
    const ReqDev& R = reqs[e.req];
    float ux = R.u[0][e.p], uy = R.u[1][e.p], uz = R.u[2][e.p];
    float kx = R.k[0][e.p], ky = R.k[1][e.p], kz = R.k[2][e.p];
    float x = e.x, F2 = e.F2;
    if (x < 0.0f) {
        const Invariants inv = invariants_f32(ux, uy, uz, kx, ky, kz);
        float v = inv.v;
        x = inv.x;
        if (inv.gamma > gamma64) invariants_f64(ux, uy, uz, kx, ky, kz, &x, &v);
        F2 = kn_F2(x);
    }
    const Philox4 rnd = draw(R.seed, R.step, kStreamAngle, (uint32_t)e.p);
    const Angle ang = kn_sample_angle(x, rnd.r0 >> 8, F2);
    collide_pair(ux, uy, uz, kx, ky, kz, x, ang, u24_closed0(rnd.r1), c64sq);
    R.u[0][e.p] = ux;
    R.u[1][e.p] = uy;
    R.u[2][e.p] = uz;
    R.k[0][e.p] = kx;
    R.k[1][e.p] = ky;
    R.k[2][e.p] = kz;
}

// One launch over a list of tiles from any mix of requests.  Per pair the
// arithmetic is that of k_scatter on explicit pairs (same device functions).
__global__ void __launch_bounds__(kServeThreads, 3)
    k_serve(const ReqDev* __restrict__ reqs, const TileDev* __restrict__ tiles, int n_tiles, float dt, float gamma64,
            float c64sq, DeviceStats* stats, MlpDev mlp)
{
    __shared__ SQEntry queue[kServeQueueCap];
    __shared__ int qn;
    const int tid = threadIdx.x;
    if (tid == 0) qn = 0;
    unsigned my_pairs = 0, my_scat = 0;
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const TileDev T = tiles[t];
        const ReqDev& R = reqs[T.req];
        __syncthreads();
        // tiles start at multiples of 1024 pairs: the thread's four pairs share one block
        const Philox4 rnd4 = draw(R.seed, R.step, kStreamScatter, (uint32_t)((T.first + tid * kServePairsPerThread) >> 2));
        const uint32_t words[4] = {rnd4.r0, rnd4.r1, rnd4.r2, rnd4.r3};
#pragma unroll
        for (int rr = 0; rr < kServePairsPerThread; ++rr) {
            const int local = tid * kServePairsPerThread + rr;
            if (local >= T.count) continue;
            const int64_t p = T.first + local;
            const float ux = R.u[0][p], uy = R.u[1][p], uz = R.u[2][p];
            const float kx = R.k[0][p], ky = R.k[1][p], kz = R.k[2][p];
            const float dens = R.dens ? R.dens[p] : R.dens_scalar;
            float x = -1.0f, F2 = 0.0f, P;
            bool analytic = true;
            if (R.mode != COMPTON_MODE_PLAIN) {
                const float g2 = fmaf(ux, ux, fmaf(uy, uy, fmaf(uz, uz, 1.0f)));
                const float e2 = fmaf(kx, kx, fmaf(ky, ky, kz * kz));
                if (mlp_in_range(mlp, g2, e2)) {
                    analytic = false;
                    P = one_minus_exp_neg(2.0f * dens * dt * R.r_mlp[p]);
                }
            }
            if (analytic) {
                const Invariants inv = invariants_f32(ux, uy, uz, kx, ky, kz);
                float v = inv.v;
                x = inv.x;
                if (inv.gamma > gamma64) invariants_f64(ux, uy, uz, kx, ky, kz, &x, &v);
                F2 = kn_F2(x);
                const float sig = 0.375f * F2;
                P = inv.eps > 0.0f ? one_minus_exp_neg(dens * dt * sig * v) : 0.0f;
            }
            ++my_pairs;
            if (u24_closed0(words[rr]) < P) {
                ++my_scat;
                atomicAdd(R.scatters, 1ull);
                const int slot = atomicAdd(&qn, 1);
                queue[slot] = SQEntry{T.req, (int32_t)p, x, F2};
            }
        }
        __syncthreads();
        int nq = qn;
        while (nq >= kServeThreads) {
            serve_resolve(reqs, queue[nq - kServeThreads + tid], gamma64, c64sq);
            nq -= kServeThreads;
        }
        __syncthreads();
        if (tid == 0) qn = nq;
    }
    __syncthreads();
    if (tid < qn) serve_resolve(reqs, queue[tid], gamma64, c64sq);
    for (int d = 16; d > 0; d >>= 1) {
        my_pairs += __shfl_xor_sync(0xffffffffu, my_pairs, d);
        my_scat += __shfl_xor_sync(0xffffffffu, my_scat, d);
    }
    if ((tid & 31) == 0 && my_pairs) {
        atomicAdd(&stats->pairs_tested, (unsigned long long)my_pairs);
        atomicAdd(&stats->scatters, (unsigned long long)my_scat);
    }
}

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

// ---------------------------------------------------------------------------
// Host engine
// ---------------------------------------------------------------------------
struct ServeReq {
    uint64_t ticket = 0;
    compton_request req{};
    int64_t tiles = 0, launched = 0, done_tiles = 0;
    int state = 0;  // 0 queued, 1 staging, 2 running, 3 copying back, 4 done
    size_t off = 0, bytes = 0;
    int dslot = -1;
    double t_submit = 0, t_admit = 0, t_done = 0;
    cudaEvent_t ev = nullptr;  // staging or copy-back completion
    compton_status status = COMPTON_OK;
    uint64_t scatters = 0;
};

struct Launch {
    cudaEvent_t ev;
    std::vector<std::pair<uint64_t, int64_t>> tiles_per_req;  // ticket, tiles in this launch
};

struct ServeEngine {
    compton_ctx* ctx = nullptr;
    int device = 0;
    void* pool = nullptr;
    size_t pool_bytes = 0;
    std::map<size_t, size_t> free_blocks;  // offset -> size
    size_t in_use = 0, peak_in_use = 0;
    int max_active = 0;
    ReqDev* reqs_dev = nullptr;
    ReqDev* reqs_host = nullptr;        // pinned staging of the table
    unsigned long long* counters = nullptr;  // per device slot
    unsigned long long* scat_host = nullptr;  // pinned copy of the counters of finished requests
    std::vector<int> free_slots;
    TileDev* tiles_dev = nullptr;
    TileDev* tiles_host = nullptr;      // pinned, kTileRing x kMaxTilesPerLaunch
    int ring = 0;
    cudaStream_t s_compute = nullptr, s_copy = nullptr;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<uint64_t> queued;
    std::unordered_map<uint64_t, ServeReq> reqs;
    std::deque<Launch> inflight;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    compton_status fatal = COMPTON_OK;
};

namespace {

bool pool_alloc(ServeEngine* E, size_t bytes, size_t* off)
{
    for (auto it = E->free_blocks.begin(); it != E->free_blocks.end(); ++it) {
        if (it->second >= bytes) {
            *off = it->first;
            const size_t rest = it->second - bytes;
            const size_t at = it->first + bytes;
            E->free_blocks.erase(it);
            if (rest) E->free_blocks[at] = rest;
            E->in_use += bytes;
            E->peak_in_use = std::max(E->peak_in_use, E->in_use);
            return true;
        }
    }
    return false;
}

void pool_free(ServeEngine* E, size_t off, size_t bytes)
{
    auto it = E->free_blocks.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != E->free_blocks.end() && it->first + it->second == next->first) {
        it->second += next->second;
        E->free_blocks.erase(next);
    }
    if (it != E->free_blocks.begin()) {
        auto prev = std::prev(it);
        if (prev->first + prev->second == it->first) {
            prev->second += it->second;
            E->free_blocks.erase(it);
        }
    }
    E->in_use -= bytes;
}

size_t request_bytes(const compton_request& r)
{
    const size_t per_pair = 7 + (r.mode != COMPTON_MODE_PLAIN ? 1 : 0);
    return align256((size_t)r.n * per_pair * sizeof(float)) + 256;
}

// Admit queued requests in arrival order while blocks fit (a request that
// does not fit waits; later, smaller ones may pass it).
void admit(ServeEngine* E)
{
    for (auto it = E->queued.begin(); it != E->queued.end();) {
        ServeReq& R = E->reqs[*it];
        if (E->free_slots.empty()) break;
        size_t off;
        if (!pool_alloc(E, R.bytes, &off)) {
            ++it;
            continue;
        }
        R.off = off;
        R.dslot = E->free_slots.back();
        E->free_slots.pop_back();
        R.state = 1;
        R.t_admit = now_s();
        const int64_t n = R.req.n;
        float* base = reinterpret_cast<float*>(static_cast<char*>(E->pool) + off);
        ReqDev d{};
        for (int c = 0; c < 3; ++c) {
            d.u[c] = base + (size_t)c * n;
            d.k[c] = base + (size_t)(3 + c) * n;
        }
        float* dens = base + (size_t)6 * n;
        d.dens = R.req.n_dens_dev ? dens : nullptr;
        d.r_mlp = R.req.mode != COMPTON_MODE_PLAIN ? base + (size_t)7 * n : nullptr;
        d.dens_scalar = R.req.n_dens;
        d.mode = (int)R.req.mode;
        d.seed = R.req.seed;
        d.step = R.req.step;
        d.scatters = E->counters + R.dslot;
        E->reqs_host[R.dslot] = d;
        cudaStream_t s = E->s_copy;
        const float* src_u[3] = {R.req.ux_in_dev, R.req.uy_in_dev, R.req.uz_in_dev};
        const float* src_k[3] = {R.req.kx_in_dev, R.req.ky_in_dev, R.req.kz_in_dev};
        for (int c = 0; c < 3; ++c) {
            cudaMemcpyAsync(d.u[c], src_u[c], n * sizeof(float), cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(d.k[c], src_k[c], n * sizeof(float), cudaMemcpyDeviceToDevice, s);
        }
        if (R.req.n_dens_dev) cudaMemcpyAsync(dens, R.req.n_dens_dev, n * sizeof(float), cudaMemcpyDeviceToDevice, s);
        cudaMemsetAsync(E->counters + R.dslot, 0, sizeof(unsigned long long), s);
        cudaMemcpyAsync(E->reqs_dev + R.dslot, E->reqs_host + R.dslot, sizeof(ReqDev), cudaMemcpyHostToDevice, s);
        if (R.req.mode != COMPTON_MODE_PLAIN)
            launch_mlp_infer(E->ctx, d.u[0], d.u[1], d.u[2], d.k[0], d.k[1], d.k[2], n, R.req.mode,
                             const_cast<float*>(d.r_mlp), s, false);
        cudaEventRecord(R.ev, s);
        it = E->queued.erase(it);
    }
}

void launch_tiles(ServeEngine* E)
{
    TileDev* th = E->tiles_host + (size_t)E->ring * kMaxTilesPerLaunch;
    TileDev* td = E->tiles_dev + (size_t)E->ring * kMaxTilesPerLaunch;
    int nt = 0;
    Launch L;
    for (auto& kv : E->reqs) {
        ServeReq& R = kv.second;
        if (R.state == 1 && cudaEventQuery(R.ev) == cudaSuccess) R.state = 2;
        if (R.state != 2 || R.launched >= R.tiles) continue;
        int64_t take = 0;
        while (R.launched < R.tiles && nt < kMaxTilesPerLaunch) {
            const int64_t first = R.launched * kPairsPerTile;
            const int64_t cnt = std::min<int64_t>(kPairsPerTile, R.req.n - first);
            th[nt++] = TileDev{R.dslot, (int32_t)cnt, first};
            ++R.launched;
            ++take;
        }
        if (take) L.tiles_per_req.emplace_back(R.ticket, take);
        if (nt >= kMaxTilesPerLaunch) break;
    }
    if (nt == 0) return;
    cudaMemcpyAsync(td, th, nt * sizeof(TileDev), cudaMemcpyHostToDevice, E->s_compute);
    int n_sm = 0;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, E->device);
    const int grid = std::min(nt, n_sm * 3);
    const compton_config& cfg = E->ctx->cfg;
    k_serve<<<grid, kServeThreads, 0, E->s_compute>>>(E->reqs_dev, td, nt, (float)cfg.dt, cfg.gamma_fp64_threshold,
                                                      cfg.collide_fp64_threshold * cfg.collide_fp64_threshold,
                                                      E->ctx->stats, E->ctx->mlp);
    cudaEventCreateWithFlags(&L.ev, cudaEventDisableTiming);
    cudaEventRecord(L.ev, E->s_compute);
    E->inflight.push_back(std::move(L));
    E->ring = (E->ring + 1) % kTileRing;
}

void retire(ServeEngine* E)
{
    while (!E->inflight.empty() && cudaEventQuery(E->inflight.front().ev) == cudaSuccess) {
        Launch& L = E->inflight.front();
        for (auto& tr : L.tiles_per_req) {
            ServeReq& R = E->reqs[tr.first];
            R.done_tiles += tr.second;
            if (R.done_tiles == R.tiles) {
                // copy back to the caller's outputs once the compute stream has finished these tiles
                const int64_t n = R.req.n;
                const ReqDev& d = E->reqs_host[R.dslot];
                float* dst_u[3] = {R.req.ux_out_dev, R.req.uy_out_dev, R.req.uz_out_dev};
                float* dst_k[3] = {R.req.kx_out_dev, R.req.ky_out_dev, R.req.kz_out_dev};
                for (int c = 0; c < 3; ++c) {
                    cudaMemcpyAsync(dst_u[c], d.u[c], n * sizeof(float), cudaMemcpyDeviceToDevice, E->s_copy);
                    cudaMemcpyAsync(dst_k[c], d.k[c], n * sizeof(float), cudaMemcpyDeviceToDevice, E->s_copy);
                }
                cudaMemcpyAsync(E->scat_host + R.dslot, E->counters + R.dslot, sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost, E->s_copy);
                cudaEventRecord(R.ev, E->s_copy);
                R.state = 3;
            }
        }
        cudaEventDestroy(L.ev);
        E->inflight.pop_front();
    }
    for (auto& kv : E->reqs) {
        ServeReq& R = kv.second;
        if (R.state == 3 && cudaEventQuery(R.ev) == cudaSuccess) {
            R.state = 4;
            R.t_done = now_s();
            R.scatters = E->scat_host[R.dslot];
            pool_free(E, R.off, R.bytes);
            E->free_slots.push_back(R.dslot);
            R.dslot = -1;
        }
    }
}

void engine_loop(ServeEngine* E)
{
    cudaSetDevice(E->device);
    std::unique_lock<std::mutex> lk(E->mu);
    while (!E->stop) {
        admit(E);
        retire(E);
        if (E->inflight.size() < 2) launch_tiles(E);
        cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) {
            set_cuda_error(E->ctx, err, "serve engine");
            E->fatal = COMPTON_ECUDA;
        }
        const bool busy = !E->inflight.empty() || !E->queued.empty() ||
                          std::any_of(E->reqs.begin(), E->reqs.end(),
                                      [](const std::pair<const uint64_t, ServeReq>& kv) {
                                          return kv.second.state >= 1 && kv.second.state <= 3;
                                      });
        if (busy) {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        } else {
            E->cv.wait_for(lk, std::chrono::milliseconds(5));
        }
    }
}

}  // namespace

void serve_stop_free(ServeEngine* E);

compton_status serve_start(compton_ctx* ctx, uint64_t pool_bytes, int32_t max_active)
{
    if (ctx->serve) return COMPTON_EINVAL;
    auto* E = new (std::nothrow) ServeEngine();
    if (!E) return COMPTON_ENOMEM;
    E->ctx = ctx;
    E->device = ctx->cfg.device;
    E->pool_bytes = pool_bytes;
    E->max_active = max_active;
    cudaError_t e = inject_fault() ? cudaErrorMemoryAllocation : cudaMalloc(&E->pool, pool_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&E->reqs_dev, sizeof(ReqDev) * max_active);
    if (e == cudaSuccess) e = cudaMalloc(&E->counters, sizeof(unsigned long long) * max_active);
    if (e == cudaSuccess) e = cudaMalloc(&E->tiles_dev, sizeof(TileDev) * kMaxTilesPerLaunch * kTileRing);
    if (e == cudaSuccess) e = cudaMallocHost(&E->reqs_host, sizeof(ReqDev) * max_active);
    if (e == cudaSuccess) e = cudaMallocHost(&E->tiles_host, sizeof(TileDev) * kMaxTilesPerLaunch * kTileRing);
    if (e == cudaSuccess) e = cudaMallocHost(&E->scat_host, sizeof(unsigned long long) * max_active);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&E->s_compute, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&E->s_copy, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaGetLastError();
        serve_stop_free(E);
        return COMPTON_ENOMEM;
    }
    E->free_blocks[0] = pool_bytes;
    for (int i = max_active - 1; i >= 0; --i) E->free_slots.push_back(i);
    ctx->serve = E;
    E->worker = std::thread(engine_loop, E);
    return COMPTON_OK;
}

void serve_stop_free(ServeEngine* E)
{
    if (E->pool) cudaFree(E->pool);
    if (E->reqs_dev) cudaFree(E->reqs_dev);
    if (E->counters) cudaFree(E->counters);
    if (E->tiles_dev) cudaFree(E->tiles_dev);
    if (E->reqs_host) cudaFreeHost(E->reqs_host);
    if (E->tiles_host) cudaFreeHost(E->tiles_host);
    if (E->scat_host) cudaFreeHost(E->scat_host);
    if (E->s_compute) cudaStreamDestroy(E->s_compute);
    if (E->s_copy) cudaStreamDestroy(E->s_copy);
    for (auto& kv : E->reqs)
        if (kv.second.ev) cudaEventDestroy(kv.second.ev);
    for (auto& L : E->inflight) cudaEventDestroy(L.ev);
    delete E;
}

compton_status serve_stop(compton_ctx* ctx)
{
    ServeEngine* E = ctx->serve;
    if (!E) return COMPTON_OK;
    {
        std::lock_guard<std::mutex> lk(E->mu);
        E->stop = true;
    }
    E->cv.notify_all();
    if (E->worker.joinable()) E->worker.join();
    cudaStreamSynchronize(E->s_compute);
    cudaStreamSynchronize(E->s_copy);
    serve_stop_free(E);
    ctx->serve = nullptr;
    return COMPTON_OK;
}

compton_status serve_submit(compton_ctx* ctx, const compton_request* r, uint64_t* ticket)
{
    ServeEngine* E = ctx->serve;
    if (!E) return COMPTON_EINVAL;
    const size_t bytes = request_bytes(*r);
    if (bytes > E->pool_bytes) return COMPTON_ERANGE;
    std::lock_guard<std::mutex> lk(E->mu);
    if (E->fatal != COMPTON_OK) return E->fatal;
    if (E->queued.size() >= 65536) return COMPTON_EBUSY;
    ServeReq R;
    R.ticket = E->next_ticket++;
    R.req = *r;
    R.tiles = (r->n + kPairsPerTile - 1) / kPairsPerTile;
    R.bytes = bytes;
    R.t_submit = now_s();
    if (cudaEventCreateWithFlags(&R.ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return COMPTON_ECUDA;
    }
    *ticket = R.ticket;
    E->reqs.emplace(R.ticket, R);
    E->queued.push_back(R.ticket);
    E->cv.notify_all();
    return COMPTON_OK;
}

compton_status serve_poll(compton_ctx* ctx, uint64_t ticket, compton_result* out)
{
    ServeEngine* E = ctx->serve;
    if (!E) return COMPTON_EINVAL;
    std::lock_guard<std::mutex> lk(E->mu);
    auto it = E->reqs.find(ticket);
    if (it == E->reqs.end()) return COMPTON_EINVAL;
    ServeReq& R = it->second;
    if (R.state != 4) return E->fatal != COMPTON_OK ? E->fatal : COMPTON_ENOTREADY;
    out->status = R.status;
    out->scatters = R.scatters;
    out->latency_s = R.t_done - R.t_submit;
    out->queue_s = R.t_admit - R.t_submit;
    cudaEventDestroy(R.ev);
    E->reqs.erase(it);
    return COMPTON_OK;
}

compton_status serve_info(compton_ctx* ctx, uint64_t* in_use, uint64_t* peak, uint64_t* pool)
{
    ServeEngine* E = ctx->serve;
    if (!E) return COMPTON_EINVAL;
    std::lock_guard<std::mutex> lk(E->mu);
    *in_use = E->in_use;
    *peak = E->peak_in_use;
    *pool = E->pool_bytes;
    return COMPTON_OK;
}

}  // namespace compton
