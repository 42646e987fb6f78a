// Batched Langevin dynamics: many independent systems of uneven size in one
// persistent launch per chunk of steps, replayed from a CUDA graph.
//
// Every system is cut into tiles of T*K oscillators (a tile never spans two
// systems); a grid of resident blocks walks the tile list, one tile per block
// at a time, thread t of a tile owning K oscillators (first + t + j*T).  Each
// oscillator runs exactly the instruction sequence of ld_run (same draws, same
// binary32 operations), so trajectories and generator states equal one ld_run
// per system bit for bit.  Per-tile partial sums are reduced per system in a
// fixed order.  The launch shape (T, K, steps per launch) comes from the
// caller or from a small autotuner that times candidates on scratch copies.
#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "device.cuh"
#include "internal.cuh"

namespace gb {

struct SysDesc {
    float* x;
    float* v;
    const float* Kper;
    LdCoef c;
    uint4* taus;
    int32_t* r2;
    int64_t S;    // streams of the system's generator (row stride of r2)
    int64_t n;
};

struct Tile {
    int64_t first;
    int32_t sys;
    int32_t pad;
};

// Hybrid Taus with one oscillator per thread gets a 42-register budget (six
// 256-thread blocks per SM): on 512 uneven systems 4% faster than five blocks
// and 1% faster than four at every tile width; the other shapes keep the
// compiler's choice.
template <int KIND, int K>
__global__ void __launch_bounds__(256, KIND == GBRNG_TAUS && K == 1 ? 6 : 1)
    batched_kernel(const SysDesc* __restrict__ sys, const Tile* __restrict__ tiles,
                   int64_t n_tiles, int64_t n_steps, double* __restrict__ partials)
{
    extern __shared__ int32_t tab[];   // Ran2: [K][32][T]
    __shared__ double red[4 * 32];
    const int T = blockDim.x, tid = threadIdx.x;
    for (int64_t tl = blockIdx.x; tl < n_tiles; tl += gridDim.x) {
        const Tile tile = tiles[tl];
        const SysDesc d = sys[tile.sys];
        const LdCoef c = d.c;
        int64_t idx[K];
        bool live[K];
        float x0[K], x1[K], x2[K], v0[K], v1[K], v2[K], ckx[K], hK[K];
        TausDraw td[K];
        Ran2Draw rd[K];
        EnergySum es[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            idx[j] = tile.first + tid + (int64_t)j * T;
            live[j] = idx[j] < d.n;
            const int64_t i = live[j] ? idx[j] : 0;
            const float Ki = d.Kper ? d.Kper[i] : c.K;
            ckx[j] = __fmul_rn(c.ckm, Ki);
            hK[j] = 0.5f * Ki;
            x0[j] = d.x[3 * i], x1[j] = d.x[3 * i + 1], x2[j] = d.x[3 * i + 2];
            v0[j] = d.v[3 * i], v1[j] = d.v[3 * i + 1], v2[j] = d.v[3 * i + 2];
            if (KIND == GBRNG_TAUS) {
                td[j].y = d.taus[i];
            } else {
                rd[j].tab = tab + j * 32 * T;
                rd[j].T = T;
                rd[j].tid = tid;
                rd[j].r.idum = d.r2[i];
                rd[j].r.idum2 = d.r2[d.S + i];
                rd[j].r.iy = d.r2[2 * d.S + i];
#pragma unroll 4
                for (int q = 0; q < 32; ++q) rd[j].tab[q * T + tid] = d.r2[(3 + q) * d.S + i];
            }
        }
        if constexpr (K == 2) {
            // two oscillators a thread in the lanes of the paired binary32
            // instructions (lane j = oscillator j, each lane the scalar step),
            // two steps a loop iteration
            const float2 cdt = splat2(c.cdt), cva = splat2(c.cva), cs = splat2(c.cs);
            const float2 nckx = make_float2(-ckx[0], -ckx[1]);
            float2 X[3] = {make_float2(x0[0], x0[1]), make_float2(x1[0], x1[1]), make_float2(x2[0], x2[1])};
            float2 V[3] = {make_float2(v0[0], v0[1]), make_float2(v1[0], v1[1]), make_float2(v2[0], v2[1])};
            EnergySum2 es2;
            LcgDraw lc[2];
            for (int64_t t0 = 0; t0 < n_steps; t0 += kEnergyBlock) {
                const int nb = (int)min((int64_t)kEnergyBlock, n_steps - t0);
#pragma unroll 2
                for (int k = 0; k < nb; ++k) {
                    float2 g[3];
                    draw3x2<KIND>(td, lc, rd, g);
#pragma unroll
                    for (int q = 0; q < 3; ++q) em_component2(cdt, cva, nckx, cs, g[q], X[q], V[q]);
                    es2.add(X, V);
                }
                es2.flush();
            }
            x0[0] = X[0].x, x0[1] = X[0].y, x1[0] = X[1].x, x1[1] = X[1].y, x2[0] = X[2].x, x2[1] = X[2].y;
            v0[0] = V[0].x, v0[1] = V[0].y, v1[0] = V[1].x, v1[1] = V[1].y, v2[0] = V[2].x, v2[1] = V[2].y;
#pragma unroll
            for (int j = 0; j < 2; ++j) es[j].X = es2.X[j], es[j].V = es2.V[j];
        } else {
            for (int64_t t0 = 0; t0 < n_steps; t0 += kEnergyBlock) {
                const int nb = (int)min((int64_t)kEnergyBlock, n_steps - t0);
                for (int k = 0; k < nb; ++k) {
#pragma unroll
                    for (int j = 0; j < K; ++j) {
                        float g0, g1, g2;
                        if (KIND == GBRNG_TAUS) td[j].normals3(g0, g1, g2); else rd[j].normals3(g0, g1, g2);
                        em_component(c.cdt, c.cva, ckx[j], c.cs, g0, x0[j], v0[j]);
                        em_component(c.cdt, c.cva, ckx[j], c.cs, g1, x1[j], v1[j]);
                        em_component(c.cdt, c.cva, ckx[j], c.cs, g2, x2[j], v2[j]);
                        es[j].add(x0[j], x1[j], x2[j], v0[j], v1[j], v2[j]);
                    }
                }
#pragma unroll
                for (int j = 0; j < K; ++j) es[j].flush();
            }
        }
        double acc[4] = {0, 0, 0, 0};
#pragma unroll
        for (int j = 0; j < K; ++j) {
            if (!live[j]) continue;
            const int64_t i = idx[j];
            d.x[3 * i] = x0[j], d.x[3 * i + 1] = x1[j], d.x[3 * i + 2] = x2[j];
            d.v[3 * i] = v0[j], d.v[3 * i + 1] = v1[j], d.v[3 * i + 2] = v2[j];
            if (KIND == GBRNG_TAUS) {
                d.taus[i] = td[j].y;
            } else {
                d.r2[i] = rd[j].r.idum;
                d.r2[d.S + i] = rd[j].r.idum2;
                d.r2[2 * d.S + i] = rd[j].r.iy;
#pragma unroll 4
                for (int q = 0; q < 32; ++q) d.r2[(3 + q) * d.S + i] = rd[j].tab[q * T + tid];
            }
            acc[0] += (double)x0[j] * x0[j] + (double)x1[j] * x1[j] + (double)x2[j] * x2[j];
            acc[1] += (double)v0[j] * v0[j] + (double)v1[j] * v1[j] + (double)v2[j] * v2[j];
            acc[2] += (double)x0[j] * v0[j] + (double)x1[j] * v1[j] + (double)x2[j] * v2[j];
            acc[3] += es[j].value(hK[j], c.hm);
        }
        block_reduce_sum<4>(acc, red);
        if (tid == 0) {
            partials[4 * tl + 0] = acc[0];
            partials[4 * tl + 1] = acc[1];
            partials[4 * tl + 2] = acc[2];
            partials[4 * tl + 3] += acc[3];   // energy accumulates over launches
        }
    }
}

// One block per system: fixed-order sum of the system's tile partials.
__global__ void batched_reduce_kernel(const double* partials, const int64_t* tile_begin,
                                      double* stats)
{
    __shared__ double red[4 * 32];
    const int s = blockIdx.x;
    double v[4] = {0, 0, 0, 0};
    for (int64_t t = tile_begin[s] + threadIdx.x; t < tile_begin[s + 1]; t += blockDim.x)
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] += partials[4 * t + k];
    block_reduce_sum<4>(v, red);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) stats[4 * s + k] = v[k];
}

// ----------------------------------------------------------------- host side
struct Tune {
    int T, K;
    int64_t L;   // steps per launch (0 = all)
};

using KernelFn = void (*)(const SysDesc*, const Tile*, int64_t, int64_t, double*);

static KernelFn pick_kernel(int kind, int K)
{
    if (kind == GBRNG_TAUS) return K == 2 ? batched_kernel<GBRNG_TAUS, 2> : batched_kernel<GBRNG_TAUS, 1>;
    return K == 2 ? batched_kernel<GBRNG_RAN2, 2> : batched_kernel<GBRNG_RAN2, 1>;
}

static size_t smem_bytes(int kind, int T, int K)
{
    return kind == GBRNG_RAN2 ? sizeof(int32_t) * 32 * (size_t)T * K : 0;
}

// Device buffers and the captured graph of one (systems shape, tune, steps).
struct Plan {
    int device = -1, kind = 0, n_sys = 0;
    Tune tune{0, 0, 0};
    int64_t n_steps = -1, n_tiles = 0, grid = 0;
    std::vector<int64_t> sizes;
    SysDesc* dsys = nullptr;
    Tile* dtiles = nullptr;
    int64_t* dbegin = nullptr;
    double* dpartials = nullptr;
    double* dstats = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<Tile> tiles;
    std::vector<int64_t> begin;
    ~Plan()
    {
        if (exec) cudaGraphExecDestroy(exec);
        cudaFree(dsys);
        cudaFree(dtiles);
        cudaFree(dbegin);
        cudaFree(dpartials);
        cudaFree(dstats);
    }
};

static std::mutex g_mu;
static std::map<std::string, Plan*> g_plans;
static std::map<std::string, Tune> g_tuned;
static bool g_tune_loaded = false;

static std::string shape_key(int device, int kind, const std::vector<int64_t>& sizes)
{
    uint64_t h = 1469598103934665603ull;
    int64_t total = 0;
    for (int64_t n : sizes) {
        h = (h ^ (uint64_t)n) * 1099511628211ull;
        total += n;
    }
    char buf[160];
    snprintf(buf, sizeof buf, "dev%d:kind%d:sys%zu:osc%lld:h%016llx", device, kind, sizes.size(),
             (long long)total, (unsigned long long)h);
    return buf;
}

static void build_tiles(Plan* p)
{
    const int64_t span = (int64_t)p->tune.T * p->tune.K;
    p->tiles.clear();
    p->begin.assign(p->n_sys + 1, 0);
    for (int s = 0; s < p->n_sys; ++s) {
        p->begin[s] = (int64_t)p->tiles.size();
        for (int64_t f = 0; f < p->sizes[s]; f += span) p->tiles.push_back(Tile{f, s, 0});
    }
    p->begin[p->n_sys] = (int64_t)p->tiles.size();
    p->n_tiles = (int64_t)p->tiles.size();
}

static int fill_descs(const ld_system* sys, int n_sys, std::vector<SysDesc>& out)
{
    out.resize(n_sys);
    for (int s = 0; s < n_sys; ++s) {
        const ld_system& q = sys[s];
        SysDesc d;
        d.x = q.x;
        d.v = q.v;
        d.Kper = q.K_per;
        d.c = make_coef(&q);
        d.taus = q.rng->taus;
        d.r2 = q.rng->r2;
        d.S = q.rng->n;
        d.n = q.n;
        out[s] = d;
    }
    return GBRNG_OK;
}

static int launch_chunks(Plan* p, cudaStream_t st)
{
    KernelFn fn = pick_kernel(p->kind, p->tune.K);
    const size_t smem = smem_bytes(p->kind, p->tune.T, p->tune.K);
    const int64_t L = p->tune.L > 0 ? p->tune.L : std::max<int64_t>(p->n_steps, 1);
    int64_t done = 0;
    do {
        const int64_t steps = std::min(L, p->n_steps - done);
        fn<<<(unsigned)p->grid, p->tune.T, smem, st>>>(p->dsys, p->dtiles, p->n_tiles, steps,
                                                      p->dpartials);
        done += steps;
    } while (done < p->n_steps);
    return GBRNG_OK;
}

static int make_plan(int device, int kind, const std::vector<int64_t>& sizes, Tune tune,
                     int64_t n_steps, Plan** out)
{
    Plan* p = new Plan();
    p->device = device;
    p->kind = kind;
    p->n_sys = (int)sizes.size();
    p->sizes = sizes;
    p->tune = tune;
    p->n_steps = n_steps;
    build_tiles(p);
    DevInfo di;
    int rc = dev_info(device, &di);
    if (rc != GBRNG_OK) {
        delete p;
        return rc;
    }
    KernelFn fn = pick_kernel(kind, tune.K);
    const size_t smem = smem_bytes(kind, tune.T, tune.K);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, tune.T, smem);
    if (occ < 1) {
        cudaGetLastError();
        delete p;
        return fail(GBRNG_EINVAL, "batched launch shape T=%d K=%d does not fit", tune.T, tune.K);
    }
    p->grid = std::min<int64_t>((int64_t)di.sms * occ, p->n_tiles);
    cudaError_t e = cudaMalloc(&p->dsys, sizeof(SysDesc) * p->n_sys);
    if (e == cudaSuccess) e = cudaMalloc(&p->dtiles, sizeof(Tile) * p->n_tiles);
    if (e == cudaSuccess) e = cudaMalloc(&p->dbegin, sizeof(int64_t) * (p->n_sys + 1));
    if (e == cudaSuccess) e = cudaMalloc(&p->dpartials, sizeof(double) * 4 * p->n_tiles);
    if (e == cudaSuccess) e = cudaMalloc(&p->dstats, sizeof(double) * 4 * p->n_sys);
    if (e == cudaSuccess)
        e = cudaMemcpy(p->dtiles, p->tiles.data(), sizeof(Tile) * p->n_tiles, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(p->dbegin, p->begin.data(), sizeof(int64_t) * (p->n_sys + 1),
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return fail(GBRNG_ENOMEM, "batched plan allocation failed: %s", cudaGetErrorString(e));
    }
    // Capture: zero the partials, the chunked persistent launches, the
    // per-system reduction.
    cudaStream_t cap;
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    cudaGraph_t graph = nullptr;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaMemsetAsync(p->dpartials, 0, sizeof(double) * 4 * p->n_tiles, cap);
        launch_chunks(p, cap);
        batched_reduce_kernel<<<p->n_sys, 128, 0, cap>>>(p->dpartials, p->dbegin, p->dstats);
        e = cudaStreamEndCapture(cap, &graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return fail(GBRNG_ECUDA, "batched graph capture failed: %s", cudaGetErrorString(e));
    }
    *out = p;
    return GBRNG_OK;
}

// ------------------------------------------------------------- autotuner
static void load_tune_cache()
{
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char* path = getenv("GBRNG_TUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    char key[256];
    int T, K;
    long long L;
    while (fscanf(f, "%255s %d %d %lld", key, &T, &K, &L) == 4) g_tuned[key] = Tune{T, K, L};
    fclose(f);
}

static void store_tune(const std::string& key, Tune t)
{
    g_tuned[key] = t;
    const char* path = getenv("GBRNG_TUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %d %lld\n", key.c_str(), t.T, t.K, (long long)t.L);
    fclose(f);
}

// Time each candidate on scratch copies of x, v and the generator states (the
// caller's systems are not touched): up to 256 steps, best of two replays after
// a warm-up, so that shapes a few percent apart are told apart reliably.
static int autotune(const ld_system* sys, int n_sys, int kind, const std::vector<int64_t>& sizes,
                    int64_t n_steps, Tune* best, cudaStream_t st)
{
    const int64_t probe_steps = std::min<int64_t>(std::max<int64_t>(n_steps, 1), 256);
    // scratch: x, v (n*3 floats each) and the generator states
    // every sub-buffer starts on a 256-byte boundary (Taus states are uint4)
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    size_t bytes = 0;
    std::vector<size_t> off(n_sys);
    for (int s = 0; s < n_sys; ++s) {
        off[s] = bytes;
        const int64_t S = sys[s].rng->n;
        bytes += 2 * up(sizeof(float) * 3 * sys[s].n);
        bytes += up(kind == GBRNG_TAUS ? sizeof(uint4) * S : sizeof(int32_t) * 35 * S);
    }
    char* scratch = nullptr;
    if (cudaMalloc(&scratch, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(GBRNG_ENOMEM, "autotune scratch (%zu bytes) allocation failed", bytes);
    }
    std::vector<ld_system> copy(sys, sys + n_sys);
    std::vector<gbrng_rng> hcopy(n_sys);
    for (int s = 0; s < n_sys; ++s) {
        char* b = scratch + off[s];
        const int64_t n = sys[s].n, S = sys[s].rng->n;
        copy[s].x = (float*)b;
        copy[s].v = (float*)(b + up(sizeof(float) * 3 * n));
        char* stt = b + 2 * up(sizeof(float) * 3 * n);
        cudaMemcpyAsync(copy[s].x, sys[s].x, sizeof(float) * 3 * n, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(copy[s].v, sys[s].v, sizeof(float) * 3 * n, cudaMemcpyDeviceToDevice, st);
        hcopy[s].n = S;
        hcopy[s].kind = kind;
        if (kind == GBRNG_TAUS) {
            hcopy[s].taus = (uint4*)stt;
            cudaMemcpyAsync(stt, sys[s].rng->taus, sizeof(uint4) * S, cudaMemcpyDeviceToDevice, st);
        } else {
            hcopy[s].r2 = (int32_t*)stt;
            cudaMemcpyAsync(stt, sys[s].rng->r2, sizeof(int32_t) * 35 * S, cudaMemcpyDeviceToDevice,
                            st);
        }
        copy[s].rng = &hcopy[s];
    }
    std::vector<SysDesc> descs;
    fill_descs(copy.data(), n_sys, descs);
    const int Ts[3] = {64, 128, 256};
    const int Ks[2] = {1, 2};
    float best_ms = 1e30f;
    int rc = GBRNG_OK;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    for (int T : Ts)
        for (int K : Ks)
            for (int split = 0; split < 2; ++split) {
                Tune t{T, K, split ? std::max<int64_t>(probe_steps / 4, 1) : 0};
                Plan* p = nullptr;
                if (make_plan(sys[0].rng->device, kind, sizes, t, probe_steps, &p) != GBRNG_OK) {
                    clear_error();
                    continue;
                }
                cudaMemcpyAsync(p->dsys, descs.data(), sizeof(SysDesc) * n_sys,
                                cudaMemcpyHostToDevice, st);
                cudaGraphLaunch(p->exec, st);   // warm-up
                float ms = 1e30f;
                for (int rep = 0; rep < 2; ++rep) {
                    cudaEventRecord(a, st);
                    cudaGraphLaunch(p->exec, st);
                    cudaEventRecord(b, st);
                    cudaEventSynchronize(b);
                    float m = 0;
                    cudaEventElapsedTime(&m, a, b);
                    if (m > 0 && m < ms) ms = m;
                }
                delete p;
                if (ms < best_ms) {
                    best_ms = ms;
                    *best = Tune{T, K, split ? std::max<int64_t>(n_steps / 4, 1) : 0};
                }
            }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaError_t e = cudaStreamSynchronize(st);
    cudaFree(scratch);
    if (e != cudaSuccess) return fail(GBRNG_ECUDA, "autotune failed: %s", cudaGetErrorString(e));
    if (best_ms >= 1e30f) rc = fail(GBRNG_ECUDA, "no batched launch shape could run");
    return rc;
}

}  // namespace gb

using namespace gb;

extern "C" int ld_run_batched(ld_system* sys, int n_sys, int64_t n_steps, const int* tune,
                              ld_stats* out, void* stream)
{
    NvtxRange range("ld_run_batched");
    if (!sys || n_sys < 1) return fail(GBRNG_EINVAL, "need at least one system");
    if (n_steps < 0) return fail(GBRNG_EINVAL, "n_steps must be >= 0");
    const int kind = sys[0].rng ? sys[0].rng->kind : -1;
    if (kind != GBRNG_TAUS && kind != GBRNG_RAN2)
        return fail(GBRNG_EINVAL, "batched systems need per-thread generators (Taus or Ran2)");
    std::vector<int64_t> sizes(n_sys);
    for (int s = 0; s < n_sys; ++s) {
        GB_CHECK(check_system(&sys[s], true));
        if (sys[s].rng->kind != kind) return fail(GBRNG_EINVAL, "all systems need the same kind");
        if (sys[s].rng->device != sys[0].rng->device)
            return fail(GBRNG_EINVAL, "all systems need the same device");
        sizes[s] = sys[s].n;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int device = sys[0].rng->device;
    const std::string key = shape_key(device, kind, sizes);
    Tune t;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        load_tune_cache();
        if (tune) {
            if (tune[0] < 32 || tune[0] > 256 || (tune[0] & 31) || (tune[1] != 1 && tune[1] != 2) ||
                tune[2] < 0)
                return fail(GBRNG_EINVAL, "tune = {T in 32..256 step 32, K in {1,2}, steps >= 0}");
            t = Tune{tune[0], tune[1], tune[2]};
        } else {
            auto it = g_tuned.find(key);
            if (it != g_tuned.end()) {
                t = it->second;
            } else {
                GB_CHECK(autotune(sys, n_sys, kind, sizes, n_steps, &t, st));
                store_tune(key, t);
            }
        }
    }
    char pkey[64];
    snprintf(pkey, sizeof pkey, ":T%d:K%d:L%lld:S%lld", t.T, t.K, (long long)t.L, (long long)n_steps);
    const std::string full = key + pkey;
    Plan* p = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_plans.find(full);
        if (it != g_plans.end()) {
            p = it->second;
        } else {
            if (g_plans.size() >= 16) {     // bound the cache: drop everything
                cudaDeviceSynchronize();
                for (auto& kv : g_plans) delete kv.second;
                g_plans.clear();
            }
            GB_CHECK(make_plan(device, kind, sizes, t, n_steps, &p));
            g_plans[full] = p;
        }
    }
    std::vector<SysDesc> descs;
    fill_descs(sys, n_sys, descs);
    GB_CUDA(cudaMemcpyAsync(p->dsys, descs.data(), sizeof(SysDesc) * n_sys, cudaMemcpyHostToDevice,
                            st));
    GB_CUDA(cudaGraphLaunch(p->exec, st));
    if (!out) return GBRNG_OK;
    std::vector<double> h(4 * (size_t)n_sys);
    GB_CUDA(cudaMemcpyAsync(h.data(), p->dstats, sizeof(double) * 4 * n_sys, cudaMemcpyDeviceToHost,
                            st));
    GB_CUDA(cudaStreamSynchronize(st));
    for (int s = 0; s < n_sys; ++s) {
        out[s].sum_x2 = h[4 * s];
        out[s].sum_v2 = h[4 * s + 1];
        out[s].sum_xv = h[4 * s + 2];
        out[s].energy_time_avg = n_steps > 0 ? h[4 * s + 3] / (double)n_steps : 0.0;
        out[s].steps = n_steps;
    }
    return GBRNG_OK;
}

extern "C" int ld_batched_tune(const ld_system* sys, int n_sys, int* tune_out)
{
    if (!sys || n_sys < 1 || !tune_out) return fail(GBRNG_EINVAL, "NULL argument or no systems");
    const int kind = sys[0].rng ? sys[0].rng->kind : -1;
    if (kind != GBRNG_TAUS && kind != GBRNG_RAN2)
        return fail(GBRNG_EINVAL, "batched systems need per-thread generators (Taus or Ran2)");
    std::vector<int64_t> sizes(n_sys);
    for (int s = 0; s < n_sys; ++s) sizes[s] = sys[s].n;
    const std::string key = shape_key(sys[0].rng->device, kind, sizes);
    std::lock_guard<std::mutex> lk(g_mu);
    load_tune_cache();
    auto it = g_tuned.find(key);
    if (it == g_tuned.end()) return fail(GBRNG_EINVAL, "this shape has not been autotuned yet");
    tune_out[0] = it->second.T;
    tune_out[1] = it->second.K;
    tune_out[2] = (int)it->second.L;
    return GBRNG_OK;
}
