// ld_run_noalloc: the fused Langevin run of the per-thread generators for
// callers that must not allocate device memory while they step a system.
//
// ld_run keeps a small scratch area in the generator handle (one slot of
// partial sums per CTA plus the final statistics) and allocates or grows it
// with cudaMalloc on demand.  Some callers cannot allow that: a real-time loop
// cannot let a step wait on cudaMalloc, which may synchronise the device; an
// application that hands the library a fixed memory budget, or owns all device
// memory through its own pool, has no room for allocations it did not make;
// and code that runs where CUDA forbids allocation has no way to make one.
// This file runs the same per-oscillator computation with its scratch in a
// file-scope device array of fixed size, so a call allocates nothing.
#include <algorithm>
#include <mutex>

#include "device.cuh"
#include "internal.cuh"

namespace gb {

// Scratch: kNoallocMaxBlocks slots of 4 partial sums, then 4 totals.  It
// belongs to every GPU that loads the library until the process exits, and it
// is shared by all calls: each call overwrites the slots it reads (nothing
// needs to start at zero), so two calls whose work overlaps on the GPU race.
constexpr int kNoallocMaxBlocks = 8192;
static __device__ __align__(256) double g_noalloc_scratch[4 * kNoallocMaxBlocks + 4];

struct NoallocArgs {
    int64_t n, n_steps;
    float* x;
    float* v;
    const float* Kper;
    LdCoef c;
    uint4* taus;
    int32_t* r2;
    int64_t S;
    double* scratch;   // device address of g_noalloc_scratch
};

// Same register budget as ld_run's per-thread kernel (six 128-thread blocks per SM).
template <int KIND>
__global__ void __launch_bounds__(128, 6) ld_noalloc_kernel(NoallocArgs a)
{
    extern __shared__ int32_t tab[];   // Ran2: [32][blockDim.x]
    __shared__ double red[4 * 32];
    const int64_t W = (int64_t)gridDim.x * blockDim.x;
    const LdCoef c = a.c;
    double acc[4] = {0, 0, 0, 0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += W) {
        const float Ki = a.Kper ? a.Kper[i] : c.K;
        float x0 = a.x[3 * i], x1 = a.x[3 * i + 1], x2 = a.x[3 * i + 2];
        float v0 = a.v[3 * i], v1 = a.v[3 * i + 1], v2 = a.v[3 * i + 2];
        TausDraw td;
        Ran2Draw rd;
        if (KIND == GBRNG_TAUS) {
            td.y = a.taus[i];
        } else {
            rd.tab = tab;
            rd.T = blockDim.x;
            rd.tid = threadIdx.x;
            rd.r.idum = a.r2[i];
            rd.r.idum2 = a.r2[a.S + i];
            rd.r.iy = a.r2[2 * a.S + i];
#pragma unroll 4
            for (int j = 0; j < 32; ++j) tab[j * blockDim.x + threadIdx.x] = a.r2[(3 + j) * a.S + i];
        }
        const float ckx = __fmul_rn(c.ckm, Ki);
        const float hK = 0.5f * Ki;
        EnergySum es;
        for (int64_t t0 = 0; t0 < a.n_steps; t0 += kEnergyBlock) {
            const int nb = (int)min((int64_t)kEnergyBlock, a.n_steps - t0);
            for (int k = 0; k < nb; ++k) {
                float g0, g1, g2;
                if (KIND == GBRNG_TAUS) td.normals3(g0, g1, g2); else rd.normals3(g0, g1, g2);
                em_component(c.cdt, c.cva, ckx, c.cs, g0, x0, v0);
                em_component(c.cdt, c.cva, ckx, c.cs, g1, x1, v1);
                em_component(c.cdt, c.cva, ckx, c.cs, g2, x2, v2);
                es.add(x0, x1, x2, v0, v1, v2);
            }
            es.flush();
        }
        a.x[3 * i] = x0, a.x[3 * i + 1] = x1, a.x[3 * i + 2] = x2;
        a.v[3 * i] = v0, a.v[3 * i + 1] = v1, a.v[3 * i + 2] = v2;
        if (KIND == GBRNG_TAUS) {
            a.taus[i] = td.y;
        } else {
            a.r2[i] = rd.r.idum;
            a.r2[a.S + i] = rd.r.idum2;
            a.r2[2 * a.S + i] = rd.r.iy;
#pragma unroll 4
            for (int j = 0; j < 32; ++j) a.r2[(3 + j) * a.S + i] = tab[j * blockDim.x + threadIdx.x];
        }
        acc[0] += (double)x0 * x0 + (double)x1 * x1 + (double)x2 * x2;
        acc[1] += (double)v0 * v0 + (double)v1 * v1 + (double)v2 * v2;
        acc[2] += (double)x0 * v0 + (double)x1 * v1 + (double)x2 * v2;
        acc[3] += es.value(hK, c.hm);
    }
    block_reduce_sum<4>(acc, red);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) a.scratch[4 * blockIdx.x + k] = acc[k];
}

// One block: fixed-order sum of `blocks` slots into the 4 totals after them.
__global__ void noalloc_finish_kernel(double* scratch, int64_t blocks)
{
    __shared__ double red[4 * 32];
    double v[4] = {0, 0, 0, 0};
    for (int64_t b = threadIdx.x; b < blocks; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] += scratch[4 * b + k];
    block_reduce_sum<4>(v, red);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) scratch[4 * kNoallocMaxBlocks + k] = v[k];
}

// Per-device setup, done once with that device current: the device address of
// the scratch array (in host code its name is only a host-side stand-in) and
// the SM count.  Fixed-size table, so the lookup allocates nothing either.
// The cached address belongs to the device's context at the first call: after
// cudaDeviceReset the module may load at another address, so a process that
// resets a device must not call ld_run_noalloc on it again.
constexpr int kNoallocMaxDevices = 64;
static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[kNoallocMaxDevices];
static int g_noalloc_sms[kNoallocMaxDevices];

static int noalloc_setup(int device, double** ptr, int* sms)
{
    if (device < 0 || device >= kNoallocMaxDevices)
        return fail(GBRNG_EINVAL, "ld_run_noalloc supports devices 0-%d", kNoallocMaxDevices - 1);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        double* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return fail(GBRNG_ECUDA, "cudaGetSymbolAddress of the no-alloc scratch failed: %s",
                        cudaGetErrorString(e));
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device);
        if (e != cudaSuccess)
            return fail(GBRNG_ECUDA, "cannot query the SM count: %s", cudaGetErrorString(e));
        g_noalloc_sms[device] = n;
        g_noalloc_ptr[device] = p;
    }
    *ptr = g_noalloc_ptr[device];
    *sms = g_noalloc_sms[device];
    return GBRNG_OK;
}

}  // namespace gb

using namespace gb;

extern "C" int ld_run_noalloc(ld_system* sys, int64_t n_steps, ld_stats* out_host, void* stream)
{
    NvtxRange range("ld_run_noalloc");
    GB_CHECK(check_system(sys, true));
    if (n_steps < 0) return fail(GBRNG_EINVAL, "n_steps must be >= 0");
    Handle* h = sys->rng;
    if (h->kind != GBRNG_TAUS && h->kind != GBRNG_RAN2)
        return fail(GBRNG_EINVAL, "ld_run_noalloc needs a per-thread generator (Taus or Ran2)");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    GB_CUDA(cudaGetDevice(&dev));
    if (dev != h->device)
        return fail(GBRNG_EINVAL, "make the generator's device current before ld_run_noalloc");
    double* scratch = nullptr;
    int sms = 0;
    GB_CHECK(noalloc_setup(dev, &scratch, &sms));
    if (out_host) {
        // the statistics are read back with a stream synchronisation, which a
        // stream in capture mode does not allow: refuse before queueing work
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        GB_CUDA(cudaStreamIsCapturing(st, &cs));
        if (cs != cudaStreamCaptureStatusNone)
            return fail(GBRNG_EINVAL,
                        "ld_run_noalloc: out_host synchronises the stream, which is capturing");
    }
    if (sys->n == 0) {
        if (out_host) *out_host = ld_stats{0, 0, 0, 0, n_steps};
        return GBRNG_OK;
    }
    // ld_run's grid shape for one oscillator a thread: one-warp blocks for Ran2
    // and small systems, else 128 threads; one full resident wave, fewer blocks
    // only when the system has fewer oscillators than that wave has threads
    // (at most SMs x 32 blocks: 4864 on a GB300, below the scratch's 8192).
    int T = 128;
    if (sys->n < (int64_t)sms * 128 * 2 || h->kind == GBRNG_RAN2) T = 32;
    const size_t smem = h->kind == GBRNG_RAN2 ? sizeof(int32_t) * 32 * T : 0;
    int occ = 0;
    if (h->kind == GBRNG_TAUS)
        GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ld_noalloc_kernel<GBRNG_TAUS>, T, smem));
    else
        GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ld_noalloc_kernel<GBRNG_RAN2>, T, smem));
    if (occ < 1) occ = 1;
    int64_t blocks = std::min<int64_t>((int64_t)sms * occ, (sys->n + T - 1) / T);
    if (blocks < 1) blocks = 1;
    if (blocks > kNoallocMaxBlocks)
        return fail(GBRNG_EINVAL,
                    "ld_run_noalloc: this launch needs %lld blocks of scratch, the fixed array "
                    "holds %d", (long long)blocks, kNoallocMaxBlocks);
    NoallocArgs a;
    a.n = sys->n;
    a.n_steps = n_steps;
    a.x = sys->x;
    a.v = sys->v;
    a.Kper = sys->K_per;
    a.c = make_coef(sys);
    a.taus = h->taus;
    a.r2 = h->r2;
    a.S = h->n;
    a.scratch = scratch;
    if (h->kind == GBRNG_TAUS)
        ld_noalloc_kernel<GBRNG_TAUS><<<(unsigned)blocks, T, smem, st>>>(a);
    else
        ld_noalloc_kernel<GBRNG_RAN2><<<(unsigned)blocks, T, smem, st>>>(a);
    GB_CUDA(cudaGetLastError());
    if (!out_host) return GBRNG_OK;
    noalloc_finish_kernel<<<1, 256, 0, st>>>(scratch, blocks);
    GB_CUDA(cudaGetLastError());
    double host[4];
    GB_CUDA(cudaMemcpyAsync(host, scratch + 4 * kNoallocMaxBlocks, sizeof host, cudaMemcpyDeviceToHost,
                            st));
    GB_CUDA(cudaStreamSynchronize(st));
    out_host->sum_x2 = host[0];
    out_host->sum_v2 = host[1];
    out_host->sum_xv = host[2];
    out_host->energy_time_avg = n_steps > 0 ? host[3] / (double)n_steps : 0.0;
    out_host->steps = n_steps;
    return GBRNG_OK;
}
