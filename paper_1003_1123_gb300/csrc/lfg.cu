// Additive Lagged Fibonacci generator shared by all threads (Algorithm 3):
//   x_p = x_{p-ll} + x_{p-(ll-sl)}  mod 2^32.
//
// The sequence is walked in chunks of consecutive positions by a persistent
// cooperative grid: chunk k goes to CTA k mod G, and each CTA takes its chunks
// in increasing order.  Position p lives in ring[p & mask] (a power-of-two ring
// of R >= ll + 8192 words, so no modulo and aligned writes).  A chunk may start
// once every chunk that
//   - wrote the values it reads (positions p - ll and p - (ll - sl)), and
//   - read the values it overwrites (positions p - R + ll and p - R + ll - sl)
// has finished.  Chunks are never wider than ll - sl, so those are always
// earlier chunks; because every CTA is resident and works in chunk order, the
// lowest unfinished chunk can always proceed.  CTA g publishes how many of
// its chunks are done in ring_done[g] (release) -- chunk j is done iff
// ring_done[j mod G] > j div G.  For the fused Langevin step a second counter
// osc_done[g] is released after the oscillators of a chunk are written, so
// the same oscillators' next step (chunk k - M) can be awaited.  Every wait is
// bounded by %globaltimer; a wait that runs out records a timeout in the
// status word and the kernel returns.
#include "device.cuh"
#include "internal.cuh"

namespace gb {

enum { LFG_U32 = 0, LFG_UNIFORM = 1, LFG_NORMAL = 2, LFG_LD = 3, LFG_LD_INIT = 4 };

struct LfgArgs {
    uint32_t* ring;
    uint32_t mask;
    int32_t ll, sl;
    int64_t base;          // first position of this launch
    int64_t n_units;       // fill: numbers; LD: oscillators N
    int64_t n_steps;       // LD: steps (init: 2)
    int64_t C;             // fill: positions per chunk; LD: oscillators per chunk
    int64_t M;             // LD: chunks per step
    int64_t total_chunks;
    void* out;
    float* x;
    float* v;
    const float* Kper;
    LdCoef c;
    uint32_t* ring_done;   // [G]
    uint32_t* osc_done;    // [G]
    int* status;
    uint64_t wait_ns;
    double* partials;      // [G][4]
    int64_t stall_chunk;   // test hook: this chunk's CTA stops publishing (-1: none)
};

template <int MODE>
__device__ __forceinline__ void chunk_range(const LfgArgs& a, int64_t k, int64_t& P0, int64_t& P1,
                                            int64_t& t, int64_t& o0)
{
    if (MODE <= LFG_NORMAL) {
        P0 = a.base + k * a.C;
        P1 = min(P0 + a.C, a.base + a.n_units);
        t = 0;
        o0 = 0;
    } else {
        t = k / a.M;
        o0 = (k - t * a.M) * a.C;
        const int64_t cnt = min(a.C, a.n_units - o0);
        P0 = a.base + 4 * (a.n_units * t + o0);
        P1 = P0 + 4 * cnt;
    }
}

template <int MODE>
__device__ __forceinline__ int64_t chunk_of(const LfgArgs& a, int64_t q)
{
    const int64_t r = q - a.base;
    if (MODE <= LFG_NORMAL) return r / a.C;
    const int64_t per_step = 4 * a.n_units;
    const int64_t t = r / per_step;
    const int64_t o = (r - t * per_step) >> 2;
    return t * a.M + o / a.C;
}

// Spin (bounded) until chunk j is done according to counter array `done`.
__device__ bool wait_chunk(const LfgArgs& a, const uint32_t* done, int64_t j, uint64_t deadline)
{
    const int64_t G = gridDim.x;
    const uint32_t* p = done + (j % G);
    const uint32_t need = (uint32_t)(j / G) + 1u;
    unsigned ns = 32;
    while (ld_acquire_u32(p) < need) {
        if (ld_volatile_i32(a.status) != DEV_OK) return false;
        if (global_ns() > deadline) {
            atomicCAS(a.status, DEV_OK, DEV_TIMEOUT);
            return false;
        }
        __nanosleep(ns);
        if (ns < 512) ns <<= 1;
    }
    return true;
}

template <int MODE>
__global__ void __launch_bounds__(256) lfg_kernel(LfgArgs a)
{
    extern __shared__ __align__(16) uint32_t vals[];   // values of the current chunk
    __shared__ double red[4 * 32];
    __shared__ int s_abort;
    const int tid = threadIdx.x, T = blockDim.x;
    const int64_t G = gridDim.x;
    const int64_t R = (int64_t)a.mask + 1;
    const int64_t offs[4] = {a.ll, a.ll - a.sl, R - a.ll + a.sl, R - a.ll};
    uint32_t done_count = 0;
    bool publish = true;
    Kahan e;
    double acc[3] = {0, 0, 0};
    if (tid == 0) s_abort = 0;
    __syncthreads();

    for (int64_t k = blockIdx.x; k < a.total_chunks; k += G) {
        int64_t P0, P1, t, o0;
        chunk_range<MODE>(a, k, P0, P1, t, o0);
        // ---- wait for the chunks this one depends on (warp 0, one lane each)
        if (tid < 32) {
            bool ok = true;
            const uint64_t deadline = global_ns() + a.wait_ns;
            if (tid < 12) {
                const int64_t off = offs[tid / 3];
                const int64_t q0 = max(P0 - off, a.base), q1 = P1 - off;
                if (q1 > a.base) {
                    const int64_t j = chunk_of<MODE>(a, q0) + tid % 3;
                    if (j <= chunk_of<MODE>(a, q1 - 1)) ok = wait_chunk(a, a.ring_done, j, deadline);
                }
            } else if (tid == 12 && MODE >= LFG_LD && k - a.M >= 0) {
                ok = wait_chunk(a, a.osc_done, k - a.M, deadline);
            }
            if (__any_sync(0xffffffffu, !ok) && tid == 0) s_abort = 1;
        }
        __syncthreads();
        if (s_abort) return;

        // ---- generate the chunk's values, element-wise and coalesced
        const int64_t len = P1 - P0;
        for (int64_t i = tid; i < len; i += T) {
            const int64_t q = P0 + i;
            const uint32_t xl = __ldcg(a.ring + ((uint64_t)(q - a.ll) & a.mask));
            const uint32_t xs = __ldcg(a.ring + ((uint64_t)(q - (a.ll - a.sl)) & a.mask));
            const uint32_t val = xl + xs;
            __stcg(a.ring + ((uint64_t)q & a.mask), val);
            if (MODE == LFG_U32)
                __stcs((uint32_t*)a.out + (q - a.base), val);
            else if (MODE == LFG_UNIFORM)
                __stcs((float*)a.out + (q - a.base), u01_from_u32(val));
            else
                vals[i] = val;
        }
        __syncthreads();
        if (k == a.stall_chunk) publish = false;
        if (tid == 0 && publish) {
            __threadfence();
            st_release_u32(a.ring_done + blockIdx.x, done_count + 1u);
        }

        // ---- consume the values (pairs / oscillators) from shared memory
        if (MODE == LFG_NORMAL) {
            const int64_t pairs = len >> 1, e0 = (P0 - a.base) >> 1;
            for (int64_t p = tid; p < pairs; p += T) {
                float2 g;
                box_muller(open01_from_u32(vals[2 * p]), open01_from_u32(vals[2 * p + 1]), g.x, g.y);
                __stcs((float2*)a.out + (e0 + p), g);
            }
        } else if (MODE >= LFG_LD) {
            const int64_t cnt = len >> 2;
            for (int64_t o = tid; o < cnt; o += T) {
                const int64_t i = o0 + o;
                const uint4 w = *reinterpret_cast<const uint4*>(vals + 4 * o);
                float g0, g1, g2;
                box_muller(open01_from_u32(w.x), open01_from_u32(w.y), g0, g1);
                g2 = box_muller_cos(open01_from_u32(w.z), open01_from_u32(w.w));
                const float Ki = a.Kper ? __ldcg(a.Kper + i) : a.c.K;
                float* xp = a.x + 3 * i;
                float* vp = a.v + 3 * i;
                if (MODE == LFG_LD_INIT) {
                    if (t == 0) {
                        const float sx = __fsqrt_rn(__fdiv_rn(a.c.kT, Ki));
                        __stcg(xp, __fmul_rn(sx, g0));
                        __stcg(xp + 1, __fmul_rn(sx, g1));
                        __stcg(xp + 2, __fmul_rn(sx, g2));
                    } else {
                        __stcg(vp, __fmul_rn(a.c.sv, g0));
                        __stcg(vp + 1, __fmul_rn(a.c.sv, g1));
                        __stcg(vp + 2, __fmul_rn(a.c.sv, g2));
                    }
                } else {
                    float x0 = __ldcg(xp), x1 = __ldcg(xp + 1), x2 = __ldcg(xp + 2);
                    float v0 = __ldcg(vp), v1 = __ldcg(vp + 1), v2 = __ldcg(vp + 2);
                    const float ckx = __fmul_rn(a.c.ckm, Ki);
                    em_component(a.c.cdt, a.c.cva, ckx, a.c.cs, g0, x0, v0);
                    em_component(a.c.cdt, a.c.cva, ckx, a.c.cs, g1, x1, v1);
                    em_component(a.c.cdt, a.c.cva, ckx, a.c.cs, g2, x2, v2);
                    __stcg(xp, x0), __stcg(xp + 1, x1), __stcg(xp + 2, x2);
                    __stcg(vp, v0), __stcg(vp + 1, v1), __stcg(vp + 2, v2);
                    const float xx = x0 * x0 + x1 * x1 + x2 * x2;
                    const float vv = v0 * v0 + v1 * v1 + v2 * v2;
                    e.add(0.5f * Ki * xx + a.c.hm * vv);
                    if (t == a.n_steps - 1) {
                        acc[0] += (double)x0 * x0 + (double)x1 * x1 + (double)x2 * x2;
                        acc[1] += (double)v0 * v0 + (double)v1 * v1 + (double)v2 * v2;
                        acc[2] += (double)x0 * v0 + (double)x1 * v1 + (double)x2 * v2;
                    }
                }
            }
            __syncthreads();
            if (tid == 0 && publish) {
                __threadfence();
                st_release_u32(a.osc_done + blockIdx.x, done_count + 1u);
            }
        }
        ++done_count;
    }
    if (MODE == LFG_LD && a.partials) {
        double v[4] = {acc[0], acc[1], acc[2], e.value()};
        block_reduce_sum<4>(v, red);
        if (tid == 0)
#pragma unroll
            for (int q = 0; q < 4; ++q) a.partials[4 * blockIdx.x + q] = v[q];
    }
}

// Seeds: ring word for position w - ll (w = 0..ll-1) is the low half of
// SplitMix64 at counter w; x_{-ll} is forced odd.
__global__ void lfg_seed_kernel(uint64_t seed, int32_t ll, uint32_t mask, uint32_t* ring)
{
    const int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (w >= ll) return;
    uint32_t v = (uint32_t)splitmix64_at(seed, (uint64_t)w);
    if (w == 0) v |= 1u;
    ring[(uint64_t)(w - ll) & mask] = v;
}

int lfg_seed(Handle* h, cudaStream_t st)
{
    h->pos = 0;
    const int T = 256;
    lfg_seed_kernel<<<(unsigned)((h->ll + T - 1) / T), T, 0, st>>>(h->seed, h->ll, h->ring_mask,
                                                                   h->ring);
    GB_CUDA(cudaGetLastError());
    return GBRNG_OK;
}

template <int MODE>
static int launch(Handle* h, LfgArgs& a, int T, size_t smem, cudaStream_t st, int64_t* G_out)
{
    DevInfo di;
    GB_CHECK(dev_info(h->device, &di));
    auto fn = lfg_kernel<MODE>;
    if (smem > 48 * 1024) GB_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       (int)smem));
    int occ = 0;
    GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, T, smem));
    if (occ < 1) return fail(GBRNG_EINVAL, "Lagged Fibonacci kernel does not fit on an SM");
    int64_t G = (int64_t)di.sms * occ;
    if (G > a.total_chunks) G = a.total_chunks;
    GB_CHECK(ensure_progress(h, 2 * G));
    if (MODE == LFG_LD) GB_CHECK(ensure_partials(h, G));
    a.ring_done = h->progress;
    a.osc_done = h->progress + G;
    a.status = h->dstatus;
    a.wait_ns = wait_limit_ns();
    a.partials = MODE == LFG_LD ? h->partials : nullptr;
    a.stall_chunk = test_stall_chunk();
    GB_CUDA(cudaMemsetAsync(h->progress, 0, sizeof(uint32_t) * 2 * G, st));
    GB_CUDA(cudaMemsetAsync(h->dstatus, 0, sizeof(int), st));
    void* args[] = {&a};
    GB_CUDA(cudaLaunchCooperativeKernel((const void*)fn, dim3((unsigned)G), dim3(T), args, smem, st));
    *G_out = G;
    return GBRNG_OK;
}

static int read_status(Handle* h, cudaStream_t st)
{
    int s = 0;
    GB_CUDA(cudaMemcpyAsync(&s, h->dstatus, sizeof(int), cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    if (s == DEV_TIMEOUT)
        return fail(GBRNG_ETIMEOUT, "Lagged Fibonacci chunk wait exceeded %llu ns",
                    (unsigned long long)wait_limit_ns());
    return GBRNG_OK;
}

int lfg_fill(Handle* h, void* dst, int64_t n, int mode, cudaStream_t st)
{
    LfgArgs a{};
    a.ring = h->ring;
    a.mask = h->ring_mask;
    a.ll = h->ll;
    a.sl = h->sl;
    a.base = h->pos;
    a.n_units = n;
    int64_t C = 4096;
    if (C > h->ll - h->sl) C = (h->ll - h->sl) & ~(int64_t)1;
    a.C = C;
    a.total_chunks = (n + C - 1) / C;
    a.out = dst;
    const int T = 256;
    int64_t G = 0;
    if (mode == LFG_U32)
        GB_CHECK(launch<LFG_U32>(h, a, T, 0, st, &G));
    else if (mode == LFG_UNIFORM)
        GB_CHECK(launch<LFG_UNIFORM>(h, a, T, 0, st, &G));
    else
        GB_CHECK(launch<LFG_NORMAL>(h, a, T, sizeof(uint32_t) * C, st, &G));
    GB_CHECK(read_status(h, st));
    h->pos += n;
    return GBRNG_OK;
}

// Final-state statistics when no step is taken.
__global__ void snapshot_kernel(const float* x, const float* v, int64_t n, double* partials)
{
    __shared__ double red[4 * 32];
    double acc[4] = {0, 0, 0, 0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double xi = x[i], vi = v[i];
        acc[0] += xi * xi;
        acc[1] += vi * vi;
        acc[2] += xi * vi;
    }
    block_reduce_sum<4>(acc, red);
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) partials[4 * blockIdx.x + k] = acc[k];
}

int lfg_ld(const ld_system* s, int64_t n_steps, int init, ld_stats* out, cudaStream_t st)
{
    Handle* h = s->rng;
    if (s->n == 0 || (!init && n_steps == 0)) {
        if (out) {
            if (s->n == 0) {
                *out = ld_stats{0, 0, 0, 0, n_steps};
                return GBRNG_OK;
            }
            GB_CHECK(ensure_partials(h, 256));
            snapshot_kernel<<<256, 256, 0, st>>>(s->x, s->v, s->n, h->partials);
            GB_CUDA(cudaGetLastError());
            return finish_stats(h, 256, 0, out, st);
        }
        return GBRNG_OK;
    }
    LfgArgs a{};
    a.ring = h->ring;
    a.mask = h->ring_mask;
    a.ll = h->ll;
    a.sl = h->sl;
    a.base = h->pos;
    a.n_units = s->n;
    a.n_steps = init ? 2 : n_steps;
    int64_t C = 256;                                  // oscillators per chunk
    if (4 * C > h->ll - h->sl) C = (h->ll - h->sl) / 4;
    if (C > s->n) C = s->n;
    a.C = C;
    a.M = (s->n + C - 1) / C;
    a.total_chunks = a.M * a.n_steps;
    a.x = s->x;
    a.v = s->v;
    a.Kper = s->K_per;
    a.c = make_coef(s);
    const int T = 256;
    const size_t smem = sizeof(uint32_t) * 4 * C;
    int64_t G = 0;
    if (init)
        GB_CHECK(launch<LFG_LD_INIT>(h, a, T, smem, st, &G));
    else
        GB_CHECK(launch<LFG_LD>(h, a, T, smem, st, &G));
    GB_CHECK(read_status(h, st));
    h->pos += 4 * s->n * a.n_steps;
    if (out) return finish_stats(h, G, n_steps, out, st);
    return GBRNG_OK;
}

}  // namespace gb
