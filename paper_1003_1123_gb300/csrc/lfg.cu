// Additive Lagged Fibonacci generator shared by all threads (Algorithm 3):
//   x_p = x_{p-ll} + x_{p-D}  mod 2^32,   D = ll - sl.
//
// Leap.  Applying the recurrence to both terms gives, for p >= ll,
//   x_p = x_{p-2ll} + 2 x_{p-ll-D} + x_{p-2D}  mod 2^32,
// the same value with the nearest dependency twice as far back (2D instead of
// D), so twice as many positions can be in flight.  Positions below ll (the
// first ll values after seeding) use the recurrence itself.
//
// Schedule.  The sequence is cut into chunks of consecutive positions (fills)
// or of one step of C oscillators (fused Langevin step, 4 positions each).  A
// persistent cooperative grid of G CTAs takes chunk k on CTA k mod G, each CTA
// in increasing order.  Position p lives in ring[p & mask], a power-of-two ring
// of R >= 2 ll + 16384 words.  A chunk may start when every chunk that wrote a
// value it reads, and every chunk that reads a value it overwrites (position
// p - R), has finished; CTA g publishes the count of its finished chunks in
// ring_done[g] (release), so chunk j is finished iff ring_done[j mod G] > j/G.
// For the fused step the oscillators of chunk k were last written by chunk
// k - M (same oscillators, previous step); osc_done[] tracks that.
//
// Pipeline.  While chunk k is computed from shared memory, the lag windows
// (two or three contiguous ring ranges), x, v and K of chunk k + G are already
// streaming into the other shared-memory stage with cp.async.  G is kept
// below the dependency distance in chunks, so the dependencies of chunk k + G
// never include a chunk of the same CTA that is not yet finished; the lowest
// unfinished chunk can therefore always proceed.  Every wait is bounded by
// %globaltimer; a wait that runs out records GBRNG_ETIMEOUT and the kernel
// returns.
#include <algorithm>

#include "device.cuh"
#include "internal.cuh"

namespace gb {

enum { LFG_U32 = 0, LFG_UNIFORM = 1, LFG_NORMAL = 2, LFG_LD = 3, LFG_LD_INIT = 4 };

constexpr int kLfgThreads = 512;   // two CTAs per SM: 32 warps hide the phase latencies
constexpr int kLfgMaxGrid = 1024;   // CTAs at most (size of the progress caches)

struct LfgArgs {
    uint32_t* ring;
    uint32_t mask;
    int32_t ll, sl;
    int64_t base;          // first position of this launch
    int64_t n_units;       // fill: numbers; LD: oscillators N
    int64_t n_steps;       // LD: steps (init: 2)
    int64_t C;             // fill: positions per chunk; LD: oscillators per chunk (2^logC)
    int logC;
    int64_t Cpos;          // positions per chunk (fill: C, LD: 4C)
    int64_t per_step;      // LD: positions per step (4N)
    double inv_per_step;   // LD: 1 / per_step
    int64_t M;             // LD: chunks per step
    int64_t total_chunks;
    int lookahead;         // 1: prefetch chunk k + G while chunk k computes
    int win_words;         // shared words per lag window (Cpos + 8)
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

// ---------------------------------------------------------------- cp.async
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// ------------------------------------------------------------ chunk geometry
template <int MODE>
__device__ __forceinline__ void chunk_range(const LfgArgs& a, int64_t k, int64_t& P0, int64_t& P1,
                                            int64_t& t, int64_t& o0)
{
    if (MODE <= LFG_NORMAL) {
        P0 = a.base + (k << a.logC);
        P1 = min(P0 + a.C, a.base + a.n_units);
        t = 0;
        o0 = 0;
    } else {
        t = (uint32_t)k / (uint32_t)a.M;   // chunk ids stay below 2^31
        o0 = (k - t * a.M) << a.logC;
        const int64_t cnt = min(a.C, a.n_units - o0);
        P0 = a.base + 4 * (a.n_units * t + o0);
        P1 = P0 + 4 * cnt;
    }
}

// Chunk holding position q >= base.  The step index uses a double-precision
// reciprocal corrected to the exact quotient (positions stay below 2^53).
template <int MODE>
__device__ __forceinline__ int64_t chunk_of(const LfgArgs& a, int64_t q)
{
    const int64_t r = q - a.base;
    if (MODE <= LFG_NORMAL) return r >> a.logC;
    int64_t t = (int64_t)((double)r * a.inv_per_step);
    if (t * a.per_step > r) --t;
    if ((t + 1) * a.per_step <= r) ++t;
    const int64_t o = (r - t * a.per_step) >> 2;
    return t * a.M + (o >> a.logC);
}

// Bounded spin until chunk j is finished according to counter array `done`.
// `known` caches, per CTA, the largest count this CTA has already acquired:
// a dependency at or below it needs no new load (the earlier acquire and the
// barriers since then already order this CTA's reads after its writes).
__device__ bool wait_chunk(const LfgArgs& a, const uint32_t* done, uint32_t* known, int64_t j,
                           uint64_t deadline)
{
    const uint32_t G = gridDim.x;
    const uint32_t g = (uint32_t)j % G;
    const uint32_t need = (uint32_t)j / G + 1u;
    if (known[g] >= need) return true;
    unsigned ns = 16;
    uint32_t seen;
    while ((seen = ld_acquire_u32(done + g)) < need) {
        if (ld_volatile_i32(a.status) != DEV_OK) return false;
        if (global_ns() > deadline) {
            atomicCAS(a.status, DEV_OK, DEV_TIMEOUT);
            return false;
        }
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;
    }
    known[g] = seen;
    return true;
}

// Lag offsets of a chunk: the recurrence (2 windows) below position ll, the
// leap (3 windows) from ll on.  Returns the number of windows.
__device__ __forceinline__ int lag_offsets(const LfgArgs& a, int64_t P0, int64_t* off)
{
    const int64_t ll = a.ll, D = (int64_t)a.ll - a.sl;
    if (P0 >= ll) {
        off[0] = 2 * ll;
        off[1] = ll + D;
        off[2] = 2 * D;
        return 3;
    }
    off[0] = ll;
    off[1] = D;
    off[2] = 0;
    return 2;
}

// Warp 0 waits for every chunk chunk k depends on; returns false (on all
// lanes) if a wait ran out.  Lanes 0-8: the ranges read (up to 3 windows x 3
// chunks); lanes 9-23: readers of the overwritten positions p - R
// (p - R + {D, ll, 2D, ll + D, 2 ll}); lane 24: the oscillators' previous step.
template <int MODE>
__device__ bool wait_deps(const LfgArgs& a, int64_t k, uint32_t* known_ring, uint32_t* known_osc)
{
    const int lane = threadIdx.x & 31;
    int64_t P0, P1, t, o0;
    chunk_range<MODE>(a, k, P0, P1, t, o0);
    const int64_t R = (int64_t)a.mask + 1, ll = a.ll, D = (int64_t)a.ll - a.sl;
    bool ok = true;
    const uint64_t deadline = global_ns() + a.wait_ns;
    int64_t off = -1;
    int sub = 0;
    if (lane < 9) {
        int64_t offs[3];
        const int nw = lag_offsets(a, P0, offs);
        if (lane / 3 < nw) off = offs[lane / 3];
        sub = lane % 3;
    } else if (lane < 24) {
        const int q = (lane - 9) / 3;
        off = q == 0 ? R - D : q == 1 ? R - ll : q == 2 ? R - 2 * D : q == 3 ? R - ll - D : R - 2 * ll;
        sub = (lane - 9) % 3;
    }
    if (off > 0) {
        const int64_t q0 = max(P0 - off, a.base), q1 = P1 - off;
        if (q1 > a.base) {
            const int64_t j = chunk_of<MODE>(a, q0) + sub;
            if (j <= chunk_of<MODE>(a, q1 - 1))
                ok = wait_chunk(a, a.ring_done, known_ring, j, deadline);
        }
    } else if (lane == 24 && MODE >= LFG_LD && k - a.M >= 0) {
        ok = wait_chunk(a, a.osc_done, known_osc, k - a.M, deadline);
    }
    return !__any_sync(0xffffffffu, !ok);
}

// Stage layout (32-bit words): 3 lag windows of win_words, then (LD) x[3C],
// v[3C], K[C].
__device__ __forceinline__ size_t stage_words(const LfgArgs& a, bool ld)
{
    return 3 * (size_t)a.win_words + (ld ? 7 * (size_t)a.C : 0);
}

// All threads: start the async copies of chunk k into `stage`.  Lag window w
// starts at position P0 - off_w; it is fetched from the 16-byte-aligned word
// below, so its values sit at stage[w*win + shift_w + i].
template <int MODE>
__device__ void issue_copies(const LfgArgs& a, int64_t k, uint32_t* stage)
{
    int64_t P0, P1, t, o0;
    chunk_range<MODE>(a, k, P0, P1, t, o0);
    const int64_t len = P1 - P0;
    int64_t offs[3];
    const int nw = lag_offsets(a, P0, offs);
    for (int w = 0; w < nw; ++w) {
        const int64_t q0 = P0 - offs[w];
        const uint64_t start = (uint64_t)q0 & ~(uint64_t)3;
        const int shift = (int)((uint64_t)q0 & 3u);
        const int nvec = (int)((len + shift + 3) >> 2);
        uint32_t* dst = stage + (size_t)w * a.win_words;
        for (int j = threadIdx.x; j < nvec; j += blockDim.x)
            cp_async16(dst + 4 * j, a.ring + ((start + 4 * (uint64_t)j) & a.mask));
    }
    if (MODE >= LFG_LD) {
        const int64_t cnt = len >> 2;
        float* sx = (float*)stage + 3 * (size_t)a.win_words;
        float* sv = sx + 3 * a.C;
        float* sk = sv + 3 * a.C;
        if (MODE == LFG_LD) {
            // x, v: 3*cnt floats from x + 3*o0 (o0 is a multiple of 4, so
            // 16-byte aligned); the tail short of a vector is loaded directly.
            const int64_t nf = 3 * cnt, nv4 = nf >> 2;
            const float* gx = a.x + 3 * o0;
            const float* gv = a.v + 3 * o0;
            for (int64_t j = threadIdx.x; j < nv4; j += blockDim.x) {
                cp_async16(sx + 4 * j, gx + 4 * j);
                cp_async16(sv + 4 * j, gv + 4 * j);
            }
            for (int64_t j = 4 * nv4 + threadIdx.x; j < nf; j += blockDim.x) {
                sx[j] = __ldcg(gx + j);
                sv[j] = __ldcg(gv + j);
            }
        }
        if (a.Kper) {
            const int64_t nk4 = cnt >> 2;
            for (int64_t j = threadIdx.x; j < nk4; j += blockDim.x)
                cp_async16(sk + 4 * j, a.Kper + o0 + 4 * j);
            for (int64_t j = 4 * nk4 + threadIdx.x; j < cnt; j += blockDim.x)
                sk[j] = __ldcg(a.Kper + o0 + j);
        }
    }
}

template <int MODE>
__global__ void __launch_bounds__(kLfgThreads, 2) lfg_kernel(LfgArgs a)
{
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ double red[4 * 32];
    __shared__ int s_abort;
    __shared__ uint32_t known_ring[kLfgMaxGrid], known_osc[kLfgMaxGrid];
    constexpr bool LD = MODE >= LFG_LD;
    const int tid = threadIdx.x, T = blockDim.x;
    const int64_t G = gridDim.x;
    const size_t sw = stage_words(a, LD);
    uint32_t* stages[2] = {smem, smem + sw};
    uint32_t* vals = smem + 2 * sw;          // values of the chunk being consumed
    uint32_t done_count = 0;
    bool publish = true;
    Kahan e;
    double acc[3] = {0, 0, 0};
    if (tid == 0) s_abort = 0;
    for (int i = tid; i < kLfgMaxGrid; i += T) known_ring[i] = known_osc[i] = 0u;
    __syncthreads();

    // prologue: the first chunk
    int64_t k = blockIdx.x;
    if (k < a.total_chunks) {
        if (tid < 32 && !wait_deps<MODE>(a, k, known_ring, known_osc) && tid == 0) s_abort = 1;
        __syncthreads();
        if (s_abort) return;
        issue_copies<MODE>(a, k, stages[0]);
    }
    cp_async_commit();
    int s = 0;
    for (; k < a.total_chunks; k += G, s ^= 1) {
        const int64_t kn = k + G;
        const bool pre = a.lookahead && kn < a.total_chunks;
        if (pre) {
            if (tid < 32 && !wait_deps<MODE>(a, kn, known_ring, known_osc) && tid == 0) s_abort = 1;
            __syncthreads();
            if (s_abort) {
                cp_async_wait<0>();
                return;
            }
            issue_copies<MODE>(a, kn, stages[s ^ 1]);
        }
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();

        // ---- values of chunk k from the staged lag windows
        int64_t P0, P1, t, o0;
        chunk_range<MODE>(a, k, P0, P1, t, o0);
        const int64_t len = P1 - P0;
        int64_t offs[3];
        const int nw = lag_offsets(a, P0, offs);
        const uint32_t* st = stages[s];
        const uint32_t* w0 = st + ((uint64_t)(P0 - offs[0]) & 3u);
        const uint32_t* w1 = st + a.win_words + ((uint64_t)(P0 - offs[1]) & 3u);
        const uint32_t* w2 = st + 2 * a.win_words + ((uint64_t)(P0 - offs[2]) & 3u);
        for (int i = tid; i < len; i += T) {
            const int64_t q = P0 + i;
            const uint32_t val = nw == 3 ? w0[i] + 2u * w1[i] + w2[i] : w0[i] + w1[i];
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
        if (tid == 0 && publish) st_release_u32(a.ring_done + blockIdx.x, done_count + 1u);

        // ---- consume the values (pairs / oscillators)
        if (MODE == LFG_NORMAL) {
            const int64_t pairs = len >> 1, e0 = (P0 - a.base) >> 1;
            for (int64_t p = tid; p < pairs; p += T) {
                float2 g;
                box_muller(open01_from_u32(vals[2 * p]), open01_from_u32(vals[2 * p + 1]), g.x, g.y);
                __stcs((float2*)a.out + (e0 + p), g);
            }
        } else if (LD) {
            const int64_t cnt = len >> 2;
            const float* sx = (const float*)st + 3 * (size_t)a.win_words;
            const float* sv = sx + 3 * a.C;
            const float* sk = sv + 3 * a.C;
            for (int64_t o = tid; o < cnt; o += T) {
                const int64_t i = o0 + o;
                const uint4 w = *reinterpret_cast<const uint4*>(vals + 4 * o);
                float g0, g1, g2;
                box_muller(open01_from_u32(w.x), open01_from_u32(w.y), g0, g1);
                g2 = box_muller_cos(open01_from_u32(w.z), open01_from_u32(w.w));
                const float Ki = a.Kper ? sk[o] : a.c.K;
                float* xp = a.x + 3 * i;
                float* vp = a.v + 3 * i;
                if (MODE == LFG_LD_INIT) {
                    if (t == 0) {
                        const float sxx = __fsqrt_rn(__fdiv_rn(a.c.kT, Ki));
                        __stcg(xp, __fmul_rn(sxx, g0));
                        __stcg(xp + 1, __fmul_rn(sxx, g1));
                        __stcg(xp + 2, __fmul_rn(sxx, g2));
                    } else {
                        __stcg(vp, __fmul_rn(a.c.sv, g0));
                        __stcg(vp + 1, __fmul_rn(a.c.sv, g1));
                        __stcg(vp + 2, __fmul_rn(a.c.sv, g2));
                    }
                } else {
                    float x0 = sx[3 * o], x1 = sx[3 * o + 1], x2 = sx[3 * o + 2];
                    float v0 = sv[3 * o], v1 = sv[3 * o + 1], v2 = sv[3 * o + 2];
                    const float ckx = __fmul_rn(a.c.ckm, Ki);
                    em_component(a.c.cdt, a.c.cva, ckx, a.c.cs, g0, x0, v0);
                    em_component(a.c.cdt, a.c.cva, ckx, a.c.cs, g1, x1, v1);
                    em_component(a.c.cdt, a.c.cva, ckx, a.c.cs, g2, x2, v2);
                    __stcg(xp, x0), __stcg(xp + 1, x1), __stcg(xp + 2, x2);
                    __stcg(vp, v0), __stcg(vp + 1, v1), __stcg(vp + 2, v2);
                    e.add(energy3(0.5f * Ki, a.c.hm, x0, x1, x2, v0, v1, v2));
                    if (t == a.n_steps - 1) {
                        acc[0] += (double)x0 * x0 + (double)x1 * x1 + (double)x2 * x2;
                        acc[1] += (double)v0 * v0 + (double)v1 * v1 + (double)v2 * v2;
                        acc[2] += (double)x0 * v0 + (double)x1 * v1 + (double)x2 * v2;
                    }
                }
            }
        }
        __syncthreads();
        if (LD && tid == 0 && publish) st_release_u32(a.osc_done + blockIdx.x, done_count + 1u);
        ++done_count;
        if (!pre && k + G < a.total_chunks) {
            // no lookahead: fetch the next chunk now
            if (tid < 32 && !wait_deps<MODE>(a, k + G, known_ring, known_osc) && tid == 0) s_abort = 1;
            __syncthreads();
            if (s_abort) {
                cp_async_wait<0>();
                return;
            }
            issue_copies<MODE>(a, k + G, stages[s ^ 1]);
            cp_async_commit();
        }
    }
    cp_async_wait<0>();
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

// Grid size: as many resident CTAs as fit, but fewer than the dependency
// distance in chunks (and than the chunks per step for the fused step), so
// that prefetching one round ahead never waits on the prefetching CTA itself.
template <int MODE>
static int launch(Handle* h, LfgArgs& a, cudaStream_t st, int64_t* G_out)
{
    DevInfo di;
    GB_CHECK(dev_info(h->device, &di));
    constexpr bool LD = MODE >= LFG_LD;
    auto fn = lfg_kernel<MODE>;
    a.win_words = (int)(a.Cpos + 8);
    const size_t sw = 3 * (size_t)a.win_words + (LD ? 7 * (size_t)a.C : 0);
    const size_t smem = sizeof(uint32_t) * (2 * sw + ((MODE == LFG_NORMAL || LD) ? a.Cpos : 0));
    if (smem > di.smem_optin) return fail(GBRNG_EINVAL, "Lagged Fibonacci stage too large");
    GB_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kLfgThreads, smem));
    if (occ < 1) return fail(GBRNG_EINVAL, "Lagged Fibonacci kernel does not fit on an SM");
    const int64_t D = (int64_t)h->ll - h->sl;
    const int64_t R = (int64_t)h->ring_mask + 1;
    const int64_t dist_pos = std::min<int64_t>(D, R - 2 * (int64_t)h->ll);   // nearest dependency
    const int64_t delta = dist_pos / a.Cpos - 1;                              // in chunks (lower bound)
    int64_t G = (int64_t)di.sms * occ;
    G = std::min<int64_t>(G, kLfgMaxGrid);
    G = std::min<int64_t>(G, a.total_chunks);
    int64_t limit = delta;
    if (LD) limit = std::min<int64_t>(limit, a.M);
    a.lookahead = (limit - 1 >= 1) ? 1 : 0;
    if (a.lookahead) G = std::min<int64_t>(G, limit - 1);
    if (G < 1) G = 1;
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
    GB_CUDA(cudaLaunchCooperativeKernel((const void*)fn, dim3((unsigned)G), dim3(kLfgThreads), args,
                                        smem, st));
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

// Largest power-of-two chunk (in units of `unit` positions) no wider than the
// nearest dependency D = ll - sl and not above `want` units.
static int log2_chunk(const Handle* h, int64_t want, int64_t unit)
{
    const int64_t D = (int64_t)h->ll - h->sl;
    const int64_t cap = std::min<int64_t>(want, D / unit);
    int lg = 0;
    while ((int64_t)2 << lg <= cap) ++lg;
    return lg;
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
    a.logC = log2_chunk(h, 2048, 1);
    const int64_t C = (int64_t)1 << a.logC;
    a.C = C;
    a.Cpos = C;
    a.total_chunks = (n + C - 1) / C;
    if (a.total_chunks >= ((int64_t)1 << 31)) return fail(GBRNG_EINVAL, "fill too large for one call");
    a.out = dst;
    int64_t G = 0;
    if (mode == LFG_U32)
        GB_CHECK(launch<LFG_U32>(h, a, st, &G));
    else if (mode == LFG_UNIFORM)
        GB_CHECK(launch<LFG_UNIFORM>(h, a, st, &G));
    else
        GB_CHECK(launch<LFG_NORMAL>(h, a, st, &G));
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
    if (((uintptr_t)s->x & 15u) || ((uintptr_t)s->v & 15u) || ((uintptr_t)s->K_per & 15u))
        return fail(GBRNG_EINVAL, "Lagged Fibonacci systems need 16-byte aligned x, v, K_per");
    LfgArgs a{};
    a.ring = h->ring;
    a.mask = h->ring_mask;
    a.ll = h->ll;
    a.sl = h->sl;
    a.base = h->pos;
    a.n_units = s->n;
    a.n_steps = init ? 2 : n_steps;
    a.logC = log2_chunk(h, 512, 4);                   // oscillators per chunk
    const int64_t C = (int64_t)1 << a.logC;
    a.C = C;
    a.Cpos = 4 * C;
    a.M = (s->n + C - 1) / C;
    a.per_step = 4 * s->n;
    a.inv_per_step = 1.0 / (double)a.per_step;
    a.total_chunks = a.M * a.n_steps;
    if (a.total_chunks >= ((int64_t)1 << 31))
        return fail(GBRNG_EINVAL, "split runs of more than 2^31 chunks (N x steps / %lld)", (long long)C);
    a.x = s->x;
    a.v = s->v;
    a.Kper = s->K_per;
    a.c = make_coef(s);
    int64_t G = 0;
    if (init)
        GB_CHECK(launch<LFG_LD_INIT>(h, a, st, &G));
    else
        GB_CHECK(launch<LFG_LD>(h, a, st, &G));
    GB_CHECK(read_status(h, st));
    h->pos += 4 * s->n * a.n_steps;
    if (out) return finish_stats(h, G, n_steps, out, st);
    return GBRNG_OK;
}

}  // namespace gb
