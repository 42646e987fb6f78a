// Additive Lagged Fibonacci generator shared by all threads (Algorithm 3):
//   x_p = x_{p-ll} + x_{p-D}  mod 2^32,   D = ll - sl.
//
// Leap.  Applying the recurrence to both terms gives, for p >= ll,
//   x_p = x_{p-2ll} + 2 x_{p-ll-D} + x_{p-2D}  mod 2^32,
// the same value with the nearest dependency twice as far back (2D instead of
// D).  Positions below ll (the first ll values after seeding) use the
// recurrence itself.
//
// Rounds.  A launch walks its positions in rounds of W consecutive positions.
// Every position of a round depends only on earlier rounds when W <= D (a
// round that starts below ll) or W <= 2D (from ll on), so a round is computed
// by the whole persistent grid at once, and rounds are separated by a grid
// barrier.  Position p lives in ring[p & mask], a power-of-two ring of
// R >= 2 ll + 2D + 16384 words; W <= R - 2 ll keeps every overwritten value
// (position p - R) out of reach of the round's readers.  For the fused
// Langevin step a round also holds at most one step (W <= 4N), so each
// oscillator is updated at most once per round.  This is the paper's
// one-step-per-launch scheme (Sec. III.C) made exact for any N: the leap turns
// its race condition ll - sl > 4N into 2(ll - sl) >= W.
//
// Within a round a warp owns blocks of 128 consecutive positions (32
// oscillator-steps): lane l reads positions 32k + l of each lag window
// (coalesced), the new values go back to the ring the same way, and a per-warp
// shared-memory buffer hands lane l positions 4l..4l+3.  A block none of whose
// windows wraps around the ring addresses each window once (32-bit slot
// arithmetic, immediate offsets).  The grid barrier is an arrival counter
// polled under a %globaltimer bound; a wait that runs out records
// GBRNG_ETIMEOUT and every CTA returns.
#include <algorithm>

#include "device.cuh"
#include "internal.cuh"

namespace gb {

enum { LFG_U32 = 0, LFG_UNIFORM = 1, LFG_NORMAL = 2, LFG_LD = 3, LFG_LD_INIT = 4 };

constexpr int kLfgThreads = 256;   // three CTAs per SM (80 registers): 24 warps to hide HBM latency;
                                   // two or four CTAs per SM: fills 5-6% slower
constexpr int kLfgWarps = kLfgThreads / 32;
constexpr int kLfgDepth = 2;     // blocks per warp with lag loads in flight

struct LfgArgs {
    uint32_t* ring;
    uint32_t mask;
    uint32_t oA, oB, oC;   // slot offsets of the leap lags: -2ll, -ll-D, -2D (mod 2^32)
    int32_t ll, sl;
    int64_t base;          // first position of this launch
    int64_t n_pos;         // positions of this launch
    int64_t N;             // LD: oscillators
    int64_t n_steps;       // LD: steps (init: 2)
    int64_t w_base;        // round width (positions) while the round starts below ll
    int64_t w_leap;        // round width from ll on
    void* out;
    float* x;
    float* v;
    const float* Kper;
    LdCoef c;
    uint64_t* arrive;      // grid-barrier arrival counter (zeroed before launch; 64-bit, never wraps)
    int* status;
    uint64_t wait_ns;
    double* partials;      // [G][4]
    int stall_cta;         // test hook: this CTA never arrives (-1: none)
};

// Grid barrier: after the CTA's threads meet, thread 0 adds one arrival with
// release semantics (publishing the CTA's writes) and polls the counter
// (relaxed loads) until every CTA of this round has arrived, then reads it once
// more with acquire semantics.  Every arrival is an atomic add to the counter,
// so that read lies in each arrival's release sequence and synchronises with
// all of them; it replaces a full acquire-release fence (3% less time a round).
// The poll is bounded by a %globaltimer deadline and stops early when another
// CTA has recorded a failure.  Returns false on every thread of the CTA on
// failure.
__device__ bool grid_barrier(const LfgArgs& a, uint64_t target, bool arrive_here)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        if (arrive_here) red_release_add_u64(a.arrive, 1ull);
        const uint64_t deadline = global_ns() + a.wait_ns;
        for (uint32_t n = 1; ld_relaxed_u64(a.arrive) < target; ++n) {
            if ((n & 15u) == 0) {
                if (ld_volatile_i32(a.status) != DEV_OK) {
                    ok = 0;
                    break;
                }
                if (global_ns() > deadline) {
                    atomicCAS(a.status, DEV_OK, DEV_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        if (ok) (void)ld_acquire_u64(a.arrive);
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// The lags of one position: value = A + 2 B + C with (A, B, C) =
// (x_{q-2ll}, x_{q-ll-D}, x_{q-2D}) from ll on (leap) and
// (x_{q-ll}, 0, x_{q-D}) below ll (the recurrence itself).
struct Lags {
    uint32_t A, B, C;
    __device__ __forceinline__ uint32_t value() const { return A + 2u * B + C; }
};

__device__ __forceinline__ Lags load_lags(const LfgArgs& a, int64_t q)
{
    const int64_t ll = a.ll, D = (int64_t)a.ll - a.sl;
    const bool leap = q >= ll;
    const uint32_t* r = a.ring;
    Lags g;
    g.A = __ldcg(r + ((uint64_t)(q - (leap ? 2 * ll : ll)) & a.mask));
    g.B = leap ? __ldcg(r + ((uint64_t)(q - ll - D) & a.mask)) : 0u;
    g.C = __ldcg(r + ((uint64_t)(q - (leap ? 2 * D : D)) & a.mask));
    return g;
}

// A block of 128 positions from q0 is "fast" when it is whole, lies at or
// above ll and none of its lag windows nor its own slots wraps around the ring.
__device__ __forceinline__ bool block_fast(const LfgArgs& a, int64_t q0, int nval)
{
    const uint32_t s = (uint32_t)q0, lim = a.mask - 127u;
    return nval == 128 && q0 >= a.ll && (s & a.mask) <= lim && ((s + a.oA) & a.mask) <= lim &&
           ((s + a.oB) & a.mask) <= lim && ((s + a.oC) & a.mask) <= lim;
}

// Issue the lag loads of lane's positions q0 + 32k + lane (k < 4, < nval).
__device__ __forceinline__ void block_load(const LfgArgs& a, int64_t q0, int nval, bool fast,
                                           Lags (&g)[4])
{
    const int lane = threadIdx.x & 31;
    if (fast) {
        const uint32_t s = (uint32_t)q0 + lane;
        const uint32_t* pA = a.ring + ((s + a.oA) & a.mask);
        const uint32_t* pB = a.ring + ((s + a.oB) & a.mask);
        const uint32_t* pC = a.ring + ((s + a.oC) & a.mask);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            g[k].A = __ldcg(pA + 32 * k);
            g[k].B = __ldcg(pB + 32 * k);
            g[k].C = __ldcg(pC + 32 * k);
        }
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (32 * k + lane < nval) g[k] = load_lags(a, q0 + 32 * k + lane);
    }
}

// Store lane's values of positions q0 + 32k + lane to the ring and to the
// warp's buffer (buf[32k + lane]).
__device__ __forceinline__ void block_store(const LfgArgs& a, int64_t q0, int nval, bool fast,
                                            const Lags (&g)[4], uint32_t* buf)
{
    const int lane = threadIdx.x & 31;
    if (fast) {
        uint32_t* p = a.ring + (((uint32_t)q0 + lane) & a.mask);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t val = g[k].value();
            __stcg(p + 32 * k, val);
            buf[32 * k + lane] = val;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = 32 * k + lane;
            const uint32_t val = g[k].value();
            if (i < nval) __stcg(a.ring + ((uint64_t)(q0 + i) & a.mask), val);
            buf[i] = val;
        }
    }
}

// Lane l's four consecutive values (positions q0 + 4l .. q0 + 4l + 3).
__device__ __forceinline__ uint4 block_transpose(const uint32_t* buf)
{
    __syncwarp();
    const uint4 w = *reinterpret_cast<const uint4*>(buf + 4 * (threadIdx.x & 31));
    __syncwarp();
    return w;
}

// Walk this warp's blocks b = first, first + step, ... < nblk of a region
// starting at q_first (positions q_first + 128 b ..), with the lag loads of
// the next kLfgDepth - 1 blocks in flight while one block is consumed.
// Positions of one round never read each other, so the early loads are exact.
// consume(b, nval, w) receives lane's four values after they are stored.
template <class F>
__device__ __forceinline__ void walk_blocks(const LfgArgs& a, int64_t q_first, int64_t n_region,
                                            int64_t first, int64_t step, uint32_t* buf, F&& consume)
{
    const int64_t nblk = (n_region + 127) >> 7;
    Lags pipe[kLfgDepth][4];
    bool fast[kLfgDepth];
    int nv[kLfgDepth];
#pragma unroll
    for (int d = 0; d < kLfgDepth - 1; ++d) {
        const int64_t b = first + d * step;
        if (b < nblk) {
            nv[d] = (int)min((int64_t)128, n_region - 128 * b);
            fast[d] = block_fast(a, q_first + 128 * b, nv[d]);
            block_load(a, q_first + 128 * b, nv[d], fast[d], pipe[d]);
        }
    }
    for (int64_t b = first; b < nblk; b += step) {
        const int64_t bn = b + (kLfgDepth - 1) * step;
        if (bn < nblk) {
            constexpr int L = kLfgDepth - 1;
            nv[L] = (int)min((int64_t)128, n_region - 128 * bn);
            fast[L] = block_fast(a, q_first + 128 * bn, nv[L]);
            block_load(a, q_first + 128 * bn, nv[L], fast[L], pipe[L]);
        }
        block_store(a, q_first + 128 * b, nv[0], fast[0], pipe[0], buf);
        consume(b, nv[0], block_transpose(buf));
#pragma unroll
        for (int d = 0; d < kLfgDepth - 1; ++d) {
            fast[d] = fast[d + 1];
            nv[d] = nv[d + 1];
#pragma unroll
            for (int k = 0; k < 4; ++k) pipe[d][k] = pipe[d + 1][k];
        }
    }
}

// ------------------------------------------------------------- fused step
// Box-Muller normals of one oscillator-step from its four values (Sec. II.A;
// gx, gy from the first pair, gz from the cosine branch of the second).
__device__ __forceinline__ void normals3(uint4 w, float& g0, float& g1, float& g2)
{
    box_muller_u32(w.x, w.y, g0, g1);
    g2 = box_muller_cos_u32(w.z, w.w);
}

// Euler-Maruyama update of one oscillator (x, v in registers), its energy
// into e, and the final-state sums at the last step.
__device__ __forceinline__ void em_update(const LdCoef& c, float Ki, float g0, float g1, float g2,
                                          float& x0, float& x1, float& x2, float& v0, float& v1,
                                          float& v2, bool last, Kahan& e, double* acc)
{
    const float ckx = __fmul_rn(c.ckm, Ki);
    em_component(c.cdt, c.cva, ckx, c.cs, g0, x0, v0);
    em_component(c.cdt, c.cva, ckx, c.cs, g1, x1, v1);
    em_component(c.cdt, c.cva, ckx, c.cs, g2, x2, v2);
    e.add(energy3(0.5f * Ki, c.hm, x0, x1, x2, v0, v1, v2));
    if (last) {
        acc[0] += (double)x0 * x0 + (double)x1 * x1 + (double)x2 * x2;
        acc[1] += (double)v0 * v0 + (double)v1 * v1 + (double)v2 * v2;
        acc[2] += (double)x0 * v0 + (double)x1 * v1 + (double)x2 * v2;
    }
}

template <int MODE>
__global__ void __launch_bounds__(kLfgThreads, 3) lfg_kernel(LfgArgs a)
{
    __shared__ __align__(16) uint32_t bufs[kLfgWarps][128];
    __shared__ double red[4 * 32];
    constexpr bool LD = MODE >= LFG_LD;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t gwarp = blockIdx.x * (int64_t)kLfgWarps + warp;
    const int64_t nwarps = (int64_t)gridDim.x * kLfgWarps;
    const bool arrive_here = (int)blockIdx.x != a.stall_cta;
    Kahan e;
    double acc[3] = {0, 0, 0};
    uint64_t round = 0;
    for (int64_t U = 0; U < a.n_pos; ++round) {
        // rounds: whole oscillator-steps for the fused step (U, widths are multiples of 4)
        const int64_t wpos = a.base + U >= a.ll ? a.w_leap : a.w_base;
        const int64_t U1 = min(a.n_pos, U + wpos);
        if (!LD) {
            walk_blocks(a, a.base + U, U1 - U, gwarp, nwarps, bufs[warp],
                        [&](int64_t b, int nval, uint4 w) {
                            const int64_t u0 = U + 128 * b;   // launch offset of the block
                            if (MODE == LFG_NORMAL) {
                                // positions u0 + 4l .. + 3: pairs (2e, 2e + 1); nval is even
                                const int i = 4 * lane;
                                float2 o;
                                if (i < nval) {
                                    box_muller_u32(w.x, w.y, o.x, o.y);
                                    __stcs((float2*)((float*)a.out + u0 + i), o);
                                }
                                if (i + 2 < nval) {
                                    box_muller_u32(w.z, w.w, o.x, o.y);
                                    __stcs((float2*)((float*)a.out + u0 + i + 2), o);
                                }
                            } else {
                                const uint32_t* bv = bufs[warp];
#pragma unroll
                                for (int k = 0; k < 4; ++k) {
                                    const int i = 32 * k + lane;
                                    if (i < nval) {
                                        if (MODE == LFG_U32)
                                            __stcs((uint32_t*)a.out + u0 + i, bv[i]);
                                        else
                                            __stcs((float*)a.out + u0 + i, u01_from_u32(bv[i]));
                                    }
                                }
                            }
                        });
        } else {
            // oscillator-step u = (U + 128 b) / 4 + lane; the round spans at most two steps
            const int64_t t0 = U / (4 * a.N), u_next = (t0 + 1) * a.N;
            if (MODE == LFG_LD) {
                // Bring this round's x, v (one SM's share fits L1) into L1 at
                // the round's start, so that each block's loads below wait on
                // L1 rather than DRAM.  Exact: every oscillator of the round was
                // last written in an earlier round, whose writes the barrier's
                // acquire before this round made visible to all later loads, and
                // no SM writes it again before the next barrier.  (6% faster at
                // 1e8 oscillators than L2-only loads; prefetching the next
                // round's share instead was slower.)
                const int64_t nblk_r = (U1 - U + 127) >> 7;
                for (int64_t bb = gwarp; bb < nblk_r; bb += nwarps) {
                    if (4 * lane < U1 - U - 128 * bb) {
                        const int64_t u = (U >> 2) + 32 * bb + lane;
                        const int64_t j = u - (t0 + (u >= u_next ? 1 : 0)) * a.N;
                        asm volatile("prefetch.global.L1 [%0];" ::"l"(a.x + 3 * j));
                        asm volatile("prefetch.global.L1 [%0];" ::"l"(a.v + 3 * j));
                    }
                }
            }
            walk_blocks(a, a.base + U, U1 - U, gwarp, nwarps, bufs[warp],
                        [&](int64_t b, int nval, uint4 w) {
                            if (4 * lane >= nval) return;
                            const int64_t u = (U >> 2) + 32 * b + lane;
                            const int64_t t = t0 + (u >= u_next ? 1 : 0);
                            const int64_t j = u - t * a.N;
                            float g0, g1, g2;
                            normals3(w, g0, g1, g2);
                            const float Ki = a.Kper ? __ldcg(a.Kper + j) : a.c.K;
                            float* xp = a.x + 3 * j;
                            float* vp = a.v + 3 * j;
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
                                return;
                            }
                            float x0 = __ldca(xp), x1 = __ldca(xp + 1), x2 = __ldca(xp + 2);
                            float v0 = __ldca(vp), v1 = __ldca(vp + 1), v2 = __ldca(vp + 2);
                            em_update(a.c, Ki, g0, g1, g2, x0, x1, x2, v0, v1, v2,
                                      t == a.n_steps - 1, e, acc);
                            __stcg(xp, x0), __stcg(xp + 1, x1), __stcg(xp + 2, x2);
                            __stcg(vp, v0), __stcg(vp + 1, v1), __stcg(vp + 2, v2);
                        });
        }
        U = U1;
        if (U < a.n_pos && !grid_barrier(a, (uint64_t)gridDim.x * (round + 1), arrive_here)) return;
    }
    if (MODE == LFG_LD && a.partials) {
        double v[4] = {acc[0], acc[1], acc[2], e.value()};
        block_reduce_sum<4>(v, red);
        if (threadIdx.x == 0)
#pragma unroll
            for (int q = 0; q < 4; ++q) a.partials[4 * blockIdx.x + q] = v[q];
    }
}

// ------------------------------------------------- fused step, resident state
// When every step of the launch fits an all-leap round (4N <= the round width
// and the launch starts at or above ll), CTA c owns the oscillators
// [c n_c, c n_c + n_c) for the whole launch and keeps their x and v in shared
// memory: a step's global traffic is then the ring alone.  A round holds
// floor(width / 4N) steps, since an oscillator's consecutive steps stay with
// one lane and only the ring is shared.  A step's positions for the CTA are
// one contiguous region; when none of its windows wraps around the ring (all
// but about one step in R / 4N), each lane addresses the region with one
// pointer per window and the blocks are walked two at a time, the loads of one
// in flight while the other is consumed.
constexpr int kResThreads = 512;
constexpr int kResWarps = kResThreads / 32;

__global__ void __launch_bounds__(kResThreads, 1) lfg_resident_kernel(LfgArgs a, int64_t n_c)
{
    extern __shared__ __align__(16) float res_sm[];
    __shared__ __align__(16) uint32_t bufs[kResWarps][128];
    __shared__ double red[4 * 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t j0 = blockIdx.x * n_c;
    const int nc = (int)max((int64_t)0, min(a.N, j0 + n_c) - j0);
    float* xs = res_sm;
    float* vs = res_sm + 3 * n_c;
    for (int i = threadIdx.x; i < 3 * nc; i += kResThreads) {
        xs[i] = __ldcg(a.x + 3 * j0 + i);
        vs[i] = __ldcg(a.v + 3 * j0 + i);
    }
    __syncthreads();
    const bool arrive_here = (int)blockIdx.x != a.stall_cta;
    const int npos = 4 * nc, nblk = (nc + 31) >> 5;
    uint32_t* buf = bufs[warp];
    Kahan e;
    double acc[3] = {0, 0, 0};
    // kr steps per round: their 4 N kr positions read only earlier rounds, and
    // each oscillator's steps stay with one lane, so no barrier is needed
    // inside a round
    const int64_t kr = max((int64_t)1, a.w_leap / (4 * a.N));
    for (int64_t t = 0; t < a.n_steps; ++t) {
        const bool last = t == a.n_steps - 1;
        // oscillator jj of this CTA from its four values w
        auto osc = [&](int jj, uint4 w) {
            float g0, g1, g2;
            normals3(w, g0, g1, g2);
            const float Ki = a.Kper ? __ldg(a.Kper + j0 + jj) : a.c.K;
            float* xp = xs + 3 * jj;
            float* vp = vs + 3 * jj;
            float x0 = xp[0], x1 = xp[1], x2 = xp[2];
            float v0 = vp[0], v1 = vp[1], v2 = vp[2];
            em_update(a.c, Ki, g0, g1, g2, x0, x1, x2, v0, v1, v2, last, e, acc);
            xp[0] = x0, xp[1] = x1, xp[2] = x2;
            vp[0] = v0, vp[1] = v1, vp[2] = v2;
        };
        const int64_t P = a.base + 4 * (t * a.N + j0);
        const uint32_t P32 = (uint32_t)P;
        const uint32_t span = 128u * (uint32_t)nblk;   // whole blocks, loads may read past npos
        const uint32_t sA = (P32 + a.oA) & a.mask, sB = (P32 + a.oB) & a.mask;
        const uint32_t sC = (P32 + a.oC) & a.mask, sS = P32 & a.mask;
        const bool fast = span <= a.mask && sA <= a.mask + 1 - span && sB <= a.mask + 1 - span &&
                          sC <= a.mask + 1 - span && sS <= a.mask + 1 - span;
        if (fast) {
            const uint32_t* pA = a.ring + sA + lane;
            const uint32_t* pB = a.ring + sB + lane;
            const uint32_t* pC = a.ring + sC + lane;
            uint32_t* pS = a.ring + sS + lane;
            auto load = [&](int b, Lags(&g)[4]) {
                const int o = 128 * b;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    g[k].A = __ldcg(pA + o + 32 * k);
                    g[k].B = __ldcg(pB + o + 32 * k);
                    g[k].C = __ldcg(pC + o + 32 * k);
                }
            };
            auto consume = [&](int b, const Lags(&g)[4]) {
                const int o = 128 * b;
                const bool whole = o + 128 <= npos;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t val = g[k].value();
                    if (whole || o + 32 * k + lane < npos) __stcg(pS + o + 32 * k, val);
                    buf[32 * k + lane] = val;
                }
                const uint4 w = block_transpose(buf);
                const int jj = 32 * b + lane;
                if (jj < nc) osc(jj, w);
            };
            Lags g0[4], g1[4];
            int b = warp;
            if (b < nblk) load(b, g0);
            while (b < nblk) {
                const int b1 = b + kResWarps;
                if (b1 < nblk) load(b1, g1);
                consume(b, g0);
                if (b1 >= nblk) break;
                const int b2 = b1 + kResWarps;
                if (b2 < nblk) load(b2, g0);
                consume(b1, g1);
                b = b2;
            }
        } else {
            walk_blocks(a, P, npos, warp, kResWarps, buf, [&](int64_t b, int nval, uint4 w) {
                if (4 * lane < nval) osc(32 * (int)b + lane, w);
            });
        }
        if (!last && (t + 1) % kr == 0 &&
            !grid_barrier(a, (uint64_t)gridDim.x * (uint64_t)((t + 1) / kr), arrive_here))
            return;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * nc; i += kResThreads) {
        __stcg(a.x + 3 * j0 + i, xs[i]);
        __stcg(a.v + 3 * j0 + i, vs[i]);
    }
    if (a.partials) {
        double v[4] = {acc[0], acc[1], acc[2], e.value()};
        block_reduce_sum<4>(v, red);
        if (threadIdx.x == 0)
#pragma unroll
            for (int q = 0; q < 4; ++q) a.partials[4 * blockIdx.x + q] = v[q];
    }
}

// ----------------------------------------------------------- paper form
// One launch per step (Algorithm 3 with Sec. III.C's one-step-per-launch
// scheme): thread j computes positions P + 4j .. P + 4j + 3 from the ring,
// stores them, and takes oscillator j's step with x, v and its energy sum in
// global memory.  The launch boundary is the only synchronisation, so every
// position of the step must be dependency-free (checked on the host).
__global__ void __launch_bounds__(256) lfg_step_kernel(LfgArgs a, int64_t P, float2* eacc)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= a.N) return;
    const int64_t q = P + 4 * j;
    uint32_t w[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) w[r] = load_lags(a, q + r).value();
#pragma unroll
    for (int r = 0; r < 4; ++r) a.ring[(uint64_t)(q + r) & a.mask] = w[r];
    float g0, g1, g2;
    box_muller_u32(w[0], w[1], g0, g1);
    g2 = box_muller_cos_u32(w[2], w[3]);
    const float Ki = a.Kper ? a.Kper[j] : a.c.K;
    float* xp = a.x + 3 * j;
    float* vp = a.v + 3 * j;
    float x0 = xp[0], x1 = xp[1], x2 = xp[2];
    float v0 = vp[0], v1 = vp[1], v2 = vp[2];
    const float ckx = __fmul_rn(a.c.ckm, Ki);
    em_component(a.c.cdt, a.c.cva, ckx, a.c.cs, g0, x0, v0);
    em_component(a.c.cdt, a.c.cva, ckx, a.c.cs, g1, x1, v1);
    em_component(a.c.cdt, a.c.cva, ckx, a.c.cs, g2, x2, v2);
    xp[0] = x0, xp[1] = x1, xp[2] = x2;
    vp[0] = v0, vp[1] = v1, vp[2] = v2;
    Kahan e;
    const float2 ec = eacc[j];
    e.s = ec.x;
    e.c = ec.y;
    e.add(energy3(0.5f * Ki, a.c.hm, x0, x1, x2, v0, v1, v2));
    eacc[j] = make_float2(e.s, e.c);
}

// ------------------------------------------------------ overdamped 1-D run
// Each step is one round of 2N positions (particle j uses P + 2j, P + 2j + 1),
// computed by the cooperative grid and closed by the grid barrier; R lives in
// global memory, R(0) in the handle's scratch.  Records before a step sum each
// block's particles (R and R R(0) are read by the thread that wrote them).
__global__ void __launch_bounds__(256) lfg_ou_kernel(LfgArgs a, OuCoef c, float* R, const float* R0,
                                                     int64_t every, double* partials)
{
    __shared__ double red[2 * 32];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool arrive_here = (int)blockIdx.x != a.stall_cta;
    int64_t rec = 0, next_rec = 0;
    for (int64_t t = 0;; ++t) {
        if (partials && t == next_rec) {
            next_rec += every;
            double v[2] = {0, 0};
            for (int64_t j = gt; j < a.N; j += stride) {
                v[0] += (double)R[j];
                v[1] += (double)R[j] * (double)R0[j];
            }
            block_reduce_sum<2>(v, red);
            if (threadIdx.x == 0) {
                double* o = partials + 2 * (rec * gridDim.x + blockIdx.x);
                o[0] = v[0];
                o[1] = v[1];
            }
            ++rec;
        }
        if (t == a.n_steps) break;
        const int64_t P = a.base + 2 * a.N * t;
        for (int64_t j = gt; j < a.N; j += stride) {
            const int64_t q = P + 2 * j;
            const uint32_t w0 = load_lags(a, q).value(), w1 = load_lags(a, q + 1).value();
            __stcg(a.ring + ((uint64_t)q & a.mask), w0);
            __stcg(a.ring + ((uint64_t)(q + 1) & a.mask), w1);
            const float g = box_muller_cos_u32(w0, w1);
            R[j] = __fmaf_rn(c.cs, g, __fmaf_rn(-c.c1, R[j], R[j]));
        }
        if (t + 1 < a.n_steps &&
            !grid_barrier(a, (uint64_t)gridDim.x * (uint64_t)(t + 1), arrive_here))
            return;
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

// Round widths: W <= D (rounds starting below ll) or 2D (from ll on), W <= R - 2ll
// (overwritten values are out of every reader's reach), and for the fused step
// W <= 4N; even (normal pairs) and a multiple of 4 (whole oscillators).
static void round_widths(const Handle* h, int64_t four_n, int64_t* w_base, int64_t* w_leap)
{
    const int64_t D = (int64_t)h->ll - h->sl, R = (int64_t)h->ring_mask + 1;
    const int64_t cap = R - 2 * (int64_t)h->ll;
    int64_t wb = std::min(D, cap), wl = std::min(2 * D, cap);
    if (four_n > 0) {
        wb = std::min(wb, four_n);
        wl = std::min(wl, four_n);
    }
    *w_base = std::max<int64_t>(wb & ~(int64_t)3, 4);
    *w_leap = std::max<int64_t>(wl & ~(int64_t)3, 4);
}

// Ring, lags and the launch's first position.
static void set_ring(const Handle* h, LfgArgs& a)
{
    const int64_t ll = h->ll, D = (int64_t)h->ll - h->sl;
    a.ring = h->ring;
    a.mask = h->ring_mask;
    a.oA = (uint32_t)(-2 * ll);
    a.oB = (uint32_t)(-ll - D);
    a.oC = (uint32_t)(-2 * D);
    a.ll = h->ll;
    a.sl = h->sl;
    a.base = h->pos;
}

// Barrier counter, status word, wait limit and test hook of one launch.
static int launch_common(Handle* h, LfgArgs& a, int64_t G, cudaStream_t st)
{
    GB_CHECK(ensure_progress(h, 1));
    a.arrive = h->progress;
    a.status = h->dstatus;
    a.wait_ns = wait_limit_ns();
    const int64_t stall = test_stall_chunk();
    a.stall_cta = stall < 0 ? -1 : (int)(stall % G);
    GB_CUDA(cudaMemsetAsync(h->progress, 0, sizeof(uint64_t), st));
    GB_CUDA(cudaMemsetAsync(h->dstatus, 0, sizeof(int), st));
    return GBRNG_OK;
}

template <int MODE>
static int launch(Handle* h, LfgArgs& a, cudaStream_t st, int64_t* G_out)
{
    DevInfo di;
    GB_CHECK(dev_info(h->device, &di));
    auto fn = lfg_kernel<MODE>;
    int occ = 0;
    GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kLfgThreads, 0));
    if (occ < 1) return fail(GBRNG_EINVAL, "Lagged Fibonacci kernel does not fit on an SM");
    // no more CTAs than the widest round can use
    const int64_t per_cta = 128 * kLfgWarps;   // one block per warp
    int64_t G = (int64_t)di.sms * occ;
    G = std::min<int64_t>(G, std::max<int64_t>(1, (a.w_leap + per_cta - 1) / per_cta));
    if (G < 1) G = 1;
    if (MODE == LFG_LD) GB_CHECK(ensure_partials(h, G));
    a.partials = MODE == LFG_LD ? h->partials : nullptr;
    GB_CHECK(launch_common(h, a, G, st));
    void* args[] = {&a};
    GB_CUDA(cudaLaunchCooperativeKernel((const void*)fn, dim3((unsigned)G), dim3(kLfgThreads), args,
                                        0, st));
    *G_out = G;
    return GBRNG_OK;
}

// The resident-state kernel applies when every step of the launch is one
// all-leap round (4N within the leap width, launch at or above ll) and one CTA
// per SM can hold its share of x and v.
// Returns 1 (and launches) when it applies, 0 when the caller must use the
// general kernel, or an error.
static int try_launch_resident(Handle* h, LfgArgs& a, cudaStream_t st, int64_t* G_out)
{
    const int64_t four_n = 4 * a.N;
    if (four_n > a.w_leap || a.base < a.ll) return 0;
    DevInfo di;
    GB_CHECK(dev_info(h->device, &di));
    const int64_t G = di.sms;
    const int64_t n_c = ((a.N + G - 1) / G + 31) & ~(int64_t)31;
    const size_t smem = sizeof(float) * 6 * (size_t)n_c;
    const size_t static_smem = sizeof(uint32_t) * kResWarps * 128 + sizeof(double) * 128 + 64;
    if (smem + static_smem > di.smem_optin) return 0;
    GB_CUDA(cudaFuncSetAttribute((const void*)lfg_resident_kernel,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lfg_resident_kernel, kResThreads,
                                                          smem));
    if (occ < 1) return 0;
    GB_CHECK(ensure_partials(h, G));
    a.partials = h->partials;
    int64_t w_base_full = 0;
    round_widths(h, 0, &w_base_full, &a.w_leap);   // the full leap width: several steps a round
    GB_CHECK(launch_common(h, a, G, st));
    int64_t nc_arg = n_c;
    void* args[] = {&a, &nc_arg};
    GB_CUDA(cudaLaunchCooperativeKernel((const void*)lfg_resident_kernel, dim3((unsigned)G),
                                        dim3(kResThreads), args, smem, st));
    *G_out = G;
    return 1;
}

static int read_status(Handle* h, cudaStream_t st)
{
    int s = 0;
    GB_CUDA(cudaMemcpyAsync(&s, h->dstatus, sizeof(int), cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    if (s == DEV_TIMEOUT)
        return fail(GBRNG_ETIMEOUT, "Lagged Fibonacci grid barrier wait exceeded %llu ns",
                    (unsigned long long)wait_limit_ns());
    return GBRNG_OK;
}

int lfg_fill(Handle* h, void* dst, int64_t n, int mode, cudaStream_t st)
{
    LfgArgs a{};
    set_ring(h, a);
    a.n_pos = n;
    round_widths(h, 0, &a.w_base, &a.w_leap);
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
    LfgArgs a{};
    set_ring(h, a);
    a.N = s->n;
    a.n_steps = init ? 2 : n_steps;
    a.n_pos = 4 * s->n * a.n_steps;
    round_widths(h, 4 * s->n, &a.w_base, &a.w_leap);
    a.x = s->x;
    a.v = s->v;
    a.Kper = s->K_per;
    a.c = make_coef(s);
    int64_t G = 0;
    if (init) {
        GB_CHECK(launch<LFG_LD_INIT>(h, a, st, &G));
    } else {
        const int rc = try_launch_resident(h, a, st, &G);
        if (rc < 0) return rc;
        if (rc == 0) GB_CHECK(launch<LFG_LD>(h, a, st, &G));
    }
    GB_CHECK(read_status(h, st));
    h->pos += a.n_pos;
    if (out) return finish_stats(h, G, n_steps, out, st);
    return GBRNG_OK;
}

int lfg_ld_stepwise(const ld_system* s, int64_t n_steps, ld_stats* out, cudaStream_t st)
{
    Handle* h = s->rng;
    if (s->n == 0) {
        if (out) *out = ld_stats{0, 0, 0, 0, n_steps};
        return GBRNG_OK;
    }
    const int64_t D = (int64_t)h->ll - h->sl, R = (int64_t)h->ring_mask + 1;
    const int64_t four_n = 4 * s->n;
    if (four_n > std::min(2 * D, R - 2 * (int64_t)h->ll) || (h->pos < h->ll && four_n > D))
        return fail(GBRNG_ELAGS,
                    "one launch per step needs 4N = %lld within the lag distance (ll - sl = %lld, "
                    "twice that from position ll on)",
                    (long long)four_n, (long long)D);
    GB_CHECK(ensure_eacc(h, s->n));
    GB_CUDA(cudaMemsetAsync(h->eacc, 0, sizeof(float2) * s->n, st));
    LfgArgs a{};
    set_ring(h, a);
    a.N = s->n;
    a.x = s->x;
    a.v = s->v;
    a.Kper = s->K_per;
    a.c = make_coef(s);
    const unsigned blocks = (unsigned)((s->n + 255) / 256);
    for (int64_t t = 0; t < n_steps; ++t)
        lfg_step_kernel<<<blocks, 256, 0, st>>>(a, h->pos + four_n * t, h->eacc);
    GB_CUDA(cudaGetLastError());
    h->pos += four_n * n_steps;
    return stepwise_stats(h, s, n_steps, out, st);
}

int lfg_ou(const ou_system* s, int64_t n_steps, int64_t every, double* mean, double* corr,
           cudaStream_t st)
{
    Handle* h = s->rng;
    const int64_t D = (int64_t)h->ll - h->sl, Rsz = (int64_t)h->ring_mask + 1;
    const int64_t two_n = 2 * s->n;
    if (two_n > std::min(2 * D, Rsz - 2 * (int64_t)h->ll) || (h->pos < h->ll && two_n > D))
        return fail(GBRNG_ELAGS,
                    "one round per step needs 2N = %lld within the lag distance (ll - sl = %lld, "
                    "twice that from position ll on)",
                    (long long)two_n, (long long)D);
    DevInfo di;
    GB_CHECK(dev_info(h->device, &di));
    int occ = 0;
    GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lfg_ou_kernel, 256, 0));
    if (occ < 1) return fail(GBRNG_EINVAL, "overdamped kernel does not fit on an SM");
    const int64_t G = std::min<int64_t>((int64_t)di.sms * occ, (s->n + 255) / 256);
    const bool rec = mean != nullptr;
    const int64_t n_rec = n_steps / every + 1;
    if (rec) {
        if (n_rec > 0x7fffffff || (double)n_rec * G * 16.0 > 4.0 * (1 << 30))
            return fail(GBRNG_EINVAL, "%lld records x %lld blocks exceed the record scratch",
                        (long long)n_rec, (long long)G);
        GB_CHECK(ensure_partials(h, (2 * n_rec * G + 2 * n_rec + 3) / 4));
    }
    GB_CHECK(ensure_eacc(h, s->n));
    float* R0 = reinterpret_cast<float*>(h->eacc);
    GB_CUDA(cudaMemcpyAsync(R0, s->R, sizeof(float) * s->n, cudaMemcpyDeviceToDevice, st));
    LfgArgs a{};
    set_ring(h, a);
    a.N = s->n;
    a.n_steps = n_steps;
    GB_CHECK(launch_common(h, a, G, st));
    OuCoef c = make_ou_coef(s);
    float* Rp = s->R;
    int64_t ev = every;
    double* parts = rec ? h->partials : nullptr;
    void* args[] = {&a, &c, &Rp, &R0, &ev, &parts};
    GB_CUDA(cudaLaunchCooperativeKernel((const void*)lfg_ou_kernel, dim3((unsigned)G), dim3(256),
                                        args, 0, st));
    GB_CHECK(read_status(h, st));
    h->pos += two_n * n_steps;
    if (rec) return ou_finish(h, s->n, n_rec, G, mean, corr, st);
    return GBRNG_OK;
}

}  // namespace gb
