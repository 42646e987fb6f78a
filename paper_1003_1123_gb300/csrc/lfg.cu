// Additive Lagged Fibonacci generator shared by all threads (Algorithm 3):
//   x_p = x_{p-ll} + x_{p-D}  mod 2^32,   D = ll - sl.
//
// Leap.  Applying the recurrence k times (in shift-operator form,
// x = (E^{-ll} + E^{-D})^k x) gives
//   x_p = sum_{j=0..k} C(k, j) x_{p - (k-j) ll - j D}  mod 2^32,
// the same value with its nearest dependency k D back instead of D.  It holds
// at p whenever the recurrence holds at every index from p - (k-1) ll on.  The
// seeds x_{-ll..-1} are extended backwards with the recurrence run in reverse,
// x_q = x_{q+ll} - x_{q+sl}, down to x_{-K ll} (K = the ring's highest order,
// 2, or 4 when that order was set before the handle was created); the
// recurrence then holds from -(K-1) ll on, so every position p >= 0 may use
// any order k <= K.  A launch uses one order k in {1, 2, 4}: k + 1 lag reads
// per value.  Order 2 is the default everywhere: order 4 halves the barrier
// rounds but its two extra lag reads cost more than the barriers they save
// (measured on every launch kind).
//
// Ring.  Position p lives in slot p mod R of a ring of R >= K (ll + D) words
// (rounded up to 32 words: 40.3 MB for the last Table I row at K = 2).  Slot
// arithmetic is 32-bit: an offset below R is added with one conditional
// subtraction of R.  The first M = min(32768, R / 4) slots are mirrored after the
// ring (words R .. R + M - 1; every store to a slot below M also stores its
// mirror), so any window of at most M positions starting at slot s < R is the
// contiguous range [s, s + M) of the allocation: lag windows never wrap, and
// only the stores of a region that reaches the seam need per-value slots.
//
// Rounds.  A launch walks its positions in rounds of W consecutive positions
// with W <= k D, so no position of a round reads another, and W <= R - k ll,
// so no position of a round overwrites (slot p - R) a value this or a later
// round still reads (p - k ll at the farthest).  The persistent cooperative
// grid computes a round at once.  For the fused Langevin step a round also
// holds at most one step (W <= 4N), so each oscillator is updated at most
// once per round.  This is the paper's one-step-per-launch scheme (Sec.
// III.C) made exact for any N: the leap turns its race condition ll - sl > 4N
// into k (ll - sl) >= W.
//
// Between rounds.  With order 2 on the exact ring (R = 2(ll + D) + r, r <
// 32) each CTA waits only for the CTAs that computed what its next share
// reads: the readers of the value a store overwrites (position q - R) are the
// positions q - back_j - r, i.e. the producers of the lag windows the same
// positions read, so waiting for the owners of [q_lo - back_j - 32, q_hi -
// back_j) covers both read after write and write after read (and, in the
// fused step, the owners of the oscillators' previous step cover their x, v).
// Each CTA publishes its completed rounds in a counter of its own
// (st.release / ld.acquire).  Other launches (order 1 or 4, and resident
// launches with several steps a round) keep a grid barrier: an arrival
// counter.  Every wait is polled under a %globaltimer bound; a wait that runs
// out records GBRNG_ETIMEOUT and every CTA returns.
//
// Within a round a warp owns blocks of 128 consecutive positions (32
// oscillator-steps): lane l reads positions 32i + l of each lag window
// (coalesced, one pointer per window through the mirror), the new values go
// back to the ring the same way, and a per-warp shared-memory buffer hands
// lane l positions 4l..4l+3.
#include <algorithm>
#include <atomic>

#include "device.cuh"
#include "internal.cuh"

namespace gb {

enum { LFG_U32 = 0, LFG_UNIFORM = 1, LFG_NORMAL = 2, LFG_LD = 3, LFG_LD_INIT = 4 };

// Round kernel CTAs: 128 threads, eight a SM for the fused step and seven for
// the fills (up to 64 and 73 registers; a few bytes spill).  With per-CTA
// dataflow waits more, smaller CTAs overlap one CTA's wait with the others'
// work: against 256 x 3 on one GB300, 1e8 oscillators 1955 -> 1865 us per
// step, 1e7 175 -> 170, 2^30 fills 2.28 -> 2.22 ms (uniform) and 2.92 -> 2.83
// (normal); 64 x 16 and 512 x 2 were slower.
constexpr int kLfgThreads = 128;
template <int MODE>
constexpr int lfg_min_blocks() { return MODE >= LFG_LD ? 8 : 7; }
constexpr int kLfgWarps = kLfgThreads / 32;
constexpr int kLfgDepth = 2;     // blocks per warp with lag loads in flight
constexpr int kMaxOrder = 4;

struct LfgArgs {
    uint32_t* ring;                  // R + M words: the ring, then the mirror of its first M slots
    uint32_t R;                      // ring slots
    uint32_t M;                      // mirrored slots
    uint32_t off[kMaxOrder + 1];     // slot offset of leap term j: -((k-j) ll + j D) mod R
    uint32_t base_slot;              // slot of position `base`
    int32_t ll, sl;
    int64_t base;          // first position of this launch
    int64_t n_pos;         // positions of this launch
    int64_t N;             // LD: oscillators
    int64_t n_steps;       // LD: steps (init: 2)
    int64_t w;             // round width (positions)
    void* out;
    float* x;
    float* v;
    const float* Kper;
    LdCoef c;
    uint64_t* arrive;      // grid-barrier arrival counter (zeroed before launch; 64-bit, never wraps)
    uint64_t* prog;        // resident kernel, dataflow mode: steps each CTA has completed, or null
    int* status;
    uint64_t wait_ns;
    double* partials;      // [G][4]
    int stall_cta;         // test hook: this CTA never arrives (-1: none)
};

// s + o mod R for s, o < R (R < 2^31).
__host__ __device__ __forceinline__ uint32_t slot_add(uint32_t s, uint32_t o, uint32_t R)
{
    const uint32_t r = s + o;
    return r >= R ? r - R : r;
}

// Slot of position p (p >= -order_max ll).
static uint32_t slot_of(int64_t p, uint32_t R)
{
    const int64_t r = p % (int64_t)R;
    return (uint32_t)(r < 0 ? r + R : r);
}

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

// The k + 1 lag terms of one position, t[j] = x_{q - (k-j) ll - j D}, and the
// value they give: sum_j C(k, j) t[j] mod 2^32.
template <int K>
struct Lags {
    uint32_t t[K + 1];
    __device__ __forceinline__ uint32_t value() const
    {
        if (K == 1) return t[0] + t[1];
        if (K == 2) return t[0] + 2u * t[1] + t[2];
        return t[0] + t[4] + 4u * (t[1] + t[3]) + 6u * t[2];   // K == 4
    }
};

// Store val to slot e of the allocation (e < R + M), keeping the mirror: the
// primary slot of a mirror word and the mirror of a primary slot below M.
__device__ __forceinline__ void ring_store(const LfgArgs& a, uint32_t e, uint32_t val)
{
    __stcg(a.ring + e, val);
    if (e >= a.R)
        __stcg(a.ring + (e - a.R), val);
    else if (e < a.M)
        __stcg(a.ring + (e + a.R), val);
}

// A region of `span` slots from s needs no mirror bookkeeping when it lies in
// [M, R).
__device__ __forceinline__ bool plain_stores(const LfgArgs& a, uint32_t s, uint32_t span)
{
    return s >= a.M && s <= a.R - span;
}

// The lags of the position in slot s.
template <int K>
__device__ __forceinline__ Lags<K> load_lags(const LfgArgs& a, uint32_t s)
{
    Lags<K> g;
#pragma unroll
    for (int j = 0; j <= K; ++j) g.t[j] = __ldcg(a.ring + slot_add(s, a.off[j], a.R));
    return g;
}

// Issue the lag loads of lane's positions (slots s0 + 32i + lane, i < 4): each
// window is contiguous through the mirror (128 <= M), and the values past a
// partial block's end are read but not used.
template <int K>
__device__ __forceinline__ void block_load(const LfgArgs& a, uint32_t s0, Lags<K> (&g)[4])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j <= K; ++j) {
        const uint32_t* p = a.ring + slot_add(s0, a.off[j], a.R) + lane;
#pragma unroll
        for (int i = 0; i < 4; ++i) g[i].t[j] = __ldcg(p + 32 * i);
    }
}

// Store lane's values of slots s0 + 32i + lane (those below nval) to the ring
// and all four to the warp's buffer (buf[32i + lane]).
template <int K>
__device__ __forceinline__ void block_store(const LfgArgs& a, uint32_t s0, int nval,
                                            const Lags<K> (&g)[4], uint32_t* buf)
{
    const int lane = threadIdx.x & 31;
    if (nval == 128 && plain_stores(a, s0, 128)) {
        uint32_t* p = a.ring + s0 + lane;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t val = g[i].value();
            __stcg(p + 32 * i, val);
            buf[32 * i + lane] = val;
        }
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int e = 32 * i + lane;
            const uint32_t val = g[i].value();
            if (e < nval) ring_store(a, s0 + e, val);
            buf[e] = val;
        }
    }
}

// Lane l's four consecutive values (positions 4l .. 4l + 3 of the block).
__device__ __forceinline__ uint4 block_transpose(const uint32_t* buf)
{
    __syncwarp();
    const uint4 w = *reinterpret_cast<const uint4*>(buf + 4 * (threadIdx.x & 31));
    __syncwarp();
    return w;
}

// Walk this warp's blocks b = first, first + step, ... < min(nblk, end) of a region of
// n_region positions whose first position lives in slot s_first (block b
// starts 128 b later, 128 b < n_region <= R), with the lag loads of the next
// kLfgDepth - 1 blocks in flight while one is consumed.  Positions of one
// round never read each other, so the early loads are exact.
// consume(b, nval, w) receives lane's four values after they are stored.
template <int K, class F>
__device__ __forceinline__ void walk_blocks(const LfgArgs& a, uint32_t s_first, int64_t n_region,
                                            int64_t first, int64_t step, int64_t end, uint32_t* buf,
                                            F&& consume)
{
    const int64_t nblk = min((n_region + 127) >> 7, end);   // blocks first, first + step, ... < end
    Lags<K> pipe[kLfgDepth][4];
    int nv[kLfgDepth];
    uint32_t sl[kLfgDepth];
#pragma unroll
    for (int d = 0; d < kLfgDepth - 1; ++d) {
        const int64_t b = first + d * step;
        if (b < nblk) {
            nv[d] = (int)min((int64_t)128, n_region - 128 * b);
            sl[d] = slot_add(s_first, (uint32_t)(128 * b), a.R);
            block_load<K>(a, sl[d], pipe[d]);
        }
    }
    for (int64_t b = first; b < nblk; b += step) {
        const int64_t bn = b + (kLfgDepth - 1) * step;
        if (bn < nblk) {
            constexpr int L = kLfgDepth - 1;
            nv[L] = (int)min((int64_t)128, n_region - 128 * bn);
            sl[L] = slot_add(s_first, (uint32_t)(128 * bn), a.R);
            block_load<K>(a, sl[L], pipe[L]);
        }
        block_store<K>(a, sl[0], nv[0], pipe[0], buf);
        consume(b, nv[0], block_transpose(buf));
#pragma unroll
        for (int d = 0; d < kLfgDepth - 1; ++d) {
            nv[d] = nv[d + 1];
            sl[d] = sl[d + 1];
#pragma unroll
            for (int i = 0; i < 4; ++i) pipe[d][i] = pipe[d + 1][i];
        }
    }
}

// ------------------------------------------------------------- fused step
// Box-Muller normals of one oscillator-step from its four values (Sec. II.A;
// gx, gy from the first pair, gz from the cosine branch of the second).
__device__ __forceinline__ void normals3(uint4 w, float& g0, float& g1, float& g2)
{
    box_muller3_u32(w.x, w.y, w.z, w.w, g0, g1, g2);
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

// Dataflow wait of the round kernel (order 2 on the exact ring, a.prog set).
// In this mode CTA c owns the contiguous blocks [c B / G, (c + 1) B / G) of each
// round of B blocks, and publishes prog[c] = rounds it has completed.  Its
// share [q_lo, q_hi) (launch offsets) of round r reads the lag windows
// [q - back_j] (back_j = (2-j) ll + j D), all in earlier rounds (W <= 2D); with
// the exact ring the reads of the values its stores overwrite are the
// positions q - back_j - r (r < 32); and in the fused step its oscillators'
// x, v were last written one step (4N >= W) earlier.  So the CTA waits until
// the owners of [q_lo - back_j - 32, q_hi - back_j) for the three windows, and
// of [q_lo - 4N, q_hi - 4N) in the fused step, have completed those rounds:
// threads 4j .. 4j + 3 each take every fourth owner of window j.  Bounded by
// the launch's wait limit; returns false on failure (GBRNG_ETIMEOUT recorded).
__device__ bool round_dataflow_wait(const LfgArgs& a, int64_t q_lo, int64_t q_hi, bool ld)
{
    const int nwin = ld ? 4 : 3;
    if (threadIdx.x >= 4 * nwin) return true;
    const int jw = threadIdx.x >> 2, m = threadIdx.x & 3;
    const int64_t D = (int64_t)a.ll - a.sl;
    const int64_t back = jw < 3 ? (int64_t)(2 - jw) * a.ll + (int64_t)jw * D : 4 * a.N;
    int64_t lo = q_lo - back - 32;
    const int64_t hi = q_hi - back;
    if (lo < 0) lo = 0;   // positions before the launch are complete
    if (hi <= lo) return true;
    const int64_t G = gridDim.x;
    // (round, owner CTA) of launch offset q as one increasing index
    auto owner = [&](int64_t q) {
        const int64_t r = q / a.w, blk = (q - r * a.w) >> 7;
        const int64_t nb = (min(a.w, a.n_pos - r * a.w) + 127) >> 7;
        return r * G + ((blk + 1) * G - 1) / nb;
    };
    const int64_t L0 = owner(lo), L1 = owner(hi - 1);
    const uint64_t deadline = global_ns() + a.wait_ns;
    for (int64_t L = L0 + m; L <= L1; L += 4) {
        const uint64_t* f = a.prog + (L % G);
        const uint64_t need = (uint64_t)(L / G) + 1;
        for (uint32_t n = 1; ld_relaxed_u64(f) < need; ++n) {
            if ((n & 15u) == 0) {
                if (ld_volatile_i32(a.status) != DEV_OK) return false;
                if (global_ns() > deadline) {
                    atomicCAS(a.status, DEV_OK, DEV_TIMEOUT);
                    return false;
                }
            }
        }
        (void)ld_acquire_u64(f);
    }
    return true;
}

template <int MODE, int K>
__global__ void __launch_bounds__(kLfgThreads, lfg_min_blocks<MODE>()) lfg_kernel(LfgArgs a)
{
    __shared__ __align__(16) uint32_t bufs[kLfgWarps][128];
    __shared__ double red[4 * 32];
    constexpr bool LD = MODE >= LFG_LD;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t gwarp = blockIdx.x * (int64_t)kLfgWarps + warp;
    const int64_t nwarps = (int64_t)gridDim.x * kLfgWarps;
    const bool arrive_here = (int)blockIdx.x != a.stall_cta;
    __shared__ int s_df_fail;
    if (threadIdx.x == 0) s_df_fail = 0;
    Kahan e;
    double acc[3] = {0, 0, 0};
    uint64_t round = 0;
    uint32_t s_round = a.base_slot;   // slot of position base + U
    for (int64_t U = 0; U < a.n_pos; ++round) {
        // rounds: whole oscillator-steps for the fused step (U, widths are multiples of 4)
        const int64_t U1 = min(a.n_pos, U + a.w);
        // this warp's blocks of the round: with dataflow waits the CTA's
        // contiguous share, walked by its warps; else every warp of the grid
        // strided over the whole round
        const int64_t nblk_r = (U1 - U + 127) >> 7;
        int64_t first = gwarp, step = nwarps, end = nblk_r;
        if (a.prog) {
            const int64_t b0 = blockIdx.x * nblk_r / gridDim.x;
            end = (blockIdx.x + 1) * nblk_r / gridDim.x;
            first = b0 + warp;
            step = kLfgWarps;
            __syncthreads();   // s_df_fail written before any thread reads it below
            if (!round_dataflow_wait(a, U + 128 * b0, min(U1, U + 128 * end), LD)) s_df_fail = 1;
            __syncthreads();
            if (s_df_fail) return;
        }
        if (!LD) {
            walk_blocks<K>(a, s_round, U1 - U, first, step, end, bufs[warp],
                           [&](int64_t b, int nval, uint4 w) {
                               const int64_t u0 = U + 128 * b;   // launch offset of the block
                               if (MODE == LFG_NORMAL) {
                                   // positions u0 + 4l .. + 3: pairs (2e, 2e + 1); nval is even
                                   // (both pairs in the paired instructions' lanes; past
                                   // nval the values are computed and dropped)
                                   const int i = 4 * lane;
                                   float2 ga, gb;
                                   box_muller_2pairs_u32(w.x, w.y, w.z, w.w, ga, gb);
                                   if (i < nval) __stcs((float2*)((float*)a.out + u0 + i), ga);
                                   if (i + 2 < nval) __stcs((float2*)((float*)a.out + u0 + i + 2), gb);
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
                for (int64_t bb = first; bb < end; bb += step) {
                    if (4 * lane < U1 - U - 128 * bb) {
                        const int64_t u = (U >> 2) + 32 * bb + lane;
                        const int64_t j = u - (t0 + (u >= u_next ? 1 : 0)) * a.N;
                        asm volatile("prefetch.global.L1 [%0];" ::"l"(a.x + 3 * j));
                        asm volatile("prefetch.global.L1 [%0];" ::"l"(a.v + 3 * j));
                    }
                }
            }
            walk_blocks<K>(a, s_round, U1 - U, first, step, end, bufs[warp],
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
        s_round = slot_add(s_round, (uint32_t)(U1 - U), a.R);
        U = U1;
        if (a.prog) {
            // publish: every ring (and x, v) store of this CTA's share is done
            __syncthreads();
            if (threadIdx.x == 0 && arrive_here) st_release_u64(a.prog + blockIdx.x, round + 1);
        } else if (U < a.n_pos &&
                   !grid_barrier(a, (uint64_t)gridDim.x * (round + 1), arrive_here)) {
            return;
        }
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
// Dataflow wait of the resident kernel (order 2 on an exact ring of R =
// 2(ll + D) + r slots, r < 32).  CTA c's step t reads the lag windows
// [q - back_j] of its positions q (back_j = (2-j) ll + j D), all in earlier
// steps (4N <= 2D).  Its stores overwrite the values of positions q - R, whose
// only readers are the positions q - R + back_j = q - back_j - r: so once the
// CTAs that computed the positions [q_lo - back_j - 32, q_hi - back_j) have
// published, both the values this step reads (read after write) and the reads
// of the values it overwrites (write after read) are complete.  The wait comes
// once a round, for all kr steps of the round at once (their windows lie in
// earlier rounds, 4N kr <= 2D), and each CTA publishes prog[c] = steps done at
// the round's end; a producer's step s is complete once prog[c] >= s + 1.  The
// (step, window, producer) triples are spread over the CTA's threads; every
// poll is bounded by the launch's wait limit.  Returns false on failure
// (GBRNG_ETIMEOUT recorded).
template <int K>
__device__ bool dataflow_wait(const LfgArgs& a, int64_t t, int64_t kr, int64_t j0, int nc,
                              int64_t n_c)
{
    // thread i takes step t + i / 12 (and every T / 12 steps after), window
    // (i % 12) / 4, every fourth producer from i % 4
    constexpr int kPer = 4 * (K + 1);
    const int64_t four_n = 4 * a.N, span = 4 * n_c, ceff = (a.N + n_c - 1) / n_c;
    const uint64_t deadline = global_ns() + a.wait_ns;
    const int jw = (threadIdx.x % kPer) >> 2, m = threadIdx.x & 3;
    const int64_t back = (int64_t)(K - jw) * a.ll + (int64_t)jw * (a.ll - a.sl);
    for (int64_t o = threadIdx.x / kPer; o < kr; o += blockDim.x / kPer) {
        const int64_t q0 = a.base + 4 * ((t + o) * a.N + j0);
        int64_t lo = q0 - back - 32;
        const int64_t hi = q0 + 4 * (int64_t)nc - back;
        if (lo < a.base) lo = a.base;   // positions before the launch are complete
        if (hi <= lo) continue;
        const int64_t r0 = lo - a.base, r1 = hi - 1 - a.base;
        const int64_t L0 = (r0 / four_n) * ceff + (r0 % four_n) / span;
        const int64_t L1 = (r1 / four_n) * ceff + (r1 % four_n) / span;
        for (int64_t L = L0 + m; L <= L1; L += 4) {
            const uint64_t* f = a.prog + (L % ceff);
            const uint64_t need = (uint64_t)(L / ceff) + 1;
            for (uint32_t n = 1; ld_relaxed_u64(f) < need; ++n) {
                if ((n & 15u) == 0) {
                    if (ld_volatile_i32(a.status) != DEV_OK) return false;
                    if (global_ns() > deadline) {
                        atomicCAS(a.status, DEV_OK, DEV_TIMEOUT);
                        return false;
                    }
                }
            }
            (void)ld_acquire_u64(f);
        }
    }
    return true;
}

// When every step of the launch fits a round (4N <= the round width) and the
// CTAs' shares of x and v fit in shared memory, CTA c owns the oscillators
// [c n_c, c n_c + n_c) for the whole launch and keeps their x and v in shared
// memory: a step's global traffic is then the ring alone.  A round holds
// floor(width / 4N) steps, since an oscillator's consecutive steps stay with
// one lane and only the ring is shared.  A step's positions for the CTA are
// one contiguous region of at most M slots, so each lane addresses each of its
// windows with one pointer (through the mirror), and the blocks are walked two
// at a time, the loads of one in flight while the other is consumed.  (Before
// the mirror, a region whose window wrapped took a slower per-block path;
// with 152 CTAs about one did so every step and held up the barrier: 13.2
// against 11.6 us per step at 1e6 oscillators on a 40 MB ring.)
// CTA size T: 512 or 640 threads, whichever leaves fewer of the CTA's
// 32-oscillator blocks per warp in a step (ties: 512).  At 1e6 oscillators
// (206 blocks a CTA) 640 threads take 11.6 us per step against 12.2 with 512
// and 11.7 with 768 (same GB300, same ring); where both sizes leave the same
// count (1e5: 21 blocks, two per warp at most either way) the smaller CTA
// has less to synchronise.
template <int K, int T>
__global__ void __launch_bounds__(T, 1) lfg_resident_kernel(LfgArgs a, int64_t n_c)
{
    constexpr int kResThreads = T;
    constexpr int kResWarps = T / 32;
    extern __shared__ __align__(16) float res_sm[];
    __shared__ __align__(16) uint32_t bufs[kResWarps][128];
    __shared__ double red[4 * 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t j0 = blockIdx.x * n_c;
    const int nc = (int)max((int64_t)0, min(a.N, j0 + n_c) - j0);
    __shared__ int s_df_fail;
    float* xs = res_sm;
    float* vs = res_sm + 3 * n_c;
    if (threadIdx.x == 0) s_df_fail = 0;
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
    const int64_t kr = max((int64_t)1, a.w / (4 * a.N));
    const uint32_t step_slots = (uint32_t)(4 * a.N);   // 4N <= w < R
    // slot of this CTA's first position in step t (4 j0 <= 4N < R)
    uint32_t sP = slot_add(a.base_slot, (uint32_t)(4 * min(j0, a.N)), a.R);
    for (int64_t t = 0; t < a.n_steps; ++t) {
        const bool last = t == a.n_steps - 1;
        if (a.prog && t % kr == 0) {
            // the round's kr steps read only earlier rounds
            const int64_t krr = min(kr, a.n_steps - t);
            if (nc > 0 && !dataflow_wait<K>(a, t, krr, j0, nc, n_c)) s_df_fail = 1;
            __syncthreads();
            if (s_df_fail) return;
        }
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
        // every window of the step's region is contiguous through the mirror
        // (whole blocks: loads may read up to 127 values past npos, span <= M)
        const uint32_t span = 128u * (uint32_t)nblk;
        const bool plain = plain_stores(a, sP, span);
        const uint32_t* pw[K + 1];
#pragma unroll
        for (int j = 0; j <= K; ++j) pw[j] = a.ring + slot_add(sP, a.off[j], a.R) + lane;
        uint32_t* pS = a.ring + sP + lane;
        auto load = [&](int b, Lags<K>(&g)[4]) {
            const int o = 128 * b;
#pragma unroll
            for (int j = 0; j <= K; ++j)
#pragma unroll
                for (int i = 0; i < 4; ++i) g[i].t[j] = __ldcg(pw[j] + o + 32 * i);
        };
        auto consume = [&](int b, const Lags<K>(&g)[4]) {
            const int o = 128 * b;
            const bool whole = o + 128 <= npos;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint32_t val = g[i].value();
                const int e = o + 32 * i + lane;
                if (whole || e < npos) {
                    if (plain)
                        __stcg(pS + o + 32 * i, val);
                    else
                        ring_store(a, sP + e, val);
                }
                buf[32 * i + lane] = val;
            }
            const uint4 w = block_transpose(buf);
            const int jj = 32 * b + lane;
            if (jj < nc) osc(jj, w);
        };
        Lags<K> g0[4], g1[4];
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
        sP = slot_add(sP, step_slots, a.R);
        if (a.prog) {
            // publish at the round's end: every ring store of its steps is done
            if ((t + 1) % kr == 0 || last) {
                __syncthreads();
                if (threadIdx.x == 0 && arrive_here)
                    st_release_u64(a.prog + blockIdx.x, (uint64_t)t + 1);
            }
        } else if (!last && (t + 1) % kr == 0 &&
                   !grid_barrier(a, (uint64_t)gridDim.x * (uint64_t)((t + 1) / kr), arrive_here)) {
            return;
        }
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
// scheme): thread j computes positions P + 4j .. P + 4j + 3 (slots from sP)
// from the ring, stores them, and takes oscillator j's step with x, v and its
// energy sum in global memory.  The launch boundary is the only
// synchronisation, so every position of the step must be dependency-free
// (checked on the host).
template <int K>
__global__ void __launch_bounds__(256) lfg_step_kernel(LfgArgs a, uint32_t sP, float2* eacc)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= a.N) return;
    const uint32_t s = slot_add(sP, (uint32_t)(4 * j), a.R);   // 4j < 4N < R
    uint32_t w[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) w[r] = load_lags<K>(a, slot_add(s, r, a.R)).value();
#pragma unroll
    for (int r = 0; r < 4; ++r) ring_store(a, slot_add(s, r, a.R), w[r]);
    float g0, g1, g2;
    box_muller3_u32(w[0], w[1], w[2], w[3], g0, g1, g2);
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
template <int K>
__global__ void __launch_bounds__(256) lfg_ou_kernel(LfgArgs a, OuCoef c, float* R, const float* R0,
                                                     int64_t every, double* partials)
{
    __shared__ double red[2 * 32];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool arrive_here = (int)blockIdx.x != a.stall_cta;
    const uint32_t step_slots = (uint32_t)(2 * a.N);   // 2N <= w < ring size
    uint32_t sP = a.base_slot;                          // slot of the step's first position
    // kr steps a round: their kr 2N positions read only earlier rounds, and a
    // particle's steps stay with one thread, so the barrier comes once a round
    // (records are per-block sums of the block's own particles)
    const int64_t kr = max((int64_t)1, a.w / (2 * a.N));
    int64_t rec = 0, next_rec = 0;
    if (a.N <= stride) {
        // one particle a thread: R stays in a register, and inside a round the
        // next step's lags (all in earlier rounds) load while this step computes
        const bool live = gt < a.N;
        float Rj = live ? R[gt] : 0.f;
        const float R0j = live ? R0[gt] : 0.f;
        Lags<K> c0, c1, n0, n1;
        for (int64_t t = 0;; ++t) {
            if (partials && t == next_rec) {
                next_rec += every;
                double v[2] = {(double)Rj, (double)Rj * (double)R0j};
                block_reduce_sum<2>(v, red);
                if (threadIdx.x == 0) {
                    double* o = partials + 2 * (rec * gridDim.x + blockIdx.x);
                    o[0] = v[0];
                    o[1] = v[1];
                }
                ++rec;
            }
            if (t == a.n_steps) break;
            const uint32_t s0 = slot_add(sP, (uint32_t)(2 * gt), a.R), s1 = slot_add(s0, 1u, a.R);
            if (t % kr == 0 && live) {   // first step of a round: nothing loaded ahead
                c0 = load_lags<K>(a, s0);
                c1 = load_lags<K>(a, s1);
            }
            const bool ahead = live && (t + 1) % kr != 0 && t + 1 < a.n_steps;
            if (ahead) {
                const uint32_t u0 = slot_add(s0, step_slots, a.R);
                n0 = load_lags<K>(a, u0);
                n1 = load_lags<K>(a, slot_add(u0, 1u, a.R));
            }
            if (live) {
                const uint32_t w0 = c0.value(), w1 = c1.value();
                ring_store(a, s0, w0);
                ring_store(a, s1, w1);
                Rj = __fmaf_rn(c.cs, box_muller_cos_u32(w0, w1), __fmaf_rn(-c.c1, Rj, Rj));
            }
            if (ahead) c0 = n0, c1 = n1;
            sP = slot_add(sP, step_slots, a.R);
            if (t + 1 < a.n_steps && (t + 1) % kr == 0 &&
                !grid_barrier(a, (uint64_t)gridDim.x * (uint64_t)((t + 1) / kr), arrive_here))
                return;
        }
        if (live) R[gt] = Rj;
        return;
    }
    // several particles a thread: one step a round (packing steps measured
    // slower here: 10.1 against 9.3 ms per 1000 steps at 1e6)
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
        for (int64_t j = gt; j < a.N; j += stride) {
            const uint32_t s0 = slot_add(sP, (uint32_t)(2 * j), a.R), s1 = slot_add(s0, 1u, a.R);
            const uint32_t w0 = load_lags<K>(a, s0).value(), w1 = load_lags<K>(a, s1).value();
            ring_store(a, s0, w0);
            ring_store(a, s1, w1);
            const float g = box_muller_cos_u32(w0, w1);
            R[j] = __fmaf_rn(c.cs, g, __fmaf_rn(-c.c1, R[j], R[j]));
        }
        sP = slot_add(sP, step_slots, a.R);
        if (t + 1 < a.n_steps &&
            !grid_barrier(a, (uint64_t)gridDim.x * (uint64_t)(t + 1), arrive_here))
            return;
    }
}

// Seeds: the value at position w - ll (w = 0..ll-1) is the low half of
// SplitMix64 at counter w, and x_{-ll} is forced odd.  Positions -K ll <= q <
// 0 live in slot q + R.
__global__ void lfg_seed_kernel(uint64_t seed, int32_t ll, LfgArgs a)
{
    const int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (w >= ll) return;
    uint32_t v = (uint32_t)splitmix64_at(seed, (uint64_t)w);
    if (w == 0) v |= 1u;
    ring_store(a, a.R - (uint32_t)ll + (uint32_t)w, v);
}

// The recurrence run backwards, x_q = x_{q+ll} - x_{q+sl}, for q in
// [q_hi - count, q_hi): every read lies at q_hi or above (count <= sl).
__global__ void lfg_extend_kernel(LfgArgs a, int64_t q_hi, int64_t count)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int64_t q = q_hi - count + i;
    const uint32_t R = a.R;
    ring_store(a, (uint32_t)(q + R),
               a.ring[(uint32_t)(q + a.ll + R)] - a.ring[(uint32_t)(q + a.sl + R)]);
}

static void set_ring(const Handle* h, LfgArgs& a, int k);

int lfg_seed(Handle* h, cudaStream_t st)
{
    h->pos = 0;
    const int T = 256;
    LfgArgs a{};
    set_ring(h, a, 1);
    lfg_seed_kernel<<<(unsigned)((h->ll + T - 1) / T), T, 0, st>>>(h->seed, h->ll, a);
    GB_CUDA(cudaGetLastError());
    // x_{-K ll} .. x_{-ll-1}, in rounds of sl positions from -ll downwards
    const int64_t lo = -(int64_t)h->order_max * h->ll;
    for (int64_t q_hi = -(int64_t)h->ll; q_hi > lo;) {
        const int64_t cnt = std::min<int64_t>(h->sl, q_hi - lo);
        lfg_extend_kernel<<<(unsigned)((cnt + T - 1) / T), T, 0, st>>>(a, q_hi, cnt);
        q_hi -= cnt;
    }
    GB_CUDA(cudaGetLastError());
    return GBRNG_OK;
}

// ------------------------------------------------------------- host side
// Leap order of a launch: the process-wide setting, else the given default,
// at most the highest order the handle's ring serves.
static std::atomic<int> g_lfg_order{0};

int lfg_order_for_new_handle() { return g_lfg_order.load() == 4 ? 4 : 2; }

static int pick_order(const Handle* h, int dflt)
{
    const int o = g_lfg_order.load();
    return std::min(o ? o : dflt, h->order_max);
}

// Round width for order k: W <= k D (no position of a round reads another),
// W <= R - k ll (no overwritten value is still to be read), and for the fused
// step W <= 4N (multiple of 4: whole oscillators; even: normal pairs).
static int64_t round_width(const Handle* h, int k, int64_t four_n)
{
    const int64_t D = (int64_t)h->ll - h->sl, R = (int64_t)h->ring_size;
    int64_t w = std::min<int64_t>((int64_t)k * D, R - (int64_t)k * h->ll);
    if (four_n > 0) w = std::min(w, four_n);
    return std::max<int64_t>(w & ~(int64_t)3, 4);
}

// Ring, order-k lag offsets and the launch's first position.
static void set_ring(const Handle* h, LfgArgs& a, int k)
{
    const int64_t ll = h->ll, D = (int64_t)h->ll - h->sl, R = (int64_t)h->ring_size;
    a.ring = h->ring;
    a.R = h->ring_size;
    a.M = ring_mirror(h->ring_size);
    for (int j = 0; j <= kMaxOrder; ++j) {
        const int64_t back = (int64_t)(k - j) * ll + (int64_t)j * D;
        a.off[j] = j <= k ? (uint32_t)((R - back % R) % R) : 0u;
    }
    a.ll = h->ll;
    a.sl = h->sl;
    a.base = h->pos;
    a.base_slot = slot_of(h->pos, h->ring_size);
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

// Round kernel synchronisation: per-CTA dataflow waits (order 2 on the exact
// ring; each CTA a contiguous share of every round) instead of the grid
// barrier between rounds, where a round fills the whole resident grid.  On
// narrower rounds the barrier is faster (measured, order 2, ms per the run:
// row 0 at 1e3 oscillators 4.35 against 5.82 per 1000 steps, row 3 at 1e6 559
// against 679 per 1000, row 6 at 1e6 (304 CTAs a round) 82.6 against 106.4 per
// 20 steps); on full-grid rounds the dataflow wait is faster (rows 7-9: 29.9,
// 27.3, 54.3 against 39.1, 36.9, 66.6 per 20 steps at 1e6-3e6).
constexpr bool kRoundDataflow = true;

template <int MODE, int K>
static int launch_k(Handle* h, LfgArgs& a, cudaStream_t st, int64_t* G_out)
{
    DevInfo di;
    GB_CHECK(dev_info(h->device, &di));
    auto fn = lfg_kernel<MODE, K>;
    int occ = 0;
    GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kLfgThreads, 0));
    if (occ < 1) return fail(GBRNG_EINVAL, "Lagged Fibonacci kernel does not fit on an SM");
    // no more CTAs than the widest round can use
    const int64_t per_cta = 128 * kLfgWarps;   // one block per warp
    int64_t G = (int64_t)di.sms * occ;
    G = std::min<int64_t>(G, std::max<int64_t>(1, (a.w + per_cta - 1) / per_cta));
    if (G < 1) G = 1;
    if (MODE == LFG_LD) GB_CHECK(ensure_partials(h, G));
    a.partials = MODE == LFG_LD ? h->partials : nullptr;
    const bool full_grid = G == (int64_t)di.sms * occ;
    const bool dataflow = kRoundDataflow && K == 2 && h->order_max == 2 && full_grid;
    if (dataflow) GB_CHECK(ensure_progress(h, 1 + G));   // before launch_common takes [0]
    GB_CHECK(launch_common(h, a, G, st));
    a.prog = nullptr;
    if (dataflow) {
        a.prog = h->progress + 1;
        GB_CUDA(cudaMemsetAsync(a.prog, 0, sizeof(uint64_t) * G, st));
    }
    void* args[] = {&a};
    GB_CUDA(cudaLaunchCooperativeKernel((const void*)fn, dim3((unsigned)G), dim3(kLfgThreads), args,
                                        0, st));
    *G_out = G;
    return GBRNG_OK;
}

template <int MODE>
static int launch(Handle* h, LfgArgs& a, int k, cudaStream_t st, int64_t* G_out)
{
    if (k == 1) return launch_k<MODE, 1>(h, a, st, G_out);
    if (k == 2) return launch_k<MODE, 2>(h, a, st, G_out);
    return launch_k<MODE, 4>(h, a, st, G_out);
}

// The resident-state kernel applies when every step of the launch fits one
// round (4N within the width) and one CTA per SM can hold its share of x and
// v.  Returns 1 (and launches) when it applies, 0 when the caller must use the
// general kernel, or an error.
// Resident kernel synchronisation: per-CTA dataflow waits (order 2 on the
// exact ring) instead of the grid barrier where every round is one step (8N >
// width).  Same GB300: 11.36 against 11.90 us per step at 1e6 oscillators,
// 7.75 against 8.08 at 6e5.  Where a round holds several steps the barrier
// stays: even waiting once a round, the dataflow polls cost more than the
// barrier there (1e5: 2.07 against 1.89 ms per 1000 steps; 1e4: 1.72 against
// 1.55; equal at 5e5).
constexpr bool kResDataflow = true;

template <int K, int T>
static int try_launch_resident_k(Handle* h, LfgArgs& a, cudaStream_t st, int64_t* G_out)
{
    constexpr int kResThreads = T;
    constexpr int kResWarps = T / 32;
    a.w = round_width(h, K, 0);   // the full width: several steps a round
    if (4 * a.N > a.w) return 0;
    DevInfo di;
    GB_CHECK(dev_info(h->device, &di));
    const int64_t G = di.sms;
    const int64_t n_c = ((a.N + G - 1) / G + 31) & ~(int64_t)31;
    if (4 * n_c > (int64_t)a.M) return 0;   // a CTA's step region must fit the mirror
    const size_t smem = sizeof(float) * 6 * (size_t)n_c;
    const size_t static_smem = sizeof(uint32_t) * kResWarps * 128 + sizeof(double) * 128 + 64;
    if (smem + static_smem > di.smem_optin) return 0;
    auto fn = lfg_resident_kernel<K, T>;
    GB_CUDA(cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    int occ = 0;
    GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kResThreads, smem));
    if (occ < 1) return 0;
    GB_CHECK(ensure_partials(h, G));
    a.partials = h->partials;
    const bool dataflow = kResDataflow && K == 2 && h->order_max == 2 && 8 * a.N > a.w;
    // per-CTA completed-step counters after the barrier counter (grown before
    // launch_common takes the barrier counter's address)
    if (dataflow) GB_CHECK(ensure_progress(h, 1 + G));
    GB_CHECK(launch_common(h, a, G, st));
    a.prog = nullptr;
    if (dataflow) {
        a.prog = h->progress + 1;
        GB_CUDA(cudaMemsetAsync(a.prog, 0, sizeof(uint64_t) * G, st));
    }
    int64_t nc_arg = n_c;
    void* args[] = {&a, &nc_arg};
    GB_CUDA(cudaLaunchCooperativeKernel((const void*)fn, dim3((unsigned)G), dim3(kResThreads), args,
                                        smem, st));
    *G_out = G;
    return 1;
}

template <int K>
static int try_launch_resident_t(Handle* h, LfgArgs& a, cudaStream_t st, int64_t* G_out)
{
    DevInfo di;
    GB_CHECK(dev_info(h->device, &di));
    const int64_t n_c = ((a.N + di.sms - 1) / di.sms + 31) & ~(int64_t)31;
    const int64_t nblk = n_c / 32;
    if ((nblk + 19) / 20 < (nblk + 15) / 16) return try_launch_resident_k<K, 640>(h, a, st, G_out);
    return try_launch_resident_k<K, 512>(h, a, st, G_out);
}

static int try_launch_resident(Handle* h, LfgArgs& a, int k, cudaStream_t st, int64_t* G_out)
{
    if (k == 1) return try_launch_resident_t<1>(h, a, st, G_out);
    if (k == 2) return try_launch_resident_t<2>(h, a, st, G_out);
    return try_launch_resident_t<4>(h, a, st, G_out);
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

// Default leap order of every launch kind (order 4, where a handle's ring
// serves it, was slower in every one: fills 2.43 -> 3.12 ms for 2^30 values,
// the resident fused step 11.9 -> 13.4 us and the streamed one 2.04 -> 2.47 ms
// at 1e6 and 1e8 oscillators).
constexpr int kOrderFill = 2, kOrderLd = 2, kOrderResident = 2, kOrderStep = 2, kOrderOu = 2;

int lfg_fill(Handle* h, void* dst, int64_t n, int mode, cudaStream_t st)
{
    const int k = pick_order(h, kOrderFill);
    LfgArgs a{};
    set_ring(h, a, k);
    a.n_pos = n;
    a.w = round_width(h, k, 0);
    a.out = dst;
    int64_t G = 0;
    if (mode == LFG_U32)
        GB_CHECK(launch<LFG_U32>(h, a, k, st, &G));
    else if (mode == LFG_UNIFORM)
        GB_CHECK(launch<LFG_UNIFORM>(h, a, k, st, &G));
    else
        GB_CHECK(launch<LFG_NORMAL>(h, a, k, st, &G));
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
    a.N = s->n;
    a.n_steps = init ? 2 : n_steps;
    a.n_pos = 4 * s->n * a.n_steps;
    a.x = s->x;
    a.v = s->v;
    a.Kper = s->K_per;
    a.c = make_coef(s);
    int64_t G = 0;
    int rc = 0;
    if (!init) {
        const int kr = pick_order(h, kOrderResident);
        set_ring(h, a, kr);
        rc = try_launch_resident(h, a, kr, st, &G);
        if (rc < 0) return rc;
    }
    if (rc == 0) {
        const int k = pick_order(h, kOrderLd);
        set_ring(h, a, k);
        a.w = round_width(h, k, 4 * s->n);
        if (init)
            GB_CHECK(launch<LFG_LD_INIT>(h, a, k, st, &G));
        else
            GB_CHECK(launch<LFG_LD>(h, a, k, st, &G));
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
    const int k = pick_order(h, kOrderStep);
    const int64_t D = (int64_t)h->ll - h->sl;
    const int64_t four_n = 4 * s->n;
    if (four_n > round_width(h, k, 0))
        return fail(GBRNG_ELAGS,
                    "one launch per step needs 4N = %lld within %d times the lag distance "
                    "(ll - sl = %lld)",
                    (long long)four_n, k, (long long)D);
    GB_CHECK(ensure_eacc(h, s->n));
    GB_CUDA(cudaMemsetAsync(h->eacc, 0, sizeof(float2) * s->n, st));
    LfgArgs a{};
    set_ring(h, a, k);
    a.N = s->n;
    a.x = s->x;
    a.v = s->v;
    a.Kper = s->K_per;
    a.c = make_coef(s);
    const unsigned blocks = (unsigned)((s->n + 255) / 256);
    uint32_t sP = a.base_slot;
    for (int64_t t = 0; t < n_steps; ++t) {
        if (k == 1)
            lfg_step_kernel<1><<<blocks, 256, 0, st>>>(a, sP, h->eacc);
        else if (k == 2)
            lfg_step_kernel<2><<<blocks, 256, 0, st>>>(a, sP, h->eacc);
        else
            lfg_step_kernel<4><<<blocks, 256, 0, st>>>(a, sP, h->eacc);
        sP = slot_add(sP, (uint32_t)four_n, a.R);
    }
    GB_CUDA(cudaGetLastError());
    h->pos += four_n * n_steps;
    return stepwise_stats(h, s, n_steps, out, st);
}

template <int K>
static int launch_ou(Handle* h, LfgArgs& a, OuCoef c, float* Rp, float* R0, int64_t ev,
                     double* parts, int64_t G, cudaStream_t st)
{
    void* args[] = {&a, &c, &Rp, &R0, &ev, &parts};
    GB_CUDA(cudaLaunchCooperativeKernel((const void*)lfg_ou_kernel<K>, dim3((unsigned)G), dim3(256),
                                        args, 0, st));
    return GBRNG_OK;
}

int lfg_ou(const ou_system* s, int64_t n_steps, int64_t every, double* mean, double* corr,
           cudaStream_t st)
{
    Handle* h = s->rng;
    const int k = pick_order(h, kOrderOu);
    const int64_t D = (int64_t)h->ll - h->sl;
    const int64_t two_n = 2 * s->n;
    if (two_n > round_width(h, k, 0))
        return fail(GBRNG_ELAGS,
                    "one round per step needs 2N = %lld within %d times the lag distance "
                    "(ll - sl = %lld)",
                    (long long)two_n, k, (long long)D);
    DevInfo di;
    GB_CHECK(dev_info(h->device, &di));
    int occ = 0;
    const void* fn = k == 1 ? (const void*)lfg_ou_kernel<1>
                            : k == 2 ? (const void*)lfg_ou_kernel<2> : (const void*)lfg_ou_kernel<4>;
    GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 256, 0));
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
    set_ring(h, a, k);
    a.N = s->n;
    a.n_steps = n_steps;
    a.w = round_width(h, k, 0);   // the full round: floor(w / 2N) steps a round
    GB_CHECK(launch_common(h, a, G, st));
    const OuCoef c = make_ou_coef(s);
    double* parts = rec ? h->partials : nullptr;
    if (k == 1)
        GB_CHECK(launch_ou<1>(h, a, c, s->R, R0, every, parts, G, st));
    else if (k == 2)
        GB_CHECK(launch_ou<2>(h, a, c, s->R, R0, every, parts, G, st));
    else
        GB_CHECK(launch_ou<4>(h, a, c, s->R, R0, every, parts, G, st));
    GB_CHECK(read_status(h, st));
    h->pos += two_n * n_steps;
    if (rec) return ou_finish(h, s->n, n_rec, G, mean, corr, st);
    return GBRNG_OK;
}

}  // namespace gb

using namespace gb;

extern "C" int gbrng_set_lfg_order(int k)
{
    if (k != 0 && k != 1 && k != 2 && k != 4)
        return fail(GBRNG_EINVAL, "Lagged Fibonacci leap order must be 0 (automatic), 1, 2 or 4");
    g_lfg_order.store(k);
    return GBRNG_OK;
}
