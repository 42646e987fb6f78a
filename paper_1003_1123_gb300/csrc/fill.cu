// Stand-alone fills for the per-thread generators (Hybrid Taus, Ran2):
// out[d*S + s] is the d-th draw of stream s.  One thread owns one stream at a
// time and keeps its state in registers (Taus) or in a shared-memory column
// (Ran2's shuffle table) for all of its draws; stores are coalesced across
// the streams of a warp.
#include "device.cuh"
#include "internal.cuh"

namespace gb {

enum { FILL_U32 = 0, FILL_UNIFORM = 1, FILL_NORMAL = 2 };

template <int MODE, class State>
__device__ __forceinline__ void emit_word(State& y, int64_t idx, void* out)
{
    if (MODE == FILL_U32) {
        ((uint32_t*)out)[idx] = next_word(y);
    } else if (MODE == FILL_UNIFORM) {
        ((float*)out)[idx] = u01_from_u32(next_word(y));
    } else {
        const uint32_t r1 = next_word(y);
        const uint32_t r2 = next_word(y);
        float2 g;
        box_muller_u32(r1, r2, g.x, g.y);
        ((float2*)out)[idx] = g;
    }
}

// n_items = numbers (u32, uniform) or pairs (normal).
// Hybrid Taus (uint4 state) and the LCG (uint32 state): one word chain per stream.
template <int MODE, class State>
__global__ void __launch_bounds__(256) word_fill_kernel(State* __restrict__ st, int64_t S,
                                                        int64_t n_items, void* __restrict__ out)
{
    const int64_t active = S < n_items ? S : n_items;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < active; s += stride) {
        State y = st[s];
        int64_t idx = s;
        // four draws in flight per iteration: independent stores, one state chain
        for (; idx + 3 * S < n_items; idx += 4 * S) {
            if (MODE == FILL_NORMAL) {
                // the four pairs two at a time in the paired instructions' lanes
                uint32_t r[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) r[q] = next_word(y);
                float2* o = (float2*)out;
                float2 ga, gb;
                box_muller_2pairs_u32(r[0], r[1], r[2], r[3], ga, gb);
                o[idx] = ga, o[idx + S] = gb;
                box_muller_2pairs_u32(r[4], r[5], r[6], r[7], ga, gb);
                o[idx + 2 * S] = ga, o[idx + 3 * S] = gb;
            } else {
                emit_word<MODE>(y, idx, out);
                emit_word<MODE>(y, idx + S, out);
                emit_word<MODE>(y, idx + 2 * S, out);
                emit_word<MODE>(y, idx + 3 * S, out);
            }
        }
        for (; idx < n_items; idx += S) emit_word<MODE>(y, idx, out);
        st[s] = y;
    }
}

template <int MODE>
__global__ void __launch_bounds__(128) ran2_fill_kernel(int32_t* __restrict__ st, int64_t S,
                                                        int64_t n_items, void* __restrict__ out)
{
    extern __shared__ int32_t tab[];      // [32][blockDim.x]
    const int T = blockDim.x, tid = threadIdx.x;
    auto iv = [&](int j) -> int32_t& { return tab[j * T + tid]; };
    const int64_t active = S < n_items ? S : n_items;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + tid; s < active; s += stride) {
        Ran2Regs r{st[s], st[S + s], st[2 * S + s]};
#pragma unroll 4
        for (int j = 0; j < 32; ++j) iv(j) = st[(3 + j) * S + s];
        auto emit = [&](int64_t idx) {
            if (MODE == FILL_U32) {
                ((uint32_t*)out)[idx] = (uint32_t)ran2_next(r, iv);
            } else if (MODE == FILL_UNIFORM) {
                ((float*)out)[idx] = u01_from_ran2(ran2_next(r, iv));
            } else {
                const float u1 = u01_from_ran2(ran2_next(r, iv));
                const float u2 = u01_from_ran2(ran2_next(r, iv));
                float2 g;
                box_muller(u1, u2, g.x, g.y);
                ((float2*)out)[idx] = g;
            }
        };
        int64_t idx = s;
        // four draws a loop iteration: one bound check for four stores
        for (; idx + 3 * S < n_items; idx += 4 * S) {
            if (MODE == FILL_NORMAL) {
                // the four pairs two at a time in the paired instructions' lanes
                float u[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) u[q] = u01_from_ran2(ran2_next(r, iv));
                float2* o = (float2*)out;
                float2 ga, gb;
                box_muller_2pairs(u[0], u[1], u[2], u[3], ga, gb);
                o[idx] = ga, o[idx + S] = gb;
                box_muller_2pairs(u[4], u[5], u[6], u[7], ga, gb);
                o[idx + 2 * S] = ga, o[idx + 3 * S] = gb;
            } else {
                emit(idx);
                emit(idx + S);
                emit(idx + 2 * S);
                emit(idx + 3 * S);
            }
        }
        for (; idx < n_items; idx += S) emit(idx);
        st[s] = r.idum;
        st[S + s] = r.idum2;
        st[2 * S + s] = r.iy;
#pragma unroll 4
        for (int j = 0; j < 32; ++j) st[(3 + j) * S + s] = iv(j);
    }
}

// Grid: one thread per stream (up to the streams a fill touches), in as many
// waves as that takes, rather than one resident wave looping over streams:
// the blocks then start, and load their streams' state, at staggered times
// instead of all together under the fill's store traffic (2^30 numbers from
// 1e6 streams: Ran2 uniform 1.15 -> 1.09 ms, normal 1.91 -> 1.82, Taus uniform
// 0.91 -> 0.87, normal 1.59 -> 1.57).  The kernels keep their stream loop, so
// any grid covers every stream.
template <int MODE>
static int fill_pt(Handle* h, void* dst, int64_t n_items, cudaStream_t st)
{
    const int64_t active = h->n < n_items ? h->n : n_items;
    if (h->kind == GBRNG_TAUS || h->kind == GBRNG_LCG) {
        const int T = 256;
        const int64_t blocks = (active + T - 1) / T;
        if (h->kind == GBRNG_TAUS)
            word_fill_kernel<MODE, uint4><<<(unsigned)blocks, T, 0, st>>>(h->taus, h->n, n_items, dst);
        else
            word_fill_kernel<MODE, uint32_t><<<(unsigned)blocks, T, 0, st>>>(h->lcg, h->n, n_items,
                                                                            dst);
    } else {
        const int T = 128;
        const size_t smem = sizeof(int32_t) * 32 * T;
        const int64_t blocks = (active + T - 1) / T;
        ran2_fill_kernel<MODE><<<(unsigned)blocks, T, smem, st>>>(h->r2, h->n, n_items, dst);
    }
    GB_CUDA(cudaGetLastError());
    return GBRNG_OK;
}

int fill_u32_pt(Handle* h, uint32_t* dst, int64_t n, cudaStream_t st)
{
    return fill_pt<FILL_U32>(h, dst, n, st);
}

int fill_uniform_pt(Handle* h, float* dst, int64_t n, cudaStream_t st)
{
    return fill_pt<FILL_UNIFORM>(h, dst, n, st);
}

int fill_normal_pt(Handle* h, float* dst, int64_t n, cudaStream_t st)
{
    return fill_pt<FILL_NORMAL>(h, dst, n / 2, st);
}

}  // namespace gb
