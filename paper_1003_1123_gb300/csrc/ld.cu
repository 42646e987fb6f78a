// Fused Langevin dynamics for the per-thread generators (Hybrid Taus, Ran2):
// one persistent launch runs every step of every oscillator.  A thread owns
// oscillators i = g, g + W, g + 2W, ... (W = threads in the grid) and, for
// each, keeps x, v, K_i and the generator state in registers (Ran2's shuffle
// table in a shared-memory column) for all n_steps; per step it draws four
// uniforms, forms three Box-Muller normals, applies the Euler-Maruyama update
// and accumulates |x|^2 and |v|^2 for the time-summed energy.  State goes back to global memory once.
#include <algorithm>

#include "device.cuh"
#include "internal.cuh"

namespace gb {

struct LdArgs {
    int64_t n, n_steps;
    float* x;
    float* v;
    const float* Kper;
    LdCoef c;
    uint4* taus;       // Taus state [streams]
    int32_t* r2;       // Ran2 state [35][streams]
    uint32_t* lcg;     // LCG state [streams]
    int64_t S;         // streams of the generator (row stride of r2)
    double* partials;  // [gridDim.x][4]
};

// Register budget (128-thread blocks per SM, measured at 1e6 oscillators):
// Hybrid Taus and Ran2 six (up to 85 registers, no spills; Taus 1% and Ran2 5%
// faster than ten and nine blocks at 48 and 56 registers, which spilled), the
// LCG seven (5% faster than ten).
template <int KIND, bool INIT>
__global__ void __launch_bounds__(128, KIND == GBRNG_LCG ? 7 : 6) ld_pt_kernel(LdArgs a)
{
    extern __shared__ int32_t tab[];   // Ran2: [32][blockDim.x]
    __shared__ double red[4 * 32];
    const int64_t W = (int64_t)gridDim.x * blockDim.x;
    const LdCoef c = a.c;
    double acc[4] = {0, 0, 0, 0};      // sum x^2, v^2, x.v, energy
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += W) {
        const float Ki = a.Kper ? a.Kper[i] : c.K;
        float x0, x1, x2, v0, v1, v2;
        if (!INIT) {
            x0 = a.x[3 * i], x1 = a.x[3 * i + 1], x2 = a.x[3 * i + 2];
            v0 = a.v[3 * i], v1 = a.v[3 * i + 1], v2 = a.v[3 * i + 2];
        }
        TausDraw td;
        LcgDraw lc;
        Ran2Draw rd;
        if (KIND == GBRNG_TAUS) {
            td.y = a.taus[i];
        } else if (KIND == GBRNG_LCG) {
            lc.x = a.lcg[i];
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
        EnergySum es;
        float hK = 0.f;
        if (INIT) {
            // draw-step 0 -> x = sqrt(kT/K_i) g, draw-step 1 -> v = sqrt(kT/m) g
            float g0, g1, g2;
            draw3<KIND>(td, lc, rd, g0, g1, g2);
            const float sx = __fsqrt_rn(__fdiv_rn(c.kT, Ki));
            x0 = __fmul_rn(sx, g0), x1 = __fmul_rn(sx, g1), x2 = __fmul_rn(sx, g2);
            draw3<KIND>(td, lc, rd, g0, g1, g2);
            v0 = __fmul_rn(c.sv, g0), v1 = __fmul_rn(c.sv, g1), v2 = __fmul_rn(c.sv, g2);
        } else {
            const float ckx = __fmul_rn(c.ckm, Ki);
            hK = 0.5f * Ki;
            for (int64_t t0 = 0; t0 < a.n_steps; t0 += kEnergyBlock) {
                const int nb = (int)min((int64_t)kEnergyBlock, a.n_steps - t0);
                // the LCG draws cheaply enough to gain from two steps a loop
                // iteration (3% faster); Taus and Ran2 lose 1-2%
#pragma unroll(KIND == GBRNG_LCG ? 2 : 1)
                for (int k = 0; k < nb; ++k) {
                    float g0, g1, g2;
                    draw3<KIND>(td, lc, rd, g0, g1, g2);
                    em_component(c.cdt, c.cva, ckx, c.cs, g0, x0, v0);
                    em_component(c.cdt, c.cva, ckx, c.cs, g1, x1, v1);
                    em_component(c.cdt, c.cva, ckx, c.cs, g2, x2, v2);
                    es.add(x0, x1, x2, v0, v1, v2);
                }
                es.flush();
            }
        }
        a.x[3 * i] = x0, a.x[3 * i + 1] = x1, a.x[3 * i + 2] = x2;
        a.v[3 * i] = v0, a.v[3 * i + 1] = v1, a.v[3 * i + 2] = v2;
        if (KIND == GBRNG_TAUS) {
            a.taus[i] = td.y;
        } else if (KIND == GBRNG_LCG) {
            a.lcg[i] = lc.x;
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
    if (a.partials) {
        block_reduce_sum<4>(acc, red);
        if (threadIdx.x == 0)
#pragma unroll
            for (int k = 0; k < 4; ++k) a.partials[4 * blockIdx.x + k] = acc[k];
    }
}

// Two oscillators a thread (Hybrid Taus, the LCG, Ran2): thread g takes the
// adjacent pairs (2p, 2p + 1) for p = g, g + W, ..., and advances both in the
// same loop, two steps an iteration, so each thread carries two independent
// generator chains, and the two oscillators' floating-point work (transforms,
// update, energy sums) runs in the two lanes of the paired binary32
// instructions.  One-warp blocks, one full resident wave; Ran2's two tables in
// shared-memory columns.  Per oscillator the draws, operations and state are
// those of ld_pt_kernel, bit for bit; only the order of the final sums over
// oscillators differs.
template <int KIND>
__global__ void __launch_bounds__(32) ld_pair_kernel(LdArgs a, int64_t n_pairs)
{
    extern __shared__ int32_t tab[];   // Ran2: [2][32][blockDim.x], one table per lane oscillator
    __shared__ double red[4 * 32];
    const int64_t W = (int64_t)gridDim.x * blockDim.x;
    const LdCoef c = a.c;
    double acc[4] = {0, 0, 0, 0};
    const float2 cdt = splat2(c.cdt), cva = splat2(c.cva), cs = splat2(c.cs);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n_pairs; p += W) {
        int64_t idx[2];
        bool live[2];
        // lane j of every pair below is oscillator 2p + j
        float2 X[3], V[3], nckx;
        float hK[2];
        TausDraw td[2];
        LcgDraw lc[2];
        Ran2Draw rd[2];
        EnergySum2 es;
        float xs[2][3], vs[2][3], ck[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            idx[j] = 2 * p + j;
            live[j] = idx[j] < a.n;
            const int64_t i = live[j] ? idx[j] : 2 * p;   // a dead second lane shadows the first
            const float Ki = a.Kper ? a.Kper[i] : c.K;
            ck[j] = -__fmul_rn(c.ckm, Ki);
            hK[j] = 0.5f * Ki;
#pragma unroll
            for (int q = 0; q < 3; ++q) xs[j][q] = a.x[3 * i + q], vs[j][q] = a.v[3 * i + q];
            if (KIND == GBRNG_TAUS) {
                td[j].y = a.taus[i];
            } else if (KIND == GBRNG_LCG) {
                lc[j].x = a.lcg[i];
            } else {
                rd[j].tab = tab + j * 32 * blockDim.x;
                rd[j].T = blockDim.x;
                rd[j].tid = threadIdx.x;
                rd[j].r.idum = a.r2[i];
                rd[j].r.idum2 = a.r2[a.S + i];
                rd[j].r.iy = a.r2[2 * a.S + i];
#pragma unroll 4
                for (int q = 0; q < 32; ++q) rd[j].tab[q * blockDim.x + threadIdx.x] = a.r2[(3 + q) * a.S + i];
            }
        }
        nckx = make_float2(ck[0], ck[1]);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            X[q] = make_float2(xs[0][q], xs[1][q]);
            V[q] = make_float2(vs[0][q], vs[1][q]);
        }
        for (int64_t t0 = 0; t0 < a.n_steps; t0 += kEnergyBlock) {
            const int nb = (int)min((int64_t)kEnergyBlock, a.n_steps - t0);
#pragma unroll 2
            for (int k = 0; k < nb; ++k) {
                float2 g[3];
                draw3x2<KIND, true>(td, lc, rd, g);   // shifts as multiplies: 2-4% faster here
#pragma unroll
                for (int q = 0; q < 3; ++q) em_component2(cdt, cva, nckx, cs, g[q], X[q], V[q]);
                es.add(X, V);
            }
            es.flush();
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            if (!live[j]) continue;
            const int64_t i = idx[j];
            const float x0 = j ? X[0].y : X[0].x, x1 = j ? X[1].y : X[1].x, x2 = j ? X[2].y : X[2].x;
            const float v0 = j ? V[0].y : V[0].x, v1 = j ? V[1].y : V[1].x, v2 = j ? V[2].y : V[2].x;
            a.x[3 * i] = x0, a.x[3 * i + 1] = x1, a.x[3 * i + 2] = x2;
            a.v[3 * i] = v0, a.v[3 * i + 1] = v1, a.v[3 * i + 2] = v2;
            if (KIND == GBRNG_TAUS) {
                a.taus[i] = td[j].y;
            } else if (KIND == GBRNG_LCG) {
                a.lcg[i] = lc[j].x;
            } else {
                a.r2[i] = rd[j].r.idum;
                a.r2[a.S + i] = rd[j].r.idum2;
                a.r2[2 * a.S + i] = rd[j].r.iy;
#pragma unroll 4
                for (int q = 0; q < 32; ++q) a.r2[(3 + q) * a.S + i] = rd[j].tab[q * blockDim.x + threadIdx.x];
            }
            acc[0] += (double)x0 * x0 + (double)x1 * x1 + (double)x2 * x2;
            acc[1] += (double)v0 * v0 + (double)v1 * v1 + (double)v2 * v2;
            acc[2] += (double)x0 * v0 + (double)x1 * v1 + (double)x2 * v2;
            acc[3] += es.value(j, hK[j], c.hm);
        }
    }
    if (a.partials) {
        block_reduce_sum<4>(acc, red);
        if (threadIdx.x == 0)
#pragma unroll
            for (int k = 0; k < 4; ++k) a.partials[4 * blockIdx.x + k] = acc[k];
    }
}

// Pair-kernel grid: one full resident wave of one-warp blocks (16 a SM for
// Taus, 20 for Ran2 at 1e6 oscillators).  Measured at 1e6 oscillators x 1000
// steps (scalar arithmetic): 5.90 ms for Hybrid Taus against 6.13 ms for one
// oscillator a thread; 64-, 128- and 256-thread blocks 6.06-6.60 ms; a grid
// trimmed so that every thread gets the same number of pairs (fewer warps a
// SM) 6.36 ms.  With the paired instructions: Taus 4.9 ms, Ran2 6.3 ms (64-
// thread blocks for Ran2 equal).  Returns 0 (and launches nothing) when the
// pairs do not fill one resident wave, where one oscillator a thread spreads
// better.
template <int KIND>
static int launch_pairs(const ld_system* s, int64_t n_steps, bool want_stats, int64_t* blocks_out,
                        cudaStream_t st)
{
    Handle* h = s->rng;
    DevInfo di;
    GB_CHECK(dev_info(h->device, &di));
    const int T = 32;
    const size_t smem = KIND == GBRNG_RAN2 ? sizeof(int32_t) * 2 * 32 * T : 0;
    int occ = 0;
    GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ld_pair_kernel<KIND>, T, smem));
    if (occ < 1) return 0;
    const int64_t pairs = (s->n + 1) / 2, wave = (int64_t)di.sms * occ * T;
    if (pairs < wave) return 0;
    const int64_t blocks = wave / T;
    if (want_stats) GB_CHECK(ensure_partials(h, blocks));
    LdArgs a;
    a.n = s->n;
    a.n_steps = n_steps;
    a.x = s->x;
    a.v = s->v;
    a.Kper = s->K_per;
    a.c = make_coef(s);
    a.taus = h->taus;
    a.r2 = h->r2;
    a.lcg = h->lcg;
    a.S = h->n;
    a.partials = want_stats ? h->partials : nullptr;
    ld_pair_kernel<KIND><<<(unsigned)blocks, T, smem, st>>>(a, pairs);
    GB_CUDA(cudaGetLastError());
    *blocks_out = blocks;
    return 1;
}

// Grid shape: threads per block T and one full resident wave (SMs x blocks
// per SM, fewer only when the system has fewer oscillators than that wave has
// threads).  Thread g takes oscillators g, g + W, ...; the last, partial round
// then falls on the lowest blocks, which the block scheduler spreads over all
// SMs, so every SM carries the same work to within one block's round.  (A grid
// cut to ceil(n / (oscillators per thread x T)) blocks leaves some SMs a block
// short and others a block over, about 9% apart at 1e6 oscillators.)
template <int KIND, bool INIT>
static int launch_ld(const ld_system* s, int64_t n_steps, bool want_stats, int64_t* blocks_out,
                     cudaStream_t st)
{
    Handle* h = s->rng;
    DevInfo di;
    GB_CHECK(dev_info(h->device, &di));
    int T = 128;
    // one-warp blocks spread small systems over all SMs, and are 1% faster for
    // Ran2 at any size (25 warps a SM at 79 registers)
    if (s->n < (int64_t)di.sms * 128 * 2 || KIND == GBRNG_RAN2) T = 32;
    const size_t smem = KIND == GBRNG_RAN2 ? sizeof(int32_t) * 32 * T : 0;
    int occ = 0;
    GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ld_pt_kernel<KIND, INIT>, T, smem));
    if (occ < 1) occ = 1;
    int64_t blocks = std::min<int64_t>((int64_t)di.sms * occ, (s->n + T - 1) / T);
    if (blocks < 1) blocks = 1;
    if (want_stats) GB_CHECK(ensure_partials(h, blocks));
    LdArgs a;
    a.n = s->n;
    a.n_steps = n_steps;
    a.x = s->x;
    a.v = s->v;
    a.Kper = s->K_per;
    a.c = make_coef(s);
    a.taus = h->taus;
    a.r2 = h->r2;
    a.lcg = h->lcg;
    a.S = h->n;
    a.partials = want_stats ? h->partials : nullptr;
    ld_pt_kernel<KIND, INIT><<<(unsigned)blocks, T, smem, st>>>(a);
    GB_CUDA(cudaGetLastError());
    *blocks_out = blocks;
    return GBRNG_OK;
}

int ld_init_pt(const ld_system* s, cudaStream_t st)
{
    int64_t blocks = 0;
    if (s->rng->kind == GBRNG_TAUS) return launch_ld<GBRNG_TAUS, true>(s, 0, false, &blocks, st);
    if (s->rng->kind == GBRNG_LCG) return launch_ld<GBRNG_LCG, true>(s, 0, false, &blocks, st);
    return launch_ld<GBRNG_RAN2, true>(s, 0, false, &blocks, st);
}

int ld_run_pt(const ld_system* s, int64_t n_steps, ld_stats* out, cudaStream_t st)
{
    if (s->n == 0) {
        if (out) *out = ld_stats{0, 0, 0, 0, n_steps};
        return GBRNG_OK;
    }
    int64_t blocks = 0;
    const bool want = out != nullptr;
    int rc = 0;
    if (s->rng->kind == GBRNG_TAUS)
        rc = launch_pairs<GBRNG_TAUS>(s, n_steps, want, &blocks, st);
    else if (s->rng->kind == GBRNG_LCG)
        rc = launch_pairs<GBRNG_LCG>(s, n_steps, want, &blocks, st);
    else if (s->rng->kind == GBRNG_RAN2)
        rc = launch_pairs<GBRNG_RAN2>(s, n_steps, want, &blocks, st);
    if (rc < 0) return rc;
    if (rc == 1) return finish_stats(s->rng, blocks, n_steps, out, st);
    if (s->rng->kind == GBRNG_TAUS)
        GB_CHECK((launch_ld<GBRNG_TAUS, false>(s, n_steps, want, &blocks, st)));
    else if (s->rng->kind == GBRNG_LCG)
        GB_CHECK((launch_ld<GBRNG_LCG, false>(s, n_steps, want, &blocks, st)));
    else
        GB_CHECK((launch_ld<GBRNG_RAN2, false>(s, n_steps, want, &blocks, st)));
    return finish_stats(s->rng, blocks, n_steps, out, st);
}

}  // namespace gb
