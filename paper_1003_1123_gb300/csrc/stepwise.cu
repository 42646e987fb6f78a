// Paper-form Langevin dynamics for the per-thread generators: one kernel
// launch per step (Algorithms 1 and 2 as printed, Fig. 2-3).  Every launch
// loads each oscillator's generator state (Ran2's shuffle table included, read
// and written in global memory), x, v and its energy sum from global memory,
// takes one step and stores them back.  Same draws and binary32 operations as
// the persistent kernel, so x, v and the generator states equal ld_run's bit
// for bit; the reference form against which the persistent design is measured.
#include "device.cuh"
#include "internal.cuh"

namespace gb {

struct StepArgs {
    int64_t n;
    float* x;
    float* v;
    const float* Kper;
    LdCoef c;
    uint4* taus;
    int32_t* r2;
    uint32_t* lcg;
    int64_t S;
    float2* eacc;   // [n] Kahan (sum, compensation) of the oscillator's energy
};

template <int KIND>
__global__ void __launch_bounds__(256) step_pt_kernel(StepArgs a)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const LdCoef c = a.c;
    const float Ki = a.Kper ? a.Kper[i] : c.K;
    float x0 = a.x[3 * i], x1 = a.x[3 * i + 1], x2 = a.x[3 * i + 2];
    float v0 = a.v[3 * i], v1 = a.v[3 * i + 1], v2 = a.v[3 * i + 2];
    float g0, g1, g2;
    if (KIND == GBRNG_TAUS) {
        TausDraw td;
        td.y = a.taus[i];
        td.normals3(g0, g1, g2);
        a.taus[i] = td.y;
    } else if (KIND == GBRNG_LCG) {
        LcgDraw lc;
        lc.x = a.lcg[i];
        lc.normals3(g0, g1, g2);
        a.lcg[i] = lc.x;
    } else {
        int32_t* r2 = a.r2;
        const int64_t S = a.S;
        Ran2Regs r{r2[i], r2[S + i], r2[2 * S + i]};
        auto iv = [r2, S, i](int j) -> int32_t& { return r2[(3 + j) * S + i]; };
        const float u1 = u01_from_ran2(ran2_next(r, iv));
        const float u2 = u01_from_ran2(ran2_next(r, iv));
        const float u3 = u01_from_ran2(ran2_next(r, iv));
        const float u4 = u01_from_ran2(ran2_next(r, iv));
        box_muller3(u1, u2, u3, u4, g0, g1, g2);
        r2[i] = r.idum;
        r2[S + i] = r.idum2;
        r2[2 * S + i] = r.iy;
    }
    const float ckx = __fmul_rn(c.ckm, Ki);
    em_component(c.cdt, c.cva, ckx, c.cs, g0, x0, v0);
    em_component(c.cdt, c.cva, ckx, c.cs, g1, x1, v1);
    em_component(c.cdt, c.cva, ckx, c.cs, g2, x2, v2);
    a.x[3 * i] = x0, a.x[3 * i + 1] = x1, a.x[3 * i + 2] = x2;
    a.v[3 * i] = v0, a.v[3 * i + 1] = v1, a.v[3 * i + 2] = v2;
    Kahan e;
    const float2 ec = a.eacc[i];
    e.s = ec.x;
    e.c = ec.y;
    e.add(energy3(0.5f * Ki, c.hm, x0, x1, x2, v0, v1, v2));
    a.eacc[i] = make_float2(e.s, e.c);
}

// Final-state sums and the oscillators' energy sums, per block.
__global__ void step_stats_kernel(const float* x, const float* v, const float2* eacc, int64_t n,
                                  double* partials)
{
    __shared__ double red[4 * 32];
    double acc[4] = {0, 0, 0, 0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        for (int k = 0; k < 3; ++k) {
            const double xi = x[3 * i + k], vi = v[3 * i + k];
            acc[0] += xi * xi;
            acc[1] += vi * vi;
            acc[2] += xi * vi;
        }
        acc[3] += (double)eacc[i].x - (double)eacc[i].y;
    }
    block_reduce_sum<4>(acc, red);
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) partials[4 * blockIdx.x + k] = acc[k];
}

int stepwise_stats(Handle* h, const ld_system* s, int64_t n_steps, ld_stats* out, cudaStream_t st)
{
    if (!out) return GBRNG_OK;
    const int64_t blocks = 256;
    GB_CHECK(ensure_partials(h, blocks));
    step_stats_kernel<<<(unsigned)blocks, 256, 0, st>>>(s->x, s->v, h->eacc, s->n, h->partials);
    GB_CUDA(cudaGetLastError());
    return finish_stats(h, blocks, n_steps, out, st);
}

int ld_run_stepwise_pt(const ld_system* s, int64_t n_steps, ld_stats* out, cudaStream_t st)
{
    Handle* h = s->rng;
    if (s->n == 0) {
        if (out) *out = ld_stats{0, 0, 0, 0, n_steps};
        return GBRNG_OK;
    }
    GB_CHECK(ensure_eacc(h, s->n));
    GB_CUDA(cudaMemsetAsync(h->eacc, 0, sizeof(float2) * s->n, st));
    StepArgs a;
    a.n = s->n;
    a.x = s->x;
    a.v = s->v;
    a.Kper = s->K_per;
    a.c = make_coef(s);
    a.taus = h->taus;
    a.r2 = h->r2;
    a.lcg = h->lcg;
    a.S = h->n;
    a.eacc = h->eacc;
    const unsigned blocks = (unsigned)((s->n + 255) / 256);
    for (int64_t t = 0; t < n_steps; ++t) {
        if (h->kind == GBRNG_TAUS)
            step_pt_kernel<GBRNG_TAUS><<<blocks, 256, 0, st>>>(a);
        else if (h->kind == GBRNG_LCG)
            step_pt_kernel<GBRNG_LCG><<<blocks, 256, 0, st>>>(a);
        else
            step_pt_kernel<GBRNG_RAN2><<<blocks, 256, 0, st>>>(a);
    }
    GB_CUDA(cudaGetLastError());
    return stepwise_stats(h, s, n_steps, out, st);
}

}  // namespace gb
