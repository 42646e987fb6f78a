// Overdamped 1-D Langevin dynamics (Sec. IV, Eq. 4-5) for the per-thread
// generators: one persistent thread per particle keeps R, R(0) and its
// generator in registers (Ran2's shuffle table in a shared-memory column) for
// all steps; every `every` steps the block sums R and R R(0) into its record
// slot, and one block per record adds the slots in a fixed order.
#include <cmath>
#include <vector>

#include "device.cuh"
#include "internal.cuh"

namespace gb {

struct OuArgs {
    int64_t n, n_steps, every;
    float* R;
    OuCoef c;
    uint4* taus;
    int32_t* r2;
    uint32_t* lcg;
    int64_t S;
    double* partials;   // [n_rec][blocks][2], or null (no records)
};

// One normal per particle-step: cosine branch of Box-Muller on two draws.
template <int KIND>
__device__ __forceinline__ float normal1(TausDraw& td, LcgDraw& lc, Ran2Draw& rd)
{
    if (KIND == GBRNG_TAUS) {
        const uint32_t r1 = taus_next(td.y);
        const uint32_t r2 = taus_next(td.y);
        return box_muller_cos_u32(r1, r2);
    } else if (KIND == GBRNG_LCG) {
        const uint32_t r1 = lcg_next(lc.x);
        const uint32_t r2 = lcg_next(lc.x);
        return box_muller_cos_u32(r1, r2);
    } else {
        const float u1 = u01_from_ran2(rd.next());
        const float u2 = u01_from_ran2(rd.next());
        return box_muller_cos(u1, u2);
    }
}

// The normals of two consecutive steps (draws of step t, then of step t + 1)
// in the two lanes of the paired binary32 instructions: each lane is
// normal1's transform, bit for bit.
template <int KIND>
__device__ __forceinline__ float2 normal2(TausDraw& td, LcgDraw& lc, Ran2Draw& rd)
{
    if (KIND == GBRNG_RAN2) {
        const float u1 = u01_from_ran2(rd.next());
        const float u2 = u01_from_ran2(rd.next());
        const float u3 = u01_from_ran2(rd.next());
        const float u4 = u01_from_ran2(rd.next());
        return box_muller_cos2(neg2log2(make_float2(u1, u3)),
                               __fmul2_rn(splat2(4.0f), make_float2(u2, u4)));
    } else {
        uint32_t r[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) r[q] = KIND == GBRNG_TAUS ? taus_next(td.y) : lcg_next(lc.x);
        const float2 u = make_float2(open01_from_u32(r[0]), open01_from_u32(r[2]));
        const float2 x = __ffma2_rn(splat2(4.0f), make_float2(mant_from_u32(r[1]), mant_from_u32(r[3])),
                                    splat2(-0x1.fffffep+1f));
        return box_muller_cos2(neg2log2(u), x);
    }
}

template <int KIND>
__global__ void __launch_bounds__(256) ou_pt_kernel(OuArgs a)
{
    extern __shared__ int32_t tab[];   // Ran2: [32][blockDim.x]
    __shared__ double red[2 * 32];
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool live = i < a.n;
    const int64_t k = live ? i : 0;
    TausDraw td;
    LcgDraw lc;
    Ran2Draw rd;
    if (KIND == GBRNG_TAUS) {
        td.y = a.taus[k];
    } else if (KIND == GBRNG_LCG) {
        lc.x = a.lcg[k];
    } else {
        rd.tab = tab;
        rd.T = blockDim.x;
        rd.tid = threadIdx.x;
        rd.r.idum = a.r2[k];
        rd.r.idum2 = a.r2[a.S + k];
        rd.r.iy = a.r2[2 * a.S + k];
#pragma unroll 4
        for (int j = 0; j < 32; ++j) tab[j * blockDim.x + threadIdx.x] = a.r2[(3 + j) * a.S + k];
    }
    float R = live ? a.R[k] : 0.f;
    const float R0 = R;
    int64_t rec = 0, next_rec = 0;
    for (int64_t t = 0;;) {
        if (a.partials && t == next_rec) {
            next_rec += a.every;
            double v[2] = {live ? (double)R : 0.0, live ? (double)R * (double)R0 : 0.0};
            block_reduce_sum<2>(v, red);
            if (threadIdx.x == 0) {
                double* o = a.partials + 2 * (rec * gridDim.x + blockIdx.x);
                o[0] = v[0];
                o[1] = v[1];
            }
            ++rec;
        }
        if (t == a.n_steps) break;
        if (t + 1 < a.n_steps && !(a.partials && t + 1 == next_rec)) {
            // two steps with no record between them
            const float2 g = normal2<KIND>(td, lc, rd);
            R = __fmaf_rn(a.c.cs, g.x, __fmaf_rn(-a.c.c1, R, R));
            R = __fmaf_rn(a.c.cs, g.y, __fmaf_rn(-a.c.c1, R, R));
            t += 2;
        } else {
            const float g = normal1<KIND>(td, lc, rd);
            R = __fmaf_rn(a.c.cs, g, __fmaf_rn(-a.c.c1, R, R));
            t += 1;
        }
    }
    if (!live) return;
    a.R[i] = R;
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
}

// One block per record: fixed-order sum of the record's block slots.
__global__ void ou_finish_kernel(const double* partials, int64_t blocks, double inv_n,
                                 double* out)
{
    __shared__ double red[2 * 32];
    const int64_t rec = blockIdx.x;
    double v[2] = {0, 0};
    for (int64_t b = threadIdx.x; b < blocks; b += blockDim.x) {
        v[0] += partials[2 * (rec * blocks + b)];
        v[1] += partials[2 * (rec * blocks + b) + 1];
    }
    block_reduce_sum<2>(v, red);
    if (threadIdx.x == 0) {
        out[2 * rec] = v[0] * inv_n;
        out[2 * rec + 1] = v[1] * inv_n;
    }
}

OuCoef make_ou_coef(const ou_system* s)
{
    OuCoef c;
    c.c1 = (float)(s->k_sp * s->dt / s->xi);
    c.cs = (float)sqrt(2.0 * s->kT * s->dt / s->xi);
    return c;
}

int ou_finish(Handle* h, int64_t n, int64_t n_rec, int64_t blocks, double* mean, double* corr,
              cudaStream_t st)
{
    double* out = h->partials + 2 * n_rec * blocks;
    ou_finish_kernel<<<(unsigned)n_rec, 256, 0, st>>>(h->partials, blocks, 1.0 / (double)n, out);
    GB_CUDA(cudaGetLastError());
    std::vector<double> host(2 * (size_t)n_rec);
    GB_CUDA(cudaMemcpyAsync(host.data(), out, sizeof(double) * 2 * n_rec, cudaMemcpyDeviceToHost,
                            st));
    GB_CUDA(cudaStreamSynchronize(st));
    for (int64_t r = 0; r < n_rec; ++r) {
        mean[r] = host[2 * r];
        corr[r] = host[2 * r + 1];
    }
    return GBRNG_OK;
}

int ou_run_pt(const ou_system* s, int64_t n_steps, int64_t every, double* mean, double* corr,
              cudaStream_t st)
{
    Handle* h = s->rng;
    const int T = 256;
    const int64_t blocks = (s->n + T - 1) / T;
    const bool rec = mean != nullptr;
    const int64_t n_rec = n_steps / every + 1;
    if (rec) {
        if (n_rec > 0x7fffffff || (double)n_rec * blocks * 16.0 > 4.0 * (1 << 30))
            return fail(GBRNG_EINVAL, "%lld records x %lld blocks exceed the record scratch",
                        (long long)n_rec, (long long)blocks);
        GB_CHECK(ensure_partials(h, (2 * n_rec * blocks + 2 * n_rec + 3) / 4));
    }
    OuArgs a;
    a.n = s->n;
    a.n_steps = n_steps;
    a.every = every;
    a.R = s->R;
    a.c = make_ou_coef(s);
    a.taus = h->taus;
    a.r2 = h->r2;
    a.lcg = h->lcg;
    a.S = h->n;
    a.partials = rec ? h->partials : nullptr;
    if (h->kind == GBRNG_TAUS)
        ou_pt_kernel<GBRNG_TAUS><<<(unsigned)blocks, T, 0, st>>>(a);
    else if (h->kind == GBRNG_LCG)
        ou_pt_kernel<GBRNG_LCG><<<(unsigned)blocks, T, 0, st>>>(a);
    else
        ou_pt_kernel<GBRNG_RAN2><<<(unsigned)blocks, T, sizeof(int32_t) * 32 * T, st>>>(a);
    GB_CUDA(cudaGetLastError());
    if (rec) return ou_finish(h, s->n, n_rec, blocks, mean, corr, st);
    return GBRNG_OK;
}

}  // namespace gb
