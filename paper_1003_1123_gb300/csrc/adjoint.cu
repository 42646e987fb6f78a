// Reverse-time adjoint of the trajectory-averaged energy
//   L = (1/S) sum_{t=1..S} sum_i ( m |v_i(t)|^2 + K_i |x_i(t)|^2 ) / 2
// under fixed noise, for the per-thread generators.
//
// Oscillators are independent, so one thread carries one oscillator through
//  A) the forward run, writing a checkpoint (x, v, generator state) at the
//     start of every segment of P steps, accumulating L and the direct part
//     of dL/dK_i, and finally the end state;
//  B) the reverse sweep, segment by segment from the last: the segment's
//     normals (3 floats per step) are either read from the history A wrote
//     when the whole run's noise fits the history limit, or regenerated
//     bit-exactly into a scratch buffer from the segment's checkpointed
//     generator state; then,
//     walking the segment backwards from its exact end state (the next
//     checkpoint, or the final state), each step is inverted,
//        v_t = (v_{t+1} + b x_{t+1} - c g_t) / (a + b dt),  x_t = x_{t+1} - dt v_t,
//     and the discrete adjoint recursion is applied:
//        lx_t = lx_{t+1} - b lv_{t+1} + [t>=1] K x_t / S,
//        lv_t = dt lx_{t+1} + a lv_{t+1} + [t>=1] m v_t / S,
//     with a = 1 - gamma dt/m, b = dt K_i/m, c = sqrt(2 gamma kT dt)/m, and
//        dL/dK_i   += -(dt/m) lv_{t+1}.x_t,
//        dL/dgamma += lv_{t+1}.(-(dt/m) v_t + c/(2 gamma) g_t),
//        dL/dkT    += lv_{t+1}.(c/(2 kT) g_t).
// Inversion only runs inside one segment (at most P steps from an exact
// state), where it is stable.  Sums over steps are Kahan-compensated binary32,
// sums over oscillators fixed-order doubles.
#include <algorithm>
#include <atomic>

#include "device.cuh"
#include "internal.cuh"

namespace gb {

struct AdjArgs {
    int64_t n, S, P, nseg;
    float* x;
    float* v;
    const float* Kper;
    LdCoef c;
    float c_over_2g, c_over_2kT, invS, m;
    uint4* taus;
    int32_t* r2;
    int64_t streams;
    float* ckpt;        // [nseg][6 + state words][n]
    float* gbuf;        // [S][3][n] history (hist) or [P][3][n] segment scratch
    int hist;
    float* dK;          // [n] or null
    double* partials;   // [grid][4]: loss, dgamma, dkT, unused
};

// 64-thread blocks with an 85-register budget: twelve blocks per SM (116736
// threads on 152 SMs), so 1e5 oscillators fit one resident wave with one
// oscillator per thread and the SMs differ by at most one block; 1% faster
// than fourteen blocks at 72 registers (at 96 registers and 128 threads the
// same system needed two oscillators per thread on 2.6 blocks per SM).
template <int KIND>
__global__ void __launch_bounds__(64, 12) adjoint_kernel(AdjArgs a)
{
    extern __shared__ int32_t tab[];   // Ran2: [32][blockDim.x]
    __shared__ double red[4 * 32];
    constexpr int SW = KIND == GBRNG_TAUS ? 4 : 35;   // state words
    constexpr int CW = 6 + SW;                         // checkpoint words
    const int64_t W = (int64_t)gridDim.x * blockDim.x;
    const LdCoef c = a.c;
    const int64_t n = a.n;
    double acc[4] = {0, 0, 0, 0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += W) {
        const float Ki = a.Kper ? a.Kper[i] : c.K;
        const float ckx = __fmul_rn(c.ckm, Ki);
        const float hK = 0.5f * Ki;
        float x[3] = {a.x[3 * i], a.x[3 * i + 1], a.x[3 * i + 2]};
        float v[3] = {a.v[3 * i], a.v[3 * i + 1], a.v[3 * i + 2]};
        TausDraw td;
        Ran2Draw rd;
        rd.tab = tab;
        rd.T = blockDim.x;
        rd.tid = threadIdx.x;
        auto load_state = [&](const float* src, int64_t stride) {
            // src == nullptr: from the generator itself
            if (KIND == GBRNG_TAUS) {
                if (!src) {
                    td.y = a.taus[i];
                } else {
                    td.y.x = __float_as_uint(src[0]);
                    td.y.y = __float_as_uint(src[stride]);
                    td.y.z = __float_as_uint(src[2 * stride]);
                    td.y.w = __float_as_uint(src[3 * stride]);
                }
            } else {
                if (!src) {
                    rd.r.idum = a.r2[i];
                    rd.r.idum2 = a.r2[a.streams + i];
                    rd.r.iy = a.r2[2 * a.streams + i];
                    #pragma unroll 4
                    for (int j = 0; j < 32; ++j)
                        tab[j * blockDim.x + threadIdx.x] = a.r2[(3 + j) * a.streams + i];
                } else {
                    rd.r.idum = __float_as_int(src[0]);
                    rd.r.idum2 = __float_as_int(src[stride]);
                    rd.r.iy = __float_as_int(src[2 * stride]);
                    #pragma unroll 4
                    for (int j = 0; j < 32; ++j)
                        tab[j * blockDim.x + threadIdx.x] = __float_as_int(src[(3 + j) * stride]);
                }
            }
        };
        auto save_state = [&](float* dst, int64_t stride) {
            if (KIND == GBRNG_TAUS) {
                dst[0] = __uint_as_float(td.y.x);
                dst[stride] = __uint_as_float(td.y.y);
                dst[2 * stride] = __uint_as_float(td.y.z);
                dst[3 * stride] = __uint_as_float(td.y.w);
            } else {
                dst[0] = __int_as_float(rd.r.idum);
                dst[stride] = __int_as_float(rd.r.idum2);
                dst[2 * stride] = __int_as_float(rd.r.iy);
                #pragma unroll 4
                for (int j = 0; j < 32; ++j)
                    dst[(3 + j) * stride] = __int_as_float(tab[j * blockDim.x + threadIdx.x]);
            }
        };
        // ---------------- A: forward with checkpoints
        load_state(nullptr, 0);
        Kahan loss, xsq;
        for (int64_t seg = 0; seg < a.nseg; ++seg) {
            float* ck = a.ckpt + seg * CW * n + i;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                ck[q * n] = x[q];
                ck[(3 + q) * n] = v[q];
            }
            save_state(ck + 6 * n, n);
            const int64_t len = min(a.P, a.S - seg * a.P);
            for (int64_t t = 0; t < len; ++t) {
                float g[3];
                if (KIND == GBRNG_TAUS) td.normals3(g[0], g[1], g[2]); else rd.normals3(g[0], g[1], g[2]);
                if (a.hist) {
#pragma unroll
                    for (int q = 0; q < 3; ++q) a.gbuf[((seg * a.P + t) * 3 + q) * n + i] = g[q];
                }
#pragma unroll
                for (int q = 0; q < 3; ++q) em_component(c.cdt, c.cva, ckx, c.cs, g[q], x[q], v[q]);
                loss.add(energy3(hK, c.hm, x[0], x[1], x[2], v[0], v[1], v[2]));
                xsq.add(__fmaf_rn(x[2], x[2], __fmaf_rn(x[1], x[1], __fmul_rn(x[0], x[0]))));
            }
        }
        // end state: the system advances exactly as ld_run would
        a.x[3 * i] = x[0], a.x[3 * i + 1] = x[1], a.x[3 * i + 2] = x[2];
        a.v[3 * i] = v[0], a.v[3 * i + 1] = v[1], a.v[3 * i + 2] = v[2];
        if (KIND == GBRNG_TAUS) {
            a.taus[i] = td.y;
        } else {
            a.r2[i] = rd.r.idum;
            a.r2[a.streams + i] = rd.r.idum2;
            a.r2[2 * a.streams + i] = rd.r.iy;
            #pragma unroll 4
            for (int j = 0; j < 32; ++j)
                a.r2[(3 + j) * a.streams + i] = tab[j * blockDim.x + threadIdx.x];
        }
        // ---------------- B: reverse sweep
        const float inv_ab = __frcp_rn(__fmaf_rn(ckx, c.cdt, c.cva));
        float lx[3], lv[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            lx[q] = Ki * x[q] * a.invS;
            lv[q] = a.m * v[q] * a.invS;
        }
        Kahan dk, dg, dT;
        float xe[3] = {x[0], x[1], x[2]}, ve[3] = {v[0], v[1], v[2]};   // segment end state
        for (int64_t seg = a.nseg - 1; seg >= 0; --seg) {
            const float* ck = a.ckpt + seg * CW * n + i;
            const int64_t len = min(a.P, a.S - seg * a.P);
            if (!a.hist) {
                load_state(ck + 6 * n, n);
                for (int64_t t = 0; t < len; ++t) {
                    float g[3];
                    if (KIND == GBRNG_TAUS) td.normals3(g[0], g[1], g[2]); else rd.normals3(g[0], g[1], g[2]);
#pragma unroll
                    for (int q = 0; q < 3; ++q) a.gbuf[(t * 3 + q) * n + i] = g[q];
                }
            }
            const float* gseg = a.gbuf + (a.hist ? seg * a.P * 3 * n : 0);
            float xn[3] = {xe[0], xe[1], xe[2]}, vn[3] = {ve[0], ve[1], ve[2]};
            for (int64_t t = len - 1; t >= 0; --t) {
                const int64_t tg = seg * a.P + t;   // global step index
                float gk[3], xt[3], vt[3];
                float ddk = 0.f, ddg = 0.f, ddT = 0.f;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    gk[q] = gseg[(t * 3 + q) * n + i];
                    vt[q] = (vn[q] + ckx * xn[q] - c.cs * gk[q]) * inv_ab;
                    xt[q] = xn[q] - c.cdt * vt[q];
                }
                if (t == 0) {   // the checkpoint holds the exact state
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        xt[q] = ck[q * n];
                        vt[q] = ck[(3 + q) * n];
                    }
                }
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    ddk += lv[q] * xt[q];
                    ddg += lv[q] * (a.c_over_2g * gk[q] - c.ckm * vt[q]);
                    ddT += lv[q] * gk[q];
                    const float w = tg >= 1 ? a.invS : 0.f;
                    const float lxn = lx[q] - ckx * lv[q] + w * Ki * xt[q];
                    const float lvn = c.cdt * lx[q] + c.cva * lv[q] + w * a.m * vt[q];
                    lx[q] = lxn;
                    lv[q] = lvn;
                }
                dk.add(-c.ckm * ddk);
                dg.add(ddg);
                dT.add(a.c_over_2kT * ddT);
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    xn[q] = xt[q];
                    vn[q] = vt[q];
                }
            }
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                xe[q] = ck[q * n];
                ve[q] = ck[(3 + q) * n];
            }
        }
        if (a.dK) a.dK[i] = (float)(dk.value() + 0.5 * (double)a.invS * xsq.value());
        acc[0] += loss.value() * (double)a.invS;
        acc[1] += dg.value();
        acc[2] += dT.value();
    }
    block_reduce_sum<4>(acc, red);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) a.partials[4 * blockIdx.x + k] = acc[k];
}

// Largest noise history (bytes) ld_backward keeps; -1: half the free device
// memory at the call.
static std::atomic<int64_t> g_hist_limit{-1};

}  // namespace gb

using namespace gb;

extern "C" int ld_set_adjoint_history_limit(int64_t bytes)
{
    if (bytes < -1) return fail(GBRNG_EINVAL, "history limit must be >= -1, got %lld", (long long)bytes);
    g_hist_limit.store(bytes);
    return GBRNG_OK;
}

extern "C" int ld_backward(ld_system* sys, int64_t n_steps, int ckpt_every, float* dK_per,
                           double* dgamma, double* dkT, double* loss, void* stream)
{
    NvtxRange range("ld_backward");
    GB_CHECK(check_system(sys, true));
    Handle* h = sys->rng;
    if (h->kind != GBRNG_TAUS && h->kind != GBRNG_RAN2)
        return fail(GBRNG_EINVAL, "ld_backward needs a per-thread generator (Taus or Ran2)");
    if (n_steps < 1 || ckpt_every < 1) return fail(GBRNG_EINVAL, "need n_steps >= 1, ckpt_every >= 1");
    if (!(sys->gamma > 0) || !(sys->kT > 0)) return fail(GBRNG_EINVAL, "need gamma > 0 and kT > 0");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = sys->n;
    if (n == 0) {
        if (dgamma) *dgamma = 0;
        if (dkT) *dkT = 0;
        if (loss) *loss = 0;
        return GBRNG_OK;
    }
    const int64_t P = std::min<int64_t>(ckpt_every, n_steps);
    const int64_t nseg = (n_steps + P - 1) / P;
    const int SW = h->kind == GBRNG_TAUS ? 4 : 35;
    const size_t ck_bytes = sizeof(float) * (size_t)nseg * (6 + SW) * (size_t)n;
    // Noise buffer: the whole run's (12 B per oscillator-step) when it fits
    // the limit, else one segment's.  The scratch stays with the handle for
    // the next call (this call synchronises its stream before returning), and
    // the automatic limit counts what the handle already holds as free.
    const size_t hist_bytes = sizeof(float) * 3 * (size_t)n_steps * (size_t)n;
    const size_t seg_bytes = sizeof(float) * (size_t)P * 3 * (size_t)n;
    int64_t limit = g_hist_limit.load();
    if (limit < 0) {
        size_t free_b = 0, total_b = 0;
        limit = cudaMemGetInfo(&free_b, &total_b) == cudaSuccess
                    ? (int64_t)((free_b + h->adj_bytes) / 2) : 0;
        cudaGetLastError();
    }
    bool hist = n_steps > P && (int64_t)hist_bytes <= limit;
    if (hist && ensure_adj(h, ck_bytes + hist_bytes) != GBRNG_OK) hist = false;
    if (!hist) GB_CHECK(ensure_adj(h, ck_bytes + seg_bytes));
    float* scratch = h->adj;
    DevInfo di;
    GB_CHECK(dev_info(h->device, &di));
    const int T = 64;
    const size_t smem = h->kind == GBRNG_RAN2 ? sizeof(int32_t) * 32 * T : 0;
    int occ = 0;
    cudaError_t e = h->kind == GBRNG_TAUS
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, adjoint_kernel<GBRNG_TAUS>, T, smem)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, adjoint_kernel<GBRNG_RAN2>, T, smem);
    if (e != cudaSuccess || occ < 1) occ = 1;
    // one full resident wave at most; oscillators i, i + W, ... per thread
    const int64_t blocks = std::min<int64_t>((int64_t)di.sms * occ, (n + T - 1) / T);
    GB_CHECK(ensure_partials(h, blocks));
    AdjArgs a;
    a.n = n;
    a.S = n_steps;
    a.P = P;
    a.nseg = nseg;
    a.x = sys->x;
    a.v = sys->v;
    a.Kper = sys->K_per;
    a.c = make_coef(sys);
    const double cval = sqrt(2.0 * sys->gamma * sys->kT * sys->dt) / sys->m;
    a.c_over_2g = (float)(cval / (2.0 * sys->gamma));
    a.c_over_2kT = (float)(cval / (2.0 * sys->kT));
    a.invS = (float)(1.0 / (double)n_steps);
    a.m = (float)sys->m;
    a.taus = h->taus;
    a.r2 = h->r2;
    a.streams = h->n;
    a.ckpt = scratch;
    a.gbuf = scratch + ck_bytes / sizeof(float);
    a.hist = hist ? 1 : 0;
    a.dK = dK_per;
    a.partials = h->partials;
    if (h->kind == GBRNG_TAUS)
        adjoint_kernel<GBRNG_TAUS><<<(unsigned)blocks, T, smem, st>>>(a);
    else
        adjoint_kernel<GBRNG_RAN2><<<(unsigned)blocks, T, smem, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(GBRNG_ECUDA, "adjoint launch failed: %s", cudaGetErrorString(e));
    ld_stats tmp;
    GB_CHECK(finish_stats(h, blocks, 1, &tmp, st));
    if (loss) *loss = tmp.sum_x2;
    if (dgamma) *dgamma = tmp.sum_v2;
    if (dkT) *dkT = tmp.sum_xv;
    return GBRNG_OK;
}
