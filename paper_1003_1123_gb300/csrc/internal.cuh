// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include <nvtx3/nvToolsExt.h>

#include "gbrng.h"

namespace gb {

// ---------------------------------------------------------------- errors
int fail(int code, const char* fmt, ...);
void clear_error();

#define GB_CUDA(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return ::gb::fail(GBRNG_ECUDA, "%s failed: %s (%s:%d)", #call,              \
                              cudaGetErrorString(e_), __FILE__, __LINE__);              \
    } while (0)

#define GB_CHECK(expr)                                                                  \
    do {                                                                                \
        int rc_ = (expr);                                                               \
        if (rc_ != GBRNG_OK) return rc_;                                                \
    } while (0)

// Status values written by kernels into the handle's device status word.
enum : int { DEV_OK = 0, DEV_TIMEOUT = 1 };

// NVTX range named after the C ABI call, open for the call's duration (a
// no-op unless a profiler or tracer is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---------------------------------------------------------------- handle
struct Handle {
    int kind = 0;
    uint64_t seed = 0;
    int64_t n = 0;       // streams (per-thread kinds) or threads per step (LFG)
    int device = 0;

    uint4* taus = nullptr;     // [n] (y1, y2, y3, y4)
    int32_t* r2 = nullptr;     // [35][n]: idum, idum2, iy, iv[0..31]
    uint32_t* lcg = nullptr;   // [n] Quick and Dirty LCG words

    // Lagged Fibonacci: the sequence value at position p (p >= -order_max ll)
    // lives in ring[p mod ring_size]; ring_size >= order_max (ll + (ll - sl)),
    // where order_max (2 or 4) is the highest leap order the ring serves.  The
    // allocation holds ring_size + ring_mirror(ring_size) words: the ring,
    // then a copy of its first ring_mirror(ring_size) slots.
    int row = -1;
    int32_t sl = 0, ll = 0;
    int order_max = 2;
    uint32_t ring_size = 0;
    uint32_t* ring = nullptr;
    int64_t pos = 0;           // next position to generate

    // scratch owned by the handle
    uint64_t* progress = nullptr;   // grid-barrier arrival counter (LFG)
    int64_t progress_cap = 0;
    int* dstatus = nullptr;         // device status word
    double* partials = nullptr;     // per-block reduction partials
    int64_t partials_cap = 0;
    double* dstats = nullptr;       // 8 doubles of final statistics
    float2* eacc = nullptr;         // paper-form runs: per-oscillator energy sum (Kahan s, c)
    int64_t eacc_cap = 0;
    float* adj = nullptr;           // adjoint checkpoints and noise (history or one segment)
    size_t adj_bytes = 0;
};

// Mirrored slots after a Lagged Fibonacci ring of R slots: 32768 (a resident
// CTA's step region at 1e6 oscillators is 26368), at most a quarter of the
// ring (so that small rings do not store every value twice), a multiple of
// 32 (R >= 6620 for every Table I row, so never below 1632 >= one block).
inline uint32_t ring_mirror(uint32_t R)
{
    const uint32_t q = (R / 4) & ~31u;
    return q < 32768u ? q : 32768u;
}

// Device attributes used for launch sizing (cached per device).
struct DevInfo {
    int sms = 0;
    int max_threads_sm = 0;
    size_t smem_optin = 0;
};
int dev_info(int device, DevInfo* out);

int ensure_partials(Handle* h, int64_t count);
int ensure_progress(Handle* h, int64_t count);

uint64_t wait_limit_ns();
int64_t test_stall_chunk();

// Kernel-side parameters of one Langevin system (binary32 coefficients,
// computed once on the host from the double parameters).
struct LdCoef {
    float cdt, cva, ckm, cs, sv, kT, K, hm;
};
LdCoef make_coef(const ld_system* s);
int check_system(const ld_system* s, bool need_rng);

// Per-thread generator entry points (fill.cu, ld.cu)
int fill_u32_pt(Handle* h, uint32_t* dst, int64_t n, cudaStream_t st);
int fill_uniform_pt(Handle* h, float* dst, int64_t n, cudaStream_t st);
int fill_normal_pt(Handle* h, float* dst, int64_t n, cudaStream_t st);
int ld_init_pt(const ld_system* s, cudaStream_t st);
int ld_run_pt(const ld_system* s, int64_t n_steps, ld_stats* out, cudaStream_t st);

// Lagged Fibonacci entry points (lfg.cu)
int lfg_seed(Handle* h, cudaStream_t st);
int lfg_order_for_new_handle();   // highest leap order a new handle's ring serves
int lfg_fill(Handle* h, void* dst, int64_t n, int mode, cudaStream_t st);  // mode 0 u32, 1 uniform, 2 normal
int lfg_ld(const ld_system* s, int64_t n_steps, int init, ld_stats* out, cudaStream_t st);

// Paper-form runs, one launch per step (stepwise.cu, lfg.cu).
int ld_run_stepwise_pt(const ld_system* s, int64_t n_steps, ld_stats* out, cudaStream_t st);
int lfg_ld_stepwise(const ld_system* s, int64_t n_steps, ld_stats* out, cudaStream_t st);
int ensure_eacc(Handle* h, int64_t n);
int ensure_adj(Handle* h, size_t bytes);
// Final-state sums and the per-oscillator energy sums of a paper-form run.
int stepwise_stats(Handle* h, const ld_system* s, int64_t n_steps, ld_stats* out, cudaStream_t st);

// Overdamped 1-D runs (ou.cu, lfg.cu).  Records land in
// partials[(rec * blocks + block) * 2 + {0, 1}] (sums of R and R R0).
struct OuCoef {
    float c1, cs;
};
OuCoef make_ou_coef(const ou_system* s);
int ou_run_pt(const ou_system* s, int64_t n_steps, int64_t every, double* mean, double* corr,
              cudaStream_t st);
int lfg_ou(const ou_system* s, int64_t n_steps, int64_t every, double* mean, double* corr,
           cudaStream_t st);
int ou_finish(Handle* h, int64_t n, int64_t n_rec, int64_t blocks, double* mean, double* corr,
              cudaStream_t st);

// Statistics: reduce `blocks` partials (4 doubles each) into h->dstats and
// copy to the host (synchronising st).
int finish_stats(Handle* h, int64_t blocks, int64_t n_steps, ld_stats* out, cudaStream_t st);

// Lagged Fibonacci Table I (row 4 as sl = 13470).
int lfg_lags(int row, int32_t* sl, int32_t* ll);
int lfg_default_row(int64_t n_threads);

}  // namespace gb

struct gbrng_rng : gb::Handle {};
