/*
 * gbrng.h -- C ABI of the GB300-native on-the-fly RNG + Langevin-dynamics
 * library (sm_103a).
 *
 * The method is that of Zhmurov, Rybnikov, Kholodov & Barsegov, "Efficient
 * pseudo-random number generators for biomolecular simulations on graphics
 * processors": three generators -- Hybrid Taus and Ran2, one generator per
 * thread (Sec. III.B, Algorithms 1-2), and the additive Lagged Fibonacci
 * generator shared by all threads (Sec. III.C, Algorithm 3, Table I) --
 * feeding Box-Muller normals (Sec. II.A) into the Langevin step of N
 * independent three-dimensional harmonic oscillators (Sec. I and IV).  Also:
 * the Quick and Dirty LCG of Eq. 1 (Sec. II.B) as a fourth per-thread kind,
 * the overdamped one-dimensional test of Sec. IV (Eq. 4-5), the paper's
 * one-launch-per-step form of the fused step, a batched graph of many
 * systems and a reverse-time adjoint.
 *
 * Conventions for every entry point:
 *  - The return value is a gbrng_status; nothing aborts.  On failure
 *    gbrng_last_error() returns a message (thread-local, valid until the next
 *    call on the same thread).
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  All device work is ordered on that stream.  Calls that return
 *    host-side results (ld_stats, state blobs, scalar gradients) synchronise
 *    that stream before returning; the others return after enqueueing.
 *  - Device pointers passed in (dst, x, v, K_per, dK_per) are owned by the
 *    caller and must be device-accessible memory of the handle's device.
 *  - The library owns generator state and scratch.  A handle allocates its
 *    state in rng_init* and frees everything in rng_destroy.
 *  - A handle is not thread-safe; calls on one handle must not overlap.
 *  - Device errors map to GBRNG_ECUDA; a device-side wait that exceeded its
 *    limit (Lagged Fibonacci grid barrier) maps to GBRNG_ETIMEOUT, after which
 *    the handle's state is undefined (rng_set_state or a new handle recovers).
 *  - Every call that launches work opens an NVTX range named after the call
 *    (a no-op unless a profiler or tracer is attached).
 */
#ifndef GBRNG_H
#define GBRNG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { GBRNG_TAUS = 0, GBRNG_RAN2 = 1, GBRNG_LAGFIB = 2, GBRNG_LCG = 3 } gbrng_kind;

typedef enum {
    GBRNG_OK = 0,
    GBRNG_EINVAL = -1,    /* bad argument (null pointer, size, kind, parameter)  */
    GBRNG_ENOMEM = -2,    /* device or host allocation failed                   */
    GBRNG_ECUDA = -3,     /* a CUDA runtime call or kernel failed               */
    GBRNG_ETIMEOUT = -4,  /* a bounded device wait ran out                      */
    GBRNG_ELAGS = -5,     /* the requested Lagged Fibonacci row cannot be used  */
    GBRNG_ESTATE = -6     /* a state blob does not match the handle             */
} gbrng_status;

typedef struct gbrng_rng* gbrng_t;   /* opaque generator handle */

/* ---------------------------------------------------------------- generators */

/* Create a generator of `kind` on the current CUDA device.
 * Hybrid Taus (Algorithm 1): n_streams independent streams, state 4 x uint32
 *   per stream (y1, y2, y3 Tausworthe words, y4 LCG word).
 * Ran2 (Algorithm 2): n_streams independent streams, state 35 x int32 per
 *   stream (idum, idum2, iy, iv[32]), initialised by the NTAB+8-step warm-up.
 * Lagged Fibonacci (Algorithm 3): one shared sequence; n_streams is the
 *   number N of threads (oscillators) per step, which selects the Table I row:
 *   the smallest row with sl > 4N and ll - sl > 4N, else the last row.
 * Quick and Dirty LCG (Eq. 1, m = 2^32: x <- 1664525 x + 1013904223, output
 *   the new word): n_streams independent streams, one uint32 each.  The
 *   paper's speed benchmark and statistical negative control; fills, ld_run,
 *   ld_run_stepwise and ou_run accept it, ld_run_batched, ld_backward and
 *   ld_run_noalloc return GBRNG_EINVAL.
 * Seeding (Sec. III.B asks for an independent source): word k of stream s is
 * the low 32 bits of SplitMix64 at counter 8s+k; Taus words 1-3 below 2, 8,
 * 16 are raised by 2, 8, 16; Ran2 idum = 1 + (word mod (m1-1)); the LCG word
 * is word 0 of its stream as it stands; Lagged
 * Fibonacci seed w (x_{w-ll}) uses counter w, and x_{-ll} is forced odd.
 * Seeding runs on the GPU.  n_streams >= 1.  *out receives the handle. */
int rng_init(gbrng_t* out, int kind, uint64_t seed, int64_t n_streams, void* stream);

/* Lagged Fibonacci with an explicit Table I row (0-9, or -1 for the default
 * row of n_threads).  Row 4 is used as (sl, ll) = (13470, 23209): the printed
 * sl = 12470 gives a reducible trinomial.  GBRNG_ELAGS for a row outside 0-9. */
int rng_init_lfg(gbrng_t* out, uint64_t seed, int64_t n_threads, int lag_row, void* stream);

/* Free the handle and everything it owns (waits for its pending work). */
int rng_destroy(gbrng_t rng);

/* New handle with an identical copy of src's state (device-to-device). */
int rng_clone(gbrng_t src, gbrng_t* out, void* stream);

/* Query a handle.  Any output pointer may be NULL.  position = number of
 * Lagged Fibonacci values generated so far (0 for per-thread kinds). */
int rng_info(gbrng_t rng, int* kind, int64_t* n_streams, int* lag_row, int64_t* position);

/* Table I lags of a row (row 4 as read above).  GBRNG_ELAGS if row not in 0-9. */
int rng_lfg_lags(int row, int32_t* sl, int32_t* ll);

/* Default Table I row for n_threads (see rng_init). */
int rng_lfg_default_row(int64_t n_threads);

/* Fill dst_dev[0..n) with raw 32-bit draws.  Per-thread kinds: dst[d*S + s]
 * is the d-th next draw of stream s (S = n_streams); when S does not divide
 * n, streams s < n mod S draw once more.  Lagged Fibonacci: dst[k] is the
 * next value x_{p+k} of the shared sequence.  Ran2 draws are its integer
 * output iy in [1, m1-1].  n >= 0; the handle advances by the draws made. */
int rng_fill_u32(gbrng_t rng, uint32_t* dst_dev, int64_t n, void* stream);

/* As rng_fill_u32 with each draw converted to binary32 in [0, 1]:
 * Taus and Lagged Fibonacci u = fl(raw) * 2^-32 (the multiplier of
 * Algorithm 1); Ran2 u = min(fl(AM * fl(iy)), RNMX) with AM = fl(1/m1) and
 * RNMX the largest float below 1 (Algorithm 2). */
int rng_fill_uniform(gbrng_t rng, float* dst_dev, int64_t n, void* stream);

/* Box-Muller normals, n even.  Pair e = (dst[2e], dst[2e+1]) =
 * sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2) from two consecutive draws of one
 * stream; pair e = d*S + s belongs to stream s (Lagged Fibonacci: the values
 * x_{p+2e}, x_{p+2e+1}).  Taus/Lagged Fibonacci map raw words to the open
 * interval u = ((raw >> 9) + 1/2) 2^-23; Ran2 uses its uniform.  dst_dev must
 * be 8-byte aligned (pairs are stored as float2). */
int rng_fill_normal(gbrng_t rng, float* dst_dev, int64_t n, void* stream);

/* Host blob holding the complete generator state:
 *   gbrng_state_header, then
 *   Taus:  uint32 [S][4]   (y1, y2, y3, y4 per stream)
 *   Ran2:  int32  [S][35]  (idum, idum2, iy, iv[0..31] per stream)
 *   Lagged Fibonacci: uint32 [ll] = x_{p-ll} .. x_{p-1} in sequence order.
 * rng_get_state / rng_set_state synchronise the device first and copy with
 * the legacy default stream.  bytes must equal rng_state_bytes; a blob whose
 * header does not match the handle gives GBRNG_ESTATE. */
typedef struct {
    uint32_t magic;       /* 0x4E524247 ("GBRN") */
    uint32_t version;     /* 1 */
    int32_t kind;
    int32_t lag_row;      /* -1 for per-thread kinds */
    int64_t n_streams;
    int64_t position;     /* Lagged Fibonacci p; 0 otherwise */
    uint64_t payload_bytes;
} gbrng_state_header;

int rng_state_bytes(gbrng_t rng, size_t* bytes);
int rng_get_state(gbrng_t rng, void* host, size_t bytes);
int rng_set_state(gbrng_t rng, const void* host, size_t bytes);

/* Bound (nanoseconds, default 2e9) on every device-side spin wait of the
 * library (the Lagged Fibonacci grid barrier between rounds).  A wait that
 * runs out makes the kernel record GBRNG_ETIMEOUT and return; the generator
 * position is then not advanced and its ring contents are unspecified (reseed
 * or set_state before further use).  Process-wide. */
int rng_set_wait_limit_ns(uint64_t ns);

/* Test hook for the bounded waits: from the next Lagged Fibonacci launch on,
 * CTA number `chunk` modulo the launch's grid size never arrives at the grid
 * barrier, so every CTA's wait runs out after the limit and a launch of more
 * than one round returns GBRNG_ETIMEOUT (no fault, no trap).  -1 switches the
 * hook off (the default).  Process-wide. */
int gbrng_test_stall_chunk(int64_t chunk);

/* Leap order k of the Lagged Fibonacci schedule (Sec. III.C, Algorithm 3, in
 * the leap form x_p = sum_j C(k, j) x_{p - (k-j) ll - j (ll - sl)}, k + 1 lag
 * reads per value, rounds of up to k (ll - sl) positions between grid
 * barriers).  0 (the default) lets each launch take its own order (2); 1, 2
 * or 4 forces that order on every later launch.  A handle's ring serves order
 * 4 only when 4 was set before the handle was created (its ring is then
 * 4 (2 ll - sl) words instead of 2 (2 ll - sl)); on other handles an order-4
 * setting runs order 2.  Every order yields the same sequence bit for bit:
 * this only trades lag reads against barrier rounds.  Process-wide;
 * GBRNG_EINVAL for other values. */
int gbrng_set_lfg_order(int k);

/* --------------------------------------------------------- Langevin dynamics */

/* One system of n independent 3-D oscillators (Sec. IV): caller-owned device
 * arrays x, v of n x 3 binary32 (oscillator-major, x[3i+c]); K_per is a
 * device array of n spring constants or NULL for the scalar K. */
typedef struct {
    int64_t n;
    float* x;
    float* v;
    const float* K_per;
    double K, m, gamma, kT, dt;
    gbrng_t rng;          /* per-thread kinds need n_streams >= n */
} ld_system;

/* Statistics of one run: the final snapshot sums over all oscillators and
 * components, and the time average over the run's steps of the total energy
 * E(t) = sum_i (m |v_i(t)|^2 + K_i |x_i(t)|^2) / 2 (states after each step). */
typedef struct {
    double sum_x2, sum_v2, sum_xv, energy_time_avg;
    int64_t steps;
} ld_stats;

/* Equilibrium start: spends two draw-steps of the generator; step 0 gives
 * x = sqrt(kT/K_i) g, step 1 gives v = sqrt(kT/m) g (three normals per
 * oscillator per step as in ld_run). */
int ld_init_equilibrium(ld_system* sys, void* stream);

/* Advance the system by n_steps of the underdamped Euler-Maruyama step of
 * m dV/dt = -gamma V - K R + G, G = g sqrt(2 gamma kT dt) (Sec. I):
 *   v' = (1 - gamma dt/m) v - (dt K_i/m) x + (sqrt(2 gamma kT dt)/m) g,
 *   x' = x + dt v,
 * with three Box-Muller normals per oscillator per step drawn from four
 * uniforms: (g_x, g_y) from (u1, u2), g_z from (u3, u4) (cosine branch).
 * Per-thread kinds: oscillator i uses stream i.  Lagged Fibonacci: oscillator
 * j at step t uses sequence positions p0 + 4(j + N t) + r, r = 0..3.
 * binary32 arithmetic order (exact, no contraction):
 *   coefficients (double, rounded once): cdt = dt, cva = 1 - (gamma dt)/m,
 *   ckm = dt/m, cs = sqrt(2 gamma kT dt)/m;  ckx = ckm * K_i;
 *   per component: t = fma(-ckx, x, cs * g); v' = fma(cva, v, t);
 *   x' = fma(cdt, v, x).
 * out_host (nullable) receives the run's statistics (synchronises stream).
 * Requirements: n >= 0, n_steps >= 0, m > 0, dt > 0, gamma >= 0, kT >= 0,
 * K > 0 (or K_per given). */
int ld_run(ld_system* sys, int64_t n_steps, ld_stats* out_host, void* stream);

/* ----------------------------------------------- overdamped 1-D Langevin */

/* n independent 1-D particles in the harmonic potential V = k_sp R^2 / 2
 * under overdamped Langevin dynamics (Sec. IV, Eq. 4-5): caller-owned device
 * array R of n binary32 positions. */
typedef struct {
    int64_t n;
    float* R;
    double k_sp, xi, kT, dt;
    gbrng_t rng;          /* per-thread kinds need n_streams >= n */
} ou_system;

/* Advance by n_steps of Eq. 5, R' = R - (k_sp dt / xi) R + g sqrt(2 kT dt / xi)
 * (the printed random term g sqrt(2 kT xi dt) is the random force times dt;
 * Eq. 4 divides it by xi), in binary32 as R' = fma(cs, g, fma(-c1, R, R)) with
 * c1 = fl(k_sp dt / xi) and cs = fl(sqrt(2 kT dt / xi)) (double expressions
 * rounded once).  One normal per particle-step: the cosine branch of
 * Box-Muller on two draws (per-thread kinds: stream i; Lagged Fibonacci:
 * positions p0 + 2(i + n t) + r, r = 0, 1).  Records r = 0 .. n_steps/every
 * after r*every steps: mean_host[r] = (1/n) sum_i R_i and corr_host[r] =
 * (1/n) sum_i R_i R_i(0), R(0) the positions on entry (the paper's <R(t)> and
 * <R(t)R(0)>); both are host arrays of n_steps/every + 1 doubles, or both NULL
 * (no records).  Lagged Fibonacci: every step is one round of 2n positions,
 * 2n <= ll - sl below position ll and <= 2(ll - sl) after, else GBRNG_ELAGS and
 * nothing runs.  Requirements: n >= 1, n_steps >= 0, every >= 1, k_sp > 0,
 * xi > 0, kT >= 0, dt > 0.  Synchronises the stream when records are
 * requested; scratch (16 bytes per record per 256 particles) is the handle's. */
int ou_run(ou_system* sys, int64_t n_steps, int64_t every, double* mean_host, double* corr_host,
           void* stream);

/* Paper-form run, the reference form of ld_run (Algorithms 1-3 as printed,
 * Fig. 2-3, Sec. III.C): one kernel launch per step; every launch loads each
 * oscillator's generator state (Ran2's shuffle table in global memory), x, v
 * and its energy sum from global memory, takes one step and stores them back.
 * Same draws, stream positions and binary32 operations as ld_run, so x, v and
 * the generator state come out bit for bit equal to ld_run's; the statistics
 * equal ld_run's up to summation order.  Lagged Fibonacci: a step's 4N
 * positions must be independent of each other, 4N <= ll - sl while the
 * generator is below position ll and 4N <= 2 (ll - sl) after (the leap form),
 * else GBRNG_ELAGS and nothing runs.  Owns 8 bytes of scratch per oscillator
 * (grown on demand, freed in rng_destroy).  out_host as in ld_run. */
int ld_run_stepwise(ld_system* sys, int64_t n_steps, ld_stats* out_host, void* stream);

/* Run n_sys independent systems (own handle, parameters and arrays each;
 * per-thread kinds only) as one persistent launch per steps-per-launch chunk,
 * captured once into a CUDA graph.  tune = {threads per block, oscillators
 * per thread, steps per launch} or NULL to autotune (results cached per shape
 * in the file named by $GBRNG_TUNE_CACHE, if set).  Trajectories and
 * generator states equal those of one ld_run per system bit for bit.
 * out (nullable) receives n_sys stats (synchronises stream). */
int ld_run_batched(ld_system* sys, int n_sys, int64_t n_steps, const int* tune,
                   ld_stats* out, void* stream);

/* The launch shape the autotuner chose for these systems' shape (their kinds
 * and sizes), as tune_out = {threads per block, oscillators per thread, steps
 * per launch (0: all steps in one launch)}; GBRNG_EINVAL if that shape has not
 * been autotuned in this process or read from $GBRNG_TUNE_CACHE.  Runs nothing
 * (an introspection call: one replay of the graph launches ceil(steps / L)
 * persistent kernels and one reduction). */
int ld_batched_tune(const ld_system* sys, int n_sys, int* tune_out);

/* Reverse-time adjoint of L = (1/S) sum_{t=1..S} E(t) (S = n_steps) under the
 * fixed noise of the generator, starting from the system's current state.
 * Generator states and (x, v) are checkpointed every ckpt_every steps.  The
 * reverse sweep reads the noise the forward run stored (12 B per
 * oscillator-step) when that history fits the limit of
 * ld_set_adjoint_history_limit, and otherwise regenerates each segment's noise
 * bit-exactly from its checkpoint; the results are identical.  The scratch
 * (checkpoints, noise) stays with the handle for later calls until
 * rng_destroy.
 * Leaves the system advanced exactly as ld_run(sys, n_steps) would.
 * dK_per (device [n], nullable) receives dL/dK_i; *dgamma, *dkT (nullable)
 * receive dL/dgamma, dL/dkT; *loss (nullable) receives L.  Per-thread kinds
 * only; requires gamma > 0, kT > 0, n_steps >= 1, ckpt_every >= 1.
 * GBRNG_ENOMEM if the scratch cannot be allocated.  Synchronises stream. */
int ld_backward(ld_system* sys, int64_t n_steps, int ckpt_every, float* dK_per,
                double* dgamma, double* dkT, double* loss, void* stream);

/* The largest noise history (bytes) ld_backward keeps instead of regenerating
 * the noise segment by segment: 0 always regenerates; -1 (the default) allows
 * half the device memory free at the call (counting the handle's own adjoint
 * scratch as free).  Process-wide; GBRNG_EINVAL for
 * values below -1.  (The paper has no adjoint; this trades memory for the
 * second generator pass of the reverse sweep.) */
int ld_set_adjoint_history_limit(int64_t bytes);

/* ld_run for callers that cannot allocate device memory when they step a
 * system.  ld_run may allocate or grow the handle's scratch with cudaMalloc on
 * any call, and some callers cannot allow that: a real-time loop cannot let a
 * step wait on cudaMalloc, which may synchronise the device; an application
 * that gives the library a fixed memory budget, or owns all device memory
 * through its own pool, has no room for allocations it did not make.  This
 * entry point performs the same run for the per-thread generators (Hybrid
 * Taus, Ran2) with the same arguments and results, and allocates nothing.
 * (The paper has no counterpart: it is a property of this library's memory
 * management.)
 * Its scratch is a fixed static device array of 8192 x 4 + 4 doubles (about
 * 256 KiB) that every GPU which loads the library holds until the process
 * exits; a launch that would need more than 8192 blocks of partial sums is
 * rejected with GBRNG_EINVAL (a launch uses at most SMs x 32 blocks, 4864 on a
 * GB300).  The first call on a device looks up the array's device address
 * (with that device current, which must be the generator's device) and keeps
 * it for the process: make that first call before any stream capture, and do
 * not call it again on a device after cudaDeviceReset.  All calls share the
 * array and each overwrites what it reads, so calls whose GPU work overlaps
 * (other streams, other threads) race; serialise them.  out_host non-NULL
 * reads the statistics back and synchronises the stream (the host waits for
 * the run); on a stream in capture mode that is refused with GBRNG_EINVAL
 * before any work is queued.  It runs one oscillator a thread, so Hybrid Taus
 * systems that fill a resident wave run about 4% slower than in ld_run, which
 * takes two.  Other requirements and errors as ld_run. */
int ld_run_noalloc(ld_system* sys, int64_t n_steps, ld_stats* out_host, void* stream);

/* ----------------------------------------------------------------- errors */
const char* gbrng_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GBRNG_H */
