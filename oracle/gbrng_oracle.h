/*
 * gbrng_oracle.h -- plain, serial CPU oracle for the on-the-fly RNG +
 * Langevin-dynamics hot path of Zhmurov, Rybnikov, Kholodov & Barsegov,
 * "Efficient pseudo-random number generators for biomolecular simulations
 * on graphics processors".
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or constant with the CUDA library: every constant
 * below is restated here from the paper (Algorithm 1, Algorithm 2, Table I)
 * or from the readings listed at the top of gbrng_oracle.c.
 *
 * Functions whose results have no external pin say "parity unpinned" in
 * their comment; every other function is pinned by tests/test_oracle_*.py.
 */
#ifndef GBRNG_ORACLE_H
#define GBRNG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_TAUS = 0, OR_RAN2 = 1, OR_LAGFIB = 2, OR_LCG = 3 };

/* One generator bundle.  Per-thread kinds hold n_streams independent
 * streams; the Lagged Fibonacci kind holds one shared sequence (ring of ll
 * words, slot p mod ll holds the latest value at a position congruent to p). */
typedef struct {
    int32_t kind;
    int32_t ll, sl;      /* Lagged Fibonacci lags (Table I); unused otherwise */
    int64_t n_streams;   /* per-thread: streams; Lagged Fibonacci: threads N  */
    int64_t pos;         /* Lagged Fibonacci: next sequence position p >= 0   */
    void*   state;       /* Taus: uint32[n][4]  (y1,y2,y3,y4)
                            Ran2: int32[n][35]  (idum, idum2, iy, iv[32])
                            Lagged Fibonacci: uint32[ll] ring
                            LCG: uint32[n]                                 */
} or_gen;

/* ---- seeding (Sec. III.B; counter-based reading) ---------------------- */
uint64_t or_splitmix64(uint64_t seed, uint64_t idx);
void     or_taus_seed(uint64_t seed, int64_t n, uint32_t* st);
void     or_ran2_seed(uint64_t seed, int64_t n, int32_t* st);
void     or_lfg_seed(uint64_t seed, int32_t ll, uint32_t* ring);
void     or_lcg_seed(uint64_t seed, int64_t n, uint32_t* st);
void     or_seed_streams(int kind, uint64_t seed, const int64_t* idx, int64_t n, void* st);
int      or_lfg_table(int row, int32_t* sl, int32_t* ll);   /* Table I */
int      or_lfg_default_row(int64_t n_threads);

/* ---- single draws ---------------------------------------------------- */
uint32_t or_taus_next(uint32_t* y);                 /* Algorithm 1 */
uint32_t or_taus_component(uint32_t y, int which);  /* one Tausworthe step */
int32_t  or_ran2_schrage(int32_t x, int which);     /* a*x mod m, Schrage */
int32_t  or_ran2_next(int32_t* st);                 /* Algorithm 2 */
uint32_t or_lfg_next(or_gen* g);                    /* Algorithm 3 */
uint32_t or_lcg_next(uint32_t* x);                  /* Eq. 1, m = 2^32 */

/* ---- conversions ------------------------------------------------------ */
float  or_u01_f32(uint32_t raw);          /* fl(raw) * 2^-32, in [0,1]       */
double or_open01(uint32_t raw);           /* ((raw>>9)+1/2) * 2^-23, in (0,1) */
float  or_ran2_u01_f32(int32_t iy);       /* min(fl(AM*fl(iy)), RNMX)        */
double or_ran2_u01_f64(int32_t iy);       /* iy / m1                         */
void   or_box_muller_f32(float u1, float u2, float* g1, float* g2);
void   or_box_muller_f64(double u1, double u2, double* g1, double* g2);

/* ---- fills (out[d*S+s] = d-th draw of stream s; LFG: out[k] = x_{pos+k}) */
int or_fill_u32(or_gen* g, int64_t n, uint32_t* out);
int or_fill_uniform(or_gen* g, int64_t n, float* out);
int or_fill_normal(or_gen* g, int64_t n, float* out);   /* n even */

/* ---- Langevin dynamics ------------------------------------------------ */
typedef struct { double K, m, gamma, kT, dt; } or_params;
/* stats[0..4] = sum x^2, sum v^2, sum x.v, time-averaged total energy, steps */
int or_ld_init_eq_f32(or_gen* g, int64_t n, const float* Kper, or_params p,
                      float* x, float* v);
int or_ld_run_f32(or_gen* g, int64_t n, const float* Kper, or_params p,
                  float* x, float* v, int64_t n_steps, double* stats);
int or_ld_init_eq_f64(or_gen* g, int64_t n, const double* Kper, or_params p,
                      double* x, double* v);
int or_ld_run_f64(or_gen* g, int64_t n, const double* Kper, or_params p,
                  double* x, double* v, int64_t n_steps, double* stats,
                  double* loss_per_osc);
/* Reverse-time adjoint of L = (1/S) sum_{t=1..S} sum_i E_i(t) (FP64).
 * Per-thread generators only.  x, v enter as the initial state and leave as
 * the state after S steps; dK[n] receives dL/dK_i, *dgamma, *dkT the global
 * gradients, loss_per_osc[n] (nullable) the per-oscillator loss terms. */
int or_ld_adjoint_f64(or_gen* g, int64_t n, const double* Kper, or_params p,
                      double* x, double* v, int64_t n_steps,
                      double* loss_per_osc, double* dK, double* dgamma,
                      double* dkT);

/* ---- overdamped 1-D Langevin (Eq. 4-5) ---------------------------------- */
typedef struct { double k_sp, xi, kT, dt; } or_ou_params;
/* R' = fma(cs, g, fma(-c1, R, R)) with c1 = fl(k_sp dt / xi) and
 * cs = fl(sqrt(2 kT dt / xi)) (double expressions rounded once), g the cosine
 * branch of Box-Muller on two draws per particle-step (shared sequence:
 * particle i at step t uses positions p0 + 2(i + n t) + r).  Records
 * r = 0 .. n_steps/every after r*every steps: mean[r] = (1/n) sum_i R_i and
 * corr[r] = (1/n) sum_i R_i R_i(0), R(0) the positions on entry. */
int or_ou_run_f32(or_gen* g, int64_t n, or_ou_params p, float* R, int64_t n_steps,
                  int64_t every, double* mean, double* corr);

/* ---- pins ------------------------------------------------------------- */
uint64_t or_taus_component_period(int which, uint32_t seed);
uint64_t or_lcg_period(uint32_t seed);
int      or_gf2_trinomial_irreducible(int32_t ll, int32_t k);

#ifdef __cplusplus
}
#endif
#endif
