/*
 * gbrng_oracle.c -- plain serial CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline/reference
 * legs load this file's library.  It is compiled with -ffp-contract=off so that
 * every float expression rounds exactly where it is written; explicit fmaf()
 * calls are the only fused operations.
 *
 * Readings of the paper taken here (the paper is silent, garbled or at odds
 * with itself at these points):
 *  R1  Taus shift constants (Appendix A) come in per-component triples
 *      (13,19,12), (2,25,4), (3,11,17) with masks 4294967294, 4294967288,
 *      4294967280; the state advances before the output (Algorithm 1).
 *  R2  Taus seeds need y1>=2, y2>=8, y3>=16 (else that word is raised by
 *      2, 8, 16); the LCG word y4 is unconstrained.
 *  R3  Seeding (Sec. III.B only asks for an independent sequence): word k of
 *      stream s is the low 32 bits of SplitMix64 (Steele, Lea & Flood 2014)
 *      evaluated at counter 8*s+k; Lagged Fibonacci ring word w uses counter w,
 *      and word 0 is forced odd.
 *  R4  Ran2 constants are not printed (the paper defers to Numerical Recipes):
 *      L'Ecuyer's 1988 pair m1=2147483563, a1=40014, m2=2147483399, a2=40692,
 *      Schrage q=m div a, r=m mod a, NTAB=32 (35-word state), NDIV=1+(m1-1)/32,
 *      AM=fl32(1/m1), RNMX = largest float below 1.
 *  R5  Ran2's iy is never initialised in Algorithm 2; it starts as iv[0].
 *  R6  Lagged Fibonacci: Algorithm 3's indices give
 *      x_p = x_{p-ll} + x_{p-(ll-sl)} mod 2^32 (Eq. 3 writes x_{n-sl}; the two
 *      trinomials are reciprocal, so both are primitive).  Ring slot p mod ll.
 *  R7  Lag row: the smallest Table I row with sl > 4N and ll-sl > 4N, else the
 *      last row (no row covers N > 252551 with 4 numbers per thread).
 *  R11 Table I row 4 prints sl = 12470 with ll = 23209, but x^23209 + x^12470 + 1
 *      is reducible over GF(2) (so not primitive, against Sec. II.D); the row is
 *      read as sl = 13470, one digit away, whose trinomial is irreducible (its
 *      reciprocal is x^23209 + x^9739 + 1).
 *  R8  Box-Muller input: Taus/LFG words use the open map
 *      u = ((raw>>9)+1/2) 2^-23 (exact in binary32, never 0 or 1); Ran2 uses its
 *      own uniform.  Four uniforms give three normals per particle-step:
 *      (g_x, g_y) from (u1, u2), g_z = rho(u3) cos(2 pi u4).
 *  R9  Langevin step: underdamped first-order Euler-Maruyama of
 *      m dV/dt = -gamma V - K R + G with G = g sqrt(2 gamma kT dt) (Sec. I; the
 *      sign of the friction term is a typo there).  Both updates use the old
 *      (x, v):  v' = (1 - gamma dt/m) v - (dt K/m) x + (sigma/m) g,
 *               x' = x + dt v.
 *  R10 ld_init_equilibrium spends two draw-steps: step 0 gives
 *      x = sqrt(kT/K) g, step 1 gives v = sqrt(kT/m) g.
 *  R12 LCG (Eq. 1, m = 2^32, the "Quick and Dirty" form): x_n = a x_{n-1} + c
 *      with a = 1664525, c = 1013904223; the output is the new word.  Stream s
 *      starts from the low 32 bits of SplitMix64 at counter 8*s (R3).
 *  R13 Overdamped step (Eq. 5): the printed random term g sqrt(2 kT xi dt) is
 *      the random force times dt; divided by xi (Eq. 4) the displacement is
 *      g sqrt(2 kT dt / xi) = g sqrt(2 D dt), D = kT/xi.  One normal per
 *      particle-step: the cosine branch of Box-Muller on two draws (as the
 *      third normal of R8).
 *
 * FP32 arithmetic order of the Langevin step (both sides implement exactly
 * this; only the transcendental functions of Box-Muller may differ in the last
 * bits):  per system  cdt=fl(dt), cva=fl(1-(gamma*dt)/m), ckm=fl(dt/m),
 * cs=fl(sqrt(2*gamma*kT*dt)/m)  (double expressions, rounded once);
 * per oscillator  ckx = ckm*K_i (binary32 multiply);  per component
 * n = cs*g;  t = fma(-ckx, x, n);  v' = fma(cva, v, t);  x' = fma(cdt, v, x).
 */
#include "gbrng_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------
 * Seeding (reading R3)
 * ---------------------------------------------------------------------- */

/* SplitMix64 output function at counter idx: z = seed + (idx+1)*golden, then
 * the two xor-shift-multiply rounds of Steele, Lea & Flood (OOPSLA 2014). */
uint64_t or_splitmix64(uint64_t seed, uint64_t idx)
{
    uint64_t z = seed + (idx + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void or_taus_seed(uint64_t seed, int64_t n, uint32_t* st)
{
    static const uint32_t lowest[3] = {2u, 8u, 16u};     /* reading R2 */
    for (int64_t s = 0; s < n; ++s) {
        for (int k = 0; k < 4; ++k) {
            uint32_t w = (uint32_t)or_splitmix64(seed, 8u * (uint64_t)s + (uint64_t)k);
            if (k < 3 && w < lowest[k]) w += lowest[k];
            st[4 * s + k] = w;
        }
    }
}

/* Ran2 parameters (reading R4). */
#define R2_M1 2147483563
#define R2_A1 40014
#define R2_M2 2147483399
#define R2_A2 40692
#define R2_NTAB 32
#define R2_IMM1 (R2_M1 - 1)
#define R2_NDIV (1 + R2_IMM1 / R2_NTAB)

/* Schrage's factorisation a*x mod m = a*(x mod q) - r*(x div q) (+m if < 0)
 * for 0 < x < m; q = m div a and r = m mod a are derived here, not tabulated.
 * which = 0: (a1, m1); which = 1: (a2, m2).  Schrage step of Algorithm 2. */
int32_t or_ran2_schrage(int32_t x, int which)
{
    const int32_t m = which ? R2_M2 : R2_M1;
    const int32_t a = which ? R2_A2 : R2_A1;
    const int32_t q = m / a, r = m % a;
    int32_t k = x / q;
    int32_t y = a * (x - k * q) - k * r;
    if (y < 0) y += m;
    return y;
}

/* Seeding part of Algorithm 2 for one stream, plus reading R5 (iy = iv[0]). */
static void ran2_init_one(int32_t idum, int32_t* st)
{
    int32_t* iv = st + 3;
    st[1] = idum;                                   /* idum2 <- idum */
    for (int j = R2_NTAB + 7; j >= 0; --j) {
        idum = or_ran2_schrage(idum, 0);
        if (j < R2_NTAB) iv[j] = idum;
    }
    st[0] = idum;
    st[2] = iv[0];
}

void or_ran2_seed(uint64_t seed, int64_t n, int32_t* st)
{
    for (int64_t s = 0; s < n; ++s) {
        uint64_t w = or_splitmix64(seed, 8u * (uint64_t)s);
        int32_t idum = 1 + (int32_t)(w % (uint64_t)R2_IMM1);   /* in [1, m1-1] */
        ran2_init_one(idum, st + 35 * s);
    }
}

/* Seed the streams with the given indices (rows of st in that order), as
 * or_taus_seed / or_ran2_seed would for those indices. */
void or_seed_streams(int kind, uint64_t seed, const int64_t* idx, int64_t n, void* st)
{
    for (int64_t j = 0; j < n; ++j) {
        const uint64_t s = (uint64_t)idx[j];
        if (kind == OR_TAUS) {
            static const uint32_t lowest[3] = {2u, 8u, 16u};
            uint32_t* y = (uint32_t*)st + 4 * j;
            for (int k = 0; k < 4; ++k) {
                uint32_t w = (uint32_t)or_splitmix64(seed, 8u * s + (uint64_t)k);
                if (k < 3 && w < lowest[k]) w += lowest[k];
                y[k] = w;
            }
        } else if (kind == OR_LCG) {
            ((uint32_t*)st)[j] = (uint32_t)or_splitmix64(seed, 8u * s);
        } else {
            uint64_t w = or_splitmix64(seed, 8u * s);
            ran2_init_one(1 + (int32_t)(w % (uint64_t)R2_IMM1), (int32_t*)st + 35 * j);
        }
    }
}

void or_lcg_seed(uint64_t seed, int64_t n, uint32_t* st)
{
    for (int64_t s = 0; s < n; ++s) st[s] = (uint32_t)or_splitmix64(seed, 8u * (uint64_t)s);
}

void or_lfg_seed(uint64_t seed, int32_t ll, uint32_t* ring)
{
    for (int32_t w = 0; w < ll; ++w) ring[w] = (uint32_t)or_splitmix64(seed, (uint64_t)w);
    ring[0] |= 1u;                                  /* one odd seed (R3) */
}

/* Table I: (sl, ll) pairs, rows 0..9 (row 4 per reading R11). */
static const int32_t kTableI[10][2] = {
    {1252, 2281},     {3004, 4423},     {5502, 9689},     {10095, 19937},
    {13470, 23209},   {23463, 44497},   {54454, 132049},  {279695, 756839},
    {288477, 859433}, {1010202, 3021377}};

int or_lfg_table(int row, int32_t* sl, int32_t* ll)
{
    if (row < 0 || row > 9) return -1;
    *sl = kTableI[row][0];
    *ll = kTableI[row][1];
    return 0;
}

/* Reading R7. */
int or_lfg_default_row(int64_t n_threads)
{
    for (int r = 0; r < 10; ++r) {
        int64_t sl = kTableI[r][0], ll = kTableI[r][1];
        if (sl > 4 * n_threads && ll - sl > 4 * n_threads) return r;
    }
    return 9;
}

/* ------------------------------------------------------------------------
 * Generators
 * ---------------------------------------------------------------------- */

/* One Tausworthe word step of Algorithm 1 with the triples of R1. */
uint32_t or_taus_component(uint32_t y, int which)
{
    static const int s1[3] = {13, 2, 3}, s2[3] = {19, 25, 11}, s3[3] = {12, 4, 17};
    static const uint32_t c[3] = {4294967294u, 4294967288u, 4294967280u};
    uint32_t b = ((y << s1[which]) ^ y) >> s2[which];
    return ((y & c[which]) << s3[which]) ^ b;
}

/* Algorithm 1: advance the three Tausworthe words and the LCG
 * (a=1664525, c=1013904223), output the xor of the four new words. */
uint32_t or_taus_next(uint32_t* y)
{
    y[0] = or_taus_component(y[0], 0);
    y[1] = or_taus_component(y[1], 1);
    y[2] = or_taus_component(y[2], 2);
    y[3] = 1664525u * y[3] + 1013904223u;
    return y[0] ^ y[1] ^ y[2] ^ y[3];
}

/* Draw of Algorithm 2: returns the integer iy in [1, m1-1]. */
int32_t or_ran2_next(int32_t* st)
{
    int32_t* iv = st + 3;
    st[0] = or_ran2_schrage(st[0], 0);                 /* idum  */
    st[1] = or_ran2_schrage(st[1], 1);                 /* idum2 */
    int32_t j = st[2] / R2_NDIV;                       /* uses the previous iy */
    int32_t iy = iv[j] - st[1];
    iv[j] = st[0];
    if (iy < 1) iy += R2_IMM1;
    st[2] = iy;
    return iy;
}

/* Eq. 1 with m = 2^32 (reading R12): the multiply and add wrap modulo 2^32. */
uint32_t or_lcg_next(uint32_t* x)
{
    *x = 1664525u * *x + 1013904223u;
    return *x;
}

/* Recurrence of Algorithm 3 for the next position p = pos. */
uint32_t or_lfg_next(or_gen* g)
{
    uint32_t* x = (uint32_t*)g->state;
    const int64_t ll = g->ll, sl = g->sl;
    int64_t slot = g->pos % ll;                 /* holds x_{p-ll}        */
    int64_t slot_s = (slot + sl) % ll;          /* (p + sl - ll) mod ll  */
    uint32_t v = x[slot] + x[slot_s];           /* mod 2^32              */
    x[slot] = v;
    g->pos += 1;
    return v;
}

/* ------------------------------------------------------------------------
 * Conversions
 * ---------------------------------------------------------------------- */

float or_u01_f32(uint32_t raw)
{
    return (float)raw * 0x1p-32f;        /* mult of Algorithm 1 */
}

double or_open01(uint32_t raw)
{
    return ((double)(raw >> 9) + 0.5) * 0x1p-23;
}

float or_ran2_u01_f32(int32_t iy)
{
    const float am = (float)(1.0 / (double)R2_M1);
    const float rnmx = 0x1.fffffep-1f;           /* largest float below 1 */
    float t = am * (float)iy;
    return t > rnmx ? rnmx : t;
}

double or_ran2_u01_f64(int32_t iy)
{
    return (double)iy / (double)R2_M1;
}

/* Box-Muller: g1 = sqrt(-2 ln u1) cos(2 pi u2), g2 = sqrt(-2 ln u1) sin(2 pi u2).
 * The binary32 variant evaluates rho, cos and sin in double and rounds each
 * once, then multiplies in binary32. */
void or_box_muller_f32(float u1, float u2, float* g1, float* g2)
{
    const double two_pi = 6.283185307179586476925286766559;
    float rho = (float)sqrt(-2.0 * log((double)u1));
    double th = two_pi * (double)u2;
    float c = (float)cos(th), s = (float)sin(th);
    *g1 = rho * c;
    *g2 = rho * s;
}

void or_box_muller_f64(double u1, double u2, double* g1, double* g2)
{
    const double two_pi = 6.283185307179586476925286766559;
    double rho = sqrt(-2.0 * log(u1));
    double th = two_pi * u2;
    *g1 = rho * cos(th);
    *g2 = rho * sin(th);
}

/* ------------------------------------------------------------------------
 * Draw helpers: stream j of a per-thread generator, or the shared sequence.
 * ---------------------------------------------------------------------- */

static uint32_t draw_u32(or_gen* g, int64_t j)
{
    if (g->kind == OR_TAUS) return or_taus_next((uint32_t*)g->state + 4 * j);
    if (g->kind == OR_RAN2) return (uint32_t)or_ran2_next((int32_t*)g->state + 35 * j);
    if (g->kind == OR_LCG) return or_lcg_next((uint32_t*)g->state + j);
    return or_lfg_next(g);
}

static float draw_uniform_f32(or_gen* g, int64_t j)
{
    if (g->kind == OR_RAN2) return or_ran2_u01_f32(or_ran2_next((int32_t*)g->state + 35 * j));
    return or_u01_f32(draw_u32(g, j));
}

/* Box-Muller input uniform (reading R8). */
static float draw_bm_f32(or_gen* g, int64_t j)
{
    if (g->kind == OR_RAN2) return or_ran2_u01_f32(or_ran2_next((int32_t*)g->state + 35 * j));
    return (float)or_open01(draw_u32(g, j));
}

static double draw_bm_f64(or_gen* g, int64_t j)
{
    if (g->kind == OR_RAN2) return or_ran2_u01_f64(or_ran2_next((int32_t*)g->state + 35 * j));
    return or_open01(draw_u32(g, j));
}

/* Three normals of one particle-step (reading R8). */
static void normals3_f32(or_gen* g, int64_t j, float* out)
{
    float u1 = draw_bm_f32(g, j), u2 = draw_bm_f32(g, j);
    float u3 = draw_bm_f32(g, j), u4 = draw_bm_f32(g, j);
    float spare;
    or_box_muller_f32(u1, u2, &out[0], &out[1]);
    or_box_muller_f32(u3, u4, &out[2], &spare);
}

static void normals3_f64(or_gen* g, int64_t j, double* out)
{
    double u1 = draw_bm_f64(g, j), u2 = draw_bm_f64(g, j);
    double u3 = draw_bm_f64(g, j), u4 = draw_bm_f64(g, j);
    double spare;
    or_box_muller_f64(u1, u2, &out[0], &out[1]);
    or_box_muller_f64(u3, u4, &out[2], &spare);
}

/* ------------------------------------------------------------------------
 * Fills
 * ---------------------------------------------------------------------- */

int or_fill_u32(or_gen* g, int64_t n, uint32_t* out)
{
    if (n < 0) return -1;
    if (g->kind == OR_LAGFIB) {
        for (int64_t k = 0; k < n; ++k) out[k] = or_lfg_next(g);
        return 0;
    }
    const int64_t S = g->n_streams;
    for (int64_t base = 0; base < n; base += S)
        for (int64_t s = 0; s < S && base + s < n; ++s) out[base + s] = draw_u32(g, s);
    return 0;
}

int or_fill_uniform(or_gen* g, int64_t n, float* out)
{
    if (n < 0) return -1;
    if (g->kind == OR_LAGFIB) {
        for (int64_t k = 0; k < n; ++k) out[k] = or_u01_f32(or_lfg_next(g));
        return 0;
    }
    const int64_t S = g->n_streams;
    for (int64_t base = 0; base < n; base += S)
        for (int64_t s = 0; s < S && base + s < n; ++s) out[base + s] = draw_uniform_f32(g, s);
    return 0;
}

/* Pair e (out[2e], out[2e+1]) comes from two consecutive draws of one stream;
 * pair e = d*S + s belongs to stream s (LFG: pair e uses x_{pos+2e}, x_{pos+2e+1}). */
int or_fill_normal(or_gen* g, int64_t n, float* out)
{
    if (n < 0 || (n & 1)) return -1;
    const int64_t pairs = n / 2;
    const int64_t S = g->kind == OR_LAGFIB ? 1 : g->n_streams;
    for (int64_t base = 0; base < pairs; base += S)
        for (int64_t s = 0; s < S && base + s < pairs; ++s) {
            float u1 = draw_bm_f32(g, s), u2 = draw_bm_f32(g, s);
            or_box_muller_f32(u1, u2, &out[2 * (base + s)], &out[2 * (base + s) + 1]);
        }
    return 0;
}

/* ------------------------------------------------------------------------
 * Langevin dynamics
 * ---------------------------------------------------------------------- */

typedef struct { float cdt, cva, ckm, cs, sv, kT; } coef32;

static coef32 make_coef32(or_params p)
{
    coef32 c;
    c.cdt = (float)p.dt;
    c.cva = (float)(1.0 - (p.gamma * p.dt) / p.m);
    c.ckm = (float)(p.dt / p.m);
    c.cs = (float)(sqrt(2.0 * p.gamma * p.kT * p.dt) / p.m);
    c.sv = (float)sqrt(p.kT / p.m);
    c.kT = (float)p.kT;
    return c;
}

static int params_ok(or_params p)
{
    return p.m > 0 && p.gamma >= 0 && p.kT >= 0 && p.dt > 0 && p.K > 0;
}

/* Energy of one oscillator: (1/2) m |v|^2 + (1/2) K |x|^2, in double. */
static double energy_d(double K, double m, const double* x, const double* v)
{
    double x2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    return 0.5 * m * v2 + 0.5 * K * x2;
}

static void step_f32(const coef32* c, float ckx, const float* g, float* x, float* v)
{
    for (int k = 0; k < 3; ++k) {
        float nk = c->cs * g[k];
        float t = fmaf(-ckx, x[k], nk);
        float vn = fmaf(c->cva, v[k], t);
        x[k] = fmaf(c->cdt, v[k], x[k]);
        v[k] = vn;
    }
}

int or_ld_init_eq_f32(or_gen* g, int64_t n, const float* Kper, or_params p, float* x, float* v)
{
    if (n < 0 || !params_ok(p)) return -1;
    coef32 c = make_coef32(p);
    float gs[3];
    /* draw-step 0: positions; draw-step 1: velocities (reading R10).  The
     * shared sequence must be consumed step-major; per-thread streams are
     * independent, so the same loop serves both. */
    for (int64_t i = 0; i < n; ++i) {
        float Ki = Kper ? Kper[i] : (float)p.K;
        float sx = sqrtf(c.kT / Ki);
        normals3_f32(g, i, gs);
        for (int k = 0; k < 3; ++k) x[3 * i + k] = sx * gs[k];
    }
    for (int64_t i = 0; i < n; ++i) {
        normals3_f32(g, i, gs);
        for (int k = 0; k < 3; ++k) v[3 * i + k] = c.sv * gs[k];
    }
    return 0;
}

static void stats_snapshot_f32(int64_t n, const float* x, const float* v, double* stats)
{
    double sx = 0, sv = 0, sxv = 0;
    for (int64_t i = 0; i < 3 * n; ++i) {
        sx += (double)x[i] * (double)x[i];
        sv += (double)v[i] * (double)v[i];
        sxv += (double)x[i] * (double)v[i];
    }
    stats[0] = sx;
    stats[1] = sv;
    stats[2] = sxv;
}

int or_ld_run_f32(or_gen* g, int64_t n, const float* Kper, or_params p, float* x, float* v,
                  int64_t n_steps, double* stats)
{
    if (n < 0 || n_steps < 0 || !params_ok(p)) return -1;
    coef32 c = make_coef32(p);
    double esum = 0.0;
    float gs[3];
    if (g->kind == OR_LAGFIB) {
        /* Shared sequence: oscillator j at step t uses positions 4(j+Nt)+r. */
        for (int64_t t = 0; t < n_steps; ++t) {
            for (int64_t i = 0; i < n; ++i) {
                float Ki = Kper ? Kper[i] : (float)p.K;
                normals3_f32(g, i, gs);
                step_f32(&c, c.ckm * Ki, gs, x + 3 * i, v + 3 * i);
                double xd[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
                double vd[3] = {v[3 * i], v[3 * i + 1], v[3 * i + 2]};
                esum += energy_d((double)Ki, p.m, xd, vd);
            }
        }
    } else {
        /* Independent streams: oscillator-major order gives the same values. */
        for (int64_t i = 0; i < n; ++i) {
            float Ki = Kper ? Kper[i] : (float)p.K;
            float ckx = c.ckm * Ki;
            for (int64_t t = 0; t < n_steps; ++t) {
                normals3_f32(g, i, gs);
                step_f32(&c, ckx, gs, x + 3 * i, v + 3 * i);
                double xd[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
                double vd[3] = {v[3 * i], v[3 * i + 1], v[3 * i + 2]};
                esum += energy_d((double)Ki, p.m, xd, vd);
            }
        }
    }
    if (stats) {
        stats_snapshot_f32(n, x, v, stats);
        stats[3] = n_steps > 0 ? esum / (double)n_steps : 0.0;
        stats[4] = (double)n_steps;
    }
    return 0;
}

/* ---- FP64 variant: identical integer streams, double arithmetic ------- */

typedef struct { double a, b_over_K, c, dt, sv; } coef64;

static coef64 make_coef64(or_params p)
{
    coef64 c;
    c.a = 1.0 - p.gamma * p.dt / p.m;
    c.b_over_K = p.dt / p.m;
    c.c = sqrt(2.0 * p.gamma * p.kT * p.dt) / p.m;
    c.dt = p.dt;
    c.sv = sqrt(p.kT / p.m);
    return c;
}

static void step_f64(const coef64* c, double b, const double* g, double* x, double* v)
{
    for (int k = 0; k < 3; ++k) {
        double vn = c->a * v[k] - b * x[k] + c->c * g[k];
        x[k] = x[k] + c->dt * v[k];
        v[k] = vn;
    }
}

int or_ld_init_eq_f64(or_gen* g, int64_t n, const double* Kper, or_params p, double* x, double* v)
{
    if (n < 0 || !params_ok(p)) return -1;
    coef64 c = make_coef64(p);
    double gs[3];
    for (int64_t i = 0; i < n; ++i) {
        double Ki = Kper ? Kper[i] : p.K;
        double sx = sqrt(p.kT / Ki);
        normals3_f64(g, i, gs);
        for (int k = 0; k < 3; ++k) x[3 * i + k] = sx * gs[k];
    }
    for (int64_t i = 0; i < n; ++i) {
        normals3_f64(g, i, gs);
        for (int k = 0; k < 3; ++k) v[3 * i + k] = c.sv * gs[k];
    }
    return 0;
}

int or_ld_run_f64(or_gen* g, int64_t n, const double* Kper, or_params p, double* x, double* v,
                  int64_t n_steps, double* stats, double* loss_per_osc)
{
    if (n < 0 || n_steps < 0 || !params_ok(p)) return -1;
    coef64 c = make_coef64(p);
    double esum = 0.0;
    double gs[3];
    if (loss_per_osc)
        for (int64_t i = 0; i < n; ++i) loss_per_osc[i] = 0.0;
    if (g->kind == OR_LAGFIB) {
        for (int64_t t = 0; t < n_steps; ++t)
            for (int64_t i = 0; i < n; ++i) {
                double Ki = Kper ? Kper[i] : p.K;
                normals3_f64(g, i, gs);
                step_f64(&c, c.b_over_K * Ki, gs, x + 3 * i, v + 3 * i);
                double e = energy_d(Ki, p.m, x + 3 * i, v + 3 * i);
                esum += e;
                if (loss_per_osc) loss_per_osc[i] += e;
            }
    } else {
        for (int64_t i = 0; i < n; ++i) {
            double Ki = Kper ? Kper[i] : p.K;
            for (int64_t t = 0; t < n_steps; ++t) {
                normals3_f64(g, i, gs);
                step_f64(&c, c.b_over_K * Ki, gs, x + 3 * i, v + 3 * i);
                double e = energy_d(Ki, p.m, x + 3 * i, v + 3 * i);
                esum += e;
                if (loss_per_osc) loss_per_osc[i] += e;
            }
        }
    }
    if (loss_per_osc && n_steps > 0)
        for (int64_t i = 0; i < n; ++i) loss_per_osc[i] /= (double)n_steps;
    if (stats) {
        double sx = 0, sv = 0, sxv = 0;
        for (int64_t i = 0; i < 3 * n; ++i) {
            sx += x[i] * x[i];
            sv += v[i] * v[i];
            sxv += x[i] * v[i];
        }
        stats[0] = sx;
        stats[1] = sv;
        stats[2] = sxv;
        stats[3] = n_steps > 0 ? esum / (double)n_steps : 0.0;
        stats[4] = (double)n_steps;
    }
    return 0;
}

/* Reverse-time adjoint, FP64.  For each oscillator (independent streams):
 * forward pass storing (x_t, v_t, g_t), then the backward recursion
 *   lx_S = K x_S / S,  lv_S = m v_S / S,
 *   lx_t = lx_{t+1} - b lv_{t+1} + [t>=1] K x_t / S,
 *   lv_t = dt lx_{t+1} + a lv_{t+1} + [t>=1] m v_t / S,
 * with a = 1 - gamma dt/m, b = dt K/m, c = sqrt(2 gamma kT dt)/m, and the
 * parameter gradients
 *   dL/dK_i   = sum_{t=1..S} |x_t|^2 / (2S) - (dt/m) sum_{t<S} lv_{t+1}.x_t,
 *   dL/dgamma = sum_{t<S} lv_{t+1}.(-(dt/m) v_t + c/(2 gamma) g_t),
 *   dL/dkT    = sum_{t<S} lv_{t+1}.(c/(2 kT) g_t).                          */
int or_ld_adjoint_f64(or_gen* g, int64_t n, const double* Kper, or_params p, double* x,
                      double* v, int64_t n_steps, double* loss_per_osc, double* dK,
                      double* dgamma, double* dkT)
{
    if (g->kind == OR_LAGFIB || g->kind == OR_LCG || n < 0 || n_steps <= 0 || !params_ok(p) ||
        p.gamma <= 0 ||
        p.kT <= 0)
        return -1;
    const int64_t S = n_steps;
    coef64 c = make_coef64(p);
    double* xs = (double*)malloc(sizeof(double) * 3 * (S + 1));
    double* vs = (double*)malloc(sizeof(double) * 3 * (S + 1));
    double* gs = (double*)malloc(sizeof(double) * 3 * S);
    if (!xs || !vs || !gs) {
        free(xs); free(vs); free(gs);
        return -2;
    }
    double dg_tot = 0.0, dkT_tot = 0.0;
    const double invS = 1.0 / (double)S;
    for (int64_t i = 0; i < n; ++i) {
        const double Ki = Kper ? Kper[i] : p.K;
        const double b = c.b_over_K * Ki;
        for (int k = 0; k < 3; ++k) {
            xs[k] = x[3 * i + k];
            vs[k] = v[3 * i + k];
        }
        double loss = 0.0, dKi = 0.0;
        for (int64_t t = 0; t < S; ++t) {
            normals3_f64(g, i, gs + 3 * t);
            for (int k = 0; k < 3; ++k) {
                xs[3 * (t + 1) + k] = xs[3 * t + k];
                vs[3 * (t + 1) + k] = vs[3 * t + k];
            }
            step_f64(&c, b, gs + 3 * t, xs + 3 * (t + 1), vs + 3 * (t + 1));
            loss += energy_d(Ki, p.m, xs + 3 * (t + 1), vs + 3 * (t + 1));
            const double* xt = xs + 3 * (t + 1);
            dKi += 0.5 * invS * (xt[0] * xt[0] + xt[1] * xt[1] + xt[2] * xt[2]);
        }
        double lx[3], lv[3];
        for (int k = 0; k < 3; ++k) {
            lx[k] = Ki * xs[3 * S + k] * invS;
            lv[k] = p.m * vs[3 * S + k] * invS;
        }
        for (int64_t t = S - 1; t >= 0; --t) {
            const double* xt = xs + 3 * t;
            const double* vt = vs + 3 * t;
            const double* gt = gs + 3 * t;
            for (int k = 0; k < 3; ++k) {
                dKi += -(p.dt / p.m) * lv[k] * xt[k];
                dg_tot += lv[k] * (-(p.dt / p.m) * vt[k] + c.c / (2.0 * p.gamma) * gt[k]);
                dkT_tot += lv[k] * (c.c / (2.0 * p.kT) * gt[k]);
                double lxn = lx[k] - b * lv[k] + (t >= 1 ? Ki * xt[k] * invS : 0.0);
                double lvn = p.dt * lx[k] + c.a * lv[k] + (t >= 1 ? p.m * vt[k] * invS : 0.0);
                lx[k] = lxn;
                lv[k] = lvn;
            }
        }
        for (int k = 0; k < 3; ++k) {
            x[3 * i + k] = xs[3 * S + k];
            v[3 * i + k] = vs[3 * S + k];
        }
        if (loss_per_osc) loss_per_osc[i] = loss * invS;
        if (dK) dK[i] = dKi;
    }
    if (dgamma) *dgamma = dg_tot;
    if (dkT) *dkT = dkT_tot;
    free(xs); free(vs); free(gs);
    return 0;
}

/* ------------------------------------------------------------------------
 * Pins: brute-force periods and GF(2) irreducibility
 * ---------------------------------------------------------------------- */

/* ------------------------------------------------------------------------
 * Overdamped 1-D Langevin dynamics (Eq. 4-5, reading R13)
 * ---------------------------------------------------------------------- */

int or_ou_run_f32(or_gen* g, int64_t n, or_ou_params p, float* R, int64_t n_steps,
                  int64_t every, double* mean, double* corr)
{
    if (n < 1 || n_steps < 0 || every < 1 || !(p.k_sp > 0) || !(p.xi > 0) || !(p.kT >= 0) ||
        !(p.dt > 0))
        return -1;
    const float c1 = (float)(p.k_sp * p.dt / p.xi);
    const float cs = (float)sqrt(2.0 * p.kT * p.dt / p.xi);
    float* R0 = (float*)malloc(sizeof(float) * (size_t)n);
    if (!R0) return -1;
    memcpy(R0, R, sizeof(float) * (size_t)n);
    int64_t rec = 0;
    for (int64_t t = 0; t <= n_steps; ++t) {
        if (t % every == 0) {
            double sm = 0.0, sc = 0.0;
            for (int64_t i = 0; i < n; ++i) {
                sm += (double)R[i];
                sc += (double)R[i] * (double)R0[i];
            }
            mean[rec] = sm / (double)n;
            corr[rec] = sc / (double)n;
            ++rec;
        }
        if (t == n_steps) break;
        /* step-major, so the shared sequence is consumed in position order */
        for (int64_t i = 0; i < n; ++i) {
            float u1 = draw_bm_f32(g, i), u2 = draw_bm_f32(g, i);
            float gc, gs;
            or_box_muller_f32(u1, u2, &gc, &gs);
            R[i] = fmaf(cs, gc, fmaf(-c1, R[i], R[i]));
        }
    }
    free(R0);
    return 0;
}

uint64_t or_taus_component_period(int which, uint32_t seed)
{
    uint32_t first = or_taus_component(seed, which);   /* state after one step */
    uint32_t y = first;
    uint64_t count = 0;
    do {
        y = or_taus_component(y, which);
        ++count;
    } while (y != first && count < (1ull << 33));
    return count;
}

uint64_t or_lcg_period(uint32_t seed)
{
    uint32_t y = seed;
    uint64_t count = 0;
    do {
        y = 1664525u * y + 1013904223u;
        ++count;
    } while (y != seed && count < (1ull << 33));
    return count;
}

/* Polynomials over GF(2) as little-endian arrays of 64-bit words. */

/* dst[0..nd) = (src >> sh), src has ns words. */
static void gf2_shr(uint64_t* dst, int64_t nd, const uint64_t* src, int64_t ns, int64_t sh)
{
    const int64_t ws = sh >> 6;
    const int bs = (int)(sh & 63);
    for (int64_t w = 0; w < nd; ++w) {
        int64_t i = w + ws;
        uint64_t lo = i < ns ? src[i] >> bs : 0;
        uint64_t hi = (bs && i + 1 < ns) ? src[i + 1] << (64 - bs) : 0;
        dst[w] = lo | hi;
    }
}

/* dst[0..nd) ^= (src << sh), src has ns words. */
static void gf2_xor_shl(uint64_t* dst, int64_t nd, const uint64_t* src, int64_t ns, int64_t sh)
{
    const int64_t ws = sh >> 6;
    const int bs = (int)(sh & 63);
    for (int64_t i = 0; i < ns; ++i) {
        int64_t w = i + ws;
        if (w >= nd) break;
        dst[w] ^= src[i] << bs;
        if (bs && w + 1 < nd) dst[w + 1] ^= src[i] >> (64 - bs);
    }
}

/* Is x^ll + x^k + 1 irreducible over GF(2)?  For prime ll (Table I lists
 * Mersenne exponents) it is iff x^(2^ll) = x mod P, since P(0) = P(1) = 1 rules
 * out linear factors.  The reciprocal trinomial x^ll + x^(ll-k) + 1 has the same
 * factorisation pattern, so the smaller exponent is used for the reduction. */
int or_gf2_trinomial_irreducible(int32_t ll, int32_t k)
{
    if (ll < 3 || k <= 0 || k >= ll) return -1;
    if (2 * k > ll) k = ll - k;
    const int64_t W = ((int64_t)ll + 63) / 64;       /* words of a reduced poly */
    const int64_t W2 = 2 * W + 1;
    uint64_t* r = (uint64_t*)calloc((size_t)W2, sizeof(uint64_t));
    uint64_t* h = (uint64_t*)calloc((size_t)W2, sizeof(uint64_t));
    uint32_t* spread = (uint32_t*)malloc(sizeof(uint32_t) * 65536);
    if (!r || !h || !spread) {
        free(r); free(h); free(spread);
        return -2;
    }
    for (uint32_t b = 0; b < 65536; ++b) {
        uint32_t s = 0;
        for (int j = 0; j < 16; ++j)
            if (b & (1u << j)) s |= 1u << (2 * j);
        spread[b] = s;
    }
    const uint64_t top_mask = (ll % 64) ? ((1ull << (ll % 64)) - 1) : ~0ull;
    r[0] = 2u;                                        /* x */
    for (int32_t it = 0; it < ll; ++it) {
        /* square in place, high words first */
        for (int64_t w = W - 1; w >= 0; --w) {
            uint64_t v = r[w];
            r[2 * w] = (uint64_t)spread[v & 0xFFFF] | ((uint64_t)spread[(v >> 16) & 0xFFFF] << 32);
            r[2 * w + 1] = (uint64_t)spread[(v >> 32) & 0xFFFF] |
                           ((uint64_t)spread[(v >> 48) & 0xFFFF] << 32);
        }
        r[2 * W] = 0;
        /* two reduction rounds: r = L + H x^ll = L + H + H x^k */
        for (int round = 0; round < 2; ++round) {
            gf2_shr(h, W, r, W2, ll);
            r[W - 1] &= top_mask;
            for (int64_t w = W; w < W2; ++w) r[w] = 0;
            for (int64_t w = 0; w < W; ++w) r[w] ^= h[w];
            gf2_xor_shl(r, W2, h, W, k);
        }
    }
    int ok = (r[0] == 2u);
    for (int64_t w = 1; w < W2 && ok; ++w)
        if (r[w]) ok = 0;
    free(r); free(h); free(spread);
    return ok;
}
