// Device-side building blocks: the three generators, conversions,
// Box-Muller, the Euler-Maruyama step and deterministic reductions.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "bm_coeffs.cuh"
#include "gbrng.h"

namespace gb {

// ------------------------------------------------------------------ seeding
// SplitMix64 (Steele, Lea & Flood 2014) evaluated at counter idx.
__host__ __device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t idx)
{
    uint64_t z = seed + (idx + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// ------------------------------------------------------------- Hybrid Taus
// One Tausworthe word step (Algorithm 1): b = ((y << S1) ^ y) >> S2,
// y = ((y & C) << S3) ^ b.
// With MUL the two left shifts are written as multiplies by 2^S (the same
// bits), which the FMA pipe's integer multiply-add can take off the ALU pipe;
// used where that measured faster (the two-oscillator fused kernel).
template <int S>
__device__ __forceinline__ uint32_t shl_mul(uint32_t y)
{
    uint32_t r;
    asm("mul.lo.u32 %0, %1, %2;" : "=r"(r) : "r"(y), "n"(1u << S));
    return r;
}

template <int S1, int S2, int S3, uint32_t C, bool MUL = false>
__device__ __forceinline__ uint32_t taus_word(uint32_t y)
{
    if (MUL) {
        const uint32_t b = (shl_mul<S1>(y) ^ y) >> S2;
        return (shl_mul<S3>(y) & (C << S3)) ^ b;
    }
    const uint32_t b = ((y << S1) ^ y) >> S2;
    return ((y & C) << S3) ^ b;
}

// Advance the three Tausworthe words and the LCG, return their xor.
template <bool MUL = false>
__device__ __forceinline__ uint32_t taus_next(uint4& s)
{
    s.x = taus_word<13, 19, 12, 0xFFFFFFFEu, MUL>(s.x);
    s.y = taus_word<2, 25, 4, 0xFFFFFFF8u, MUL>(s.y);
    s.z = taus_word<3, 11, 17, 0xFFFFFFF0u, MUL>(s.z);
    s.w = 1664525u * s.w + 1013904223u;
    return s.x ^ s.y ^ s.z ^ s.w;
}

// ------------------------------------------------------ Quick and Dirty LCG
// Eq. 1 with m = 2^32: the multiply and add wrap; the output is the new word.
__device__ __forceinline__ uint32_t lcg_next(uint32_t& x)
{
    x = 1664525u * x + 1013904223u;
    return x;
}

// The per-thread 32-bit generators behind one name for the fill kernels.
__device__ __forceinline__ uint32_t next_word(uint4& y) { return taus_next(y); }
__device__ __forceinline__ uint32_t next_word(uint32_t& x) { return lcg_next(x); }

// -------------------------------------------------------------------- Ran2
// L'Ecuyer's pair (m1, a1) = (2147483563, 40014), (m2, a2) = (2147483399,
// 40692) with Schrage's q = m div a, r = m mod a; 32-entry shuffle table.
constexpr int32_t kR2M1 = 2147483563, kR2A1 = 40014, kR2Q1 = 53668, kR2R1 = 12211;
constexpr int32_t kR2M2 = 2147483399, kR2A2 = 40692, kR2Q2 = 52774, kR2R2 = 3791;
constexpr int32_t kR2Imm1 = kR2M1 - 1;
constexpr int32_t kR2Ndiv = 1 + kR2Imm1 / 32;
static_assert(kR2Q1 == kR2M1 / kR2A1 && kR2R1 == kR2M1 % kR2A1, "Schrage constants");
static_assert(kR2Q2 == kR2M2 / kR2A2 && kR2R2 == kR2M2 % kR2A2, "Schrage constants");

// a*x mod m for 0 < x < m (Schrage step of Algorithm 2).  x is positive, so the
// quotient uses unsigned division by a constant (a multiply-high).
template <int32_t A, int32_t M, int32_t Q, int32_t R>
__host__ __device__ __forceinline__ int32_t schrage(int32_t x)
{
    const int32_t k = (int32_t)((uint32_t)x / (uint32_t)Q);
    int32_t y = A * (x - k * Q) - k * R;
    return y < 0 ? y + M : y;
}

// The same a*x mod m from the 64-bit product, for m = 2^31 - d: 2^31 = d
// (mod m), so p = hi 2^31 + lo = hi d + lo (mod m), and r = hi d + lo <
// 2^31 + 2^24 < 2m needs one conditional subtraction, taken as the unsigned
// minimum of r and r - m (for r < m the difference wraps above r).  Equal to
// schrage() for every 0 < x < m (checked exhaustively for both moduli); one
// wide multiply instead of Schrage's quotient and three multiplies.
template <int32_t A, int32_t M>
__host__ __device__ __forceinline__ int32_t mulmod_m31(int32_t x)
{
    constexpr uint32_t d = 2147483648u - (uint32_t)M;
    const uint64_t p = (uint64_t)(uint32_t)A * (uint32_t)x;
    const uint32_t r = (uint32_t)(p >> 31) * d + ((uint32_t)p & 0x7fffffffu);
    const uint32_t rm = r - (uint32_t)M;
    return (int32_t)(rm < r ? rm : r);
}

// One Ran2 draw; the shuffle table is addressed through `iv(j)` so that it can
// live in shared memory ([32][threads]) or global memory.
struct Ran2Regs {
    int32_t idum, idum2, iy;
};

template <class TableRef>
__device__ __forceinline__ int32_t ran2_next(Ran2Regs& r, TableRef iv)
{
    r.idum = mulmod_m31<kR2A1, kR2M1>(r.idum);
    r.idum2 = mulmod_m31<kR2A2, kR2M2>(r.idum2);
    const int j = (int)((uint32_t)r.iy / (uint32_t)kR2Ndiv);   // previous iy
    int32_t y = iv(j) - r.idum2;
    iv(j) = r.idum;
    if (y < 1) y += kR2Imm1;
    r.iy = y;
    return y;
}

// ------------------------------------------------------------- conversions
// Taus / Lagged Fibonacci uniform: fl(raw) * 2^-32 in [0, 1].
__device__ __forceinline__ float u01_from_u32(uint32_t raw)
{
    return __fmul_rn(__uint2float_rn(raw), 0x1p-32f);
}

// Ran2 uniform: min(fl(AM * fl(iy)), RNMX), AM = fl(1/m1), RNMX < 1.
__device__ __forceinline__ float u01_from_ran2(int32_t iy)
{
    const float am = 0x1p-31f;   // fl32(1/2147483563) rounds to 2^-31 exactly
    const float rnmx = 0x1.fffffep-1f;
    return fminf(__fmul_rn(am, __int2float_rn(iy)), rnmx);
}

// Open-interval Box-Muller input ((raw >> 9) + 1/2) * 2^-23, exact in
// binary32: the bits 0x3f800000 + (raw >> 9) are m = 1 + k 2^-23 (k = raw >> 9),
// and subtracting 1 - 2^-24 leaves k 2^-23 + 2^-24 with no rounding.
__device__ __forceinline__ float mant_from_u32(uint32_t raw)
{
    return __uint_as_float(0x3f800000u + (raw >> 9));
}

__device__ __forceinline__ float open01_from_u32(uint32_t raw)
{
    return __fsub_rn(mant_from_u32(raw), 0x1.fffffep-1f);
}

// 4u for the same u, in one fused step: 4m - (4 - 2^-22) = 4 k 2^-23 + 2^-22
// is exact (below 4 the spacing is at most 2^-22).
__device__ __forceinline__ float quarter_turns_from_u32(uint32_t raw)
{
    return __fmaf_rn(4.0f, mant_from_u32(raw), -0x1.fffffep+1f);
}

// ---------------------------------------------------------------- Box-Muller
// The transcendentals of the transform, reduced to the ranges the generators
// produce (u a positive normal binary32 below 1) with polynomial coefficients
// fitted by fit_bm_coeffs.py; all within 2 ulp on those ranges.

// R's coefficients in the variable g = -2f: c'_i = -c_i (-1)^i / 2^(i+1), exact
// power-of-two rescalings of kLogR.
__host__ __device__ constexpr float log_g_coef(int i)
{
    return -kLogR[i] * ((i & 1) ? -1.0f : 1.0f) / (float)(2 << i);
}
constexpr float kLogG[9] = {log_g_coef(0), log_g_coef(1), log_g_coef(2),
                            log_g_coef(3), log_g_coef(4), log_g_coef(5),
                            log_g_coef(6), log_g_coef(7), log_g_coef(8)};

// -2 ln(u): u = 2^e m with m in [2/3, 4/3) (exponent split at the bits of 2/3),
// f = m - 1 exact, ln m = f + f^2 R(f), ln u = e ln2 + ln m (ln2 in two parts).
// Evaluated in g = -2f (exact), where every Estrin term is the f-form term
// times an exact power of two, so the result equals -2 times the f-form ln u
// bit for bit without the final multiply.
__device__ __forceinline__ float neg2log(float u)
{
    const int bits = __float_as_int(u);
    const int e = (bits - 0x3f2aaaab) >> 23;
    const float g = __fmaf_rn(__int_as_float(bits - (e << 23)), -2.0f, 2.0f);
    const float g2 = __fmul_rn(g, g);
    const float g4 = __fmul_rn(g2, g2);
    const float p01 = __fmaf_rn(kLogG[1], g, kLogG[0]);
    const float p23 = __fmaf_rn(kLogG[3], g, kLogG[2]);
    const float p45 = __fmaf_rn(kLogG[5], g, kLogG[4]);
    const float p67 = __fmaf_rn(kLogG[7], g, kLogG[6]);
    const float p03 = __fmaf_rn(p23, g2, p01);
    const float p47 = __fmaf_rn(p67, g2, p45);
    const float p48 = __fmaf_rn(kLogG[8], g4, p47);
    const float R = __fmaf_rn(p48, g4, p03);
    const float l2m = __fmaf_rn(g2, R, g);
    const float ef = (float)e;
    return __fmaf_rn(ef, 0x1.05c610p-28f, __fmaf_rn(ef, -0x1.62e430p+0f, l2m));
}

// sqrt(y) for a positive normal y: the hardware approximation, within 1 ulp of
// the correctly rounded root on the whole range the transform produces
// ([2^-24, 64), checked exhaustively).
__device__ __forceinline__ float sqrt_pos(float y)
{
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(y));
    return r;
}

// sin and cos of (pi/2) x for x = 4u in (0, 4), with no integer work: n =
// rint(x / 2) in {0, 1, 2} (x / 2 added to 1.5 * 2^23, where the addition's
// round-to-nearest drops the fraction, and the constant taken off again),
// y = x - 2n in [-1, 1] (exact: either x itself or a difference within a
// factor of two), the sign (-1)^n = (2n - 4) n + 1 (exact for those n), and
// sin(pi x / 2) = (-1)^n sin(pi y / 2), cos(pi x / 2) = (-1)^n cos(pi y / 2).
// With z = y^2: cos(pi y / 2) = (1 - z)(1 + z Q1(z)), the factor 1 - z
// rounded once so that the zeros at y = +-1 keep their relative accuracy;
// sin(pi y / 2) = y c0 + y z P1(z), the head y c0 added in the last FMA.
struct HalfTurn {
    float sgn, y, z, f1;
};

__device__ __forceinline__ HalfTurn half_turn(float x)
{
    const float nf = __fsub_rn(__fmaf_rn(x, 0.5f, 0x1.8p+23f), 0x1.8p+23f);
    HalfTurn h;
    h.y = __fmaf_rn(nf, -2.0f, x);
    h.sgn = __fmaf_rn(__fmaf_rn(nf, 2.0f, -4.0f), nf, 1.0f);
    h.z = __fmul_rn(h.y, h.y);
    h.f1 = __fmaf_rn(-h.y, h.y, 1.0f);
    return h;
}

__device__ __forceinline__ float cos_half(const HalfTurn& h)
{
    const float z = h.z;
    const float q = __fmaf_rn(__fmaf_rn(__fmaf_rn(kCosQ1[3], z, kCosQ1[2]), z, kCosQ1[1]), z, kCosQ1[0]);
    return __fmaf_rn(__fmul_rn(h.f1, z), q, h.f1);
}

__device__ __forceinline__ float sin_half(const HalfTurn& h)
{
    const float z = h.z;
    const float p = __fmaf_rn(
        __fmaf_rn(__fmaf_rn(__fmaf_rn(kSinP1[4], z, kSinP1[3]), z, kSinP1[2]), z, kSinP1[1]), z,
        kSinP1[0]);
    return __fmaf_rn(h.y, kSinC0, __fmul_rn(__fmul_rn(h.y, z), p));
}

// Box-Muller from m = -2 ln u1 and x = 4 u2: the pair (rho cos, rho sin) and
// the cosine branch alone (third normal of a particle-step), rho = sqrt(m).
// The sign (-1)^n goes on rho (exact), so each result is one rounding of rho
// times the signed cos or sin.
__device__ __forceinline__ void box_muller_x(float m2log, float x, float& g1, float& g2)
{
    const HalfTurn h = half_turn(x);
    const float sr = __fmul_rn(h.sgn, sqrt_pos(m2log));
    g1 = __fmul_rn(sr, cos_half(h));
    g2 = __fmul_rn(sr, sin_half(h));
}

__device__ __forceinline__ float box_muller_cos_x(float m2log, float x)
{
    const HalfTurn h = half_turn(x);
    return __fmul_rn(__fmul_rn(h.sgn, sqrt_pos(m2log)), cos_half(h));
}

// From two uniforms in (0, 1) (Ran2; 4u is exact).
__device__ __forceinline__ void box_muller(float u1, float u2, float& g1, float& g2)
{
    box_muller_x(neg2log(u1), __fmul_rn(4.0f, u2), g1, g2);
}

__device__ __forceinline__ float box_muller_cos(float u1, float u2)
{
    return box_muller_cos_x(neg2log(u1), __fmul_rn(4.0f, u2));
}

// From raw 32-bit draws (u = open01_from_u32), with 4u formed directly from
// the draw (Hybrid Taus, the LCG, Lagged Fibonacci).
__device__ __forceinline__ void box_muller_u32(uint32_t r1, uint32_t r2, float& g1, float& g2)
{
    box_muller_x(neg2log(open01_from_u32(r1)), quarter_turns_from_u32(r2), g1, g2);
}

__device__ __forceinline__ float box_muller_cos_u32(uint32_t r1, uint32_t r2)
{
    return box_muller_cos_x(neg2log(open01_from_u32(r1)), quarter_turns_from_u32(r2));
}

// ------------------------------------------- paired Box-Muller (f32x2 lanes)
// Two transforms side by side in the two lanes of the paired binary32
// instructions (FFMA2 / FMUL2 / FADD2: one instruction, two independent
// correctly rounded operations), halving the floating-point instructions.
// Each lane performs exactly the operations of the scalar functions above, in
// the same order, so the normals are the same bit for bit; only the integer
// exponent split and sqrt stay per lane.  The lanes hold either a
// particle-step's two transforms (the pair from draws 1, 2 and the cosine
// branch from draws 3, 4) or the same transform of two oscillators.
__device__ __forceinline__ float2 splat2(float a) { return make_float2(a, a); }

// -2 ln u in both lanes (neg2log, lane by lane).  u must not come straight
// from a paired instruction: reading such a lane's bit pattern for the
// exponent split measured wrong in the first lane, so callers form u lane by
// lane.
__device__ __forceinline__ float2 neg2log2(float2 u)
{
    const int bx = __float_as_int(u.x), by = __float_as_int(u.y);
    const int ex = (bx - 0x3f2aaaab) >> 23, ey = (by - 0x3f2aaaab) >> 23;
    const float2 m = make_float2(__int_as_float(bx - (ex << 23)), __int_as_float(by - (ey << 23)));
    const float2 g = __ffma2_rn(m, splat2(-2.0f), splat2(2.0f));
    const float2 g2 = __fmul2_rn(g, g);
    const float2 g4 = __fmul2_rn(g2, g2);
    const float2 p01 = __ffma2_rn(splat2(kLogG[1]), g, splat2(kLogG[0]));
    const float2 p23 = __ffma2_rn(splat2(kLogG[3]), g, splat2(kLogG[2]));
    const float2 p45 = __ffma2_rn(splat2(kLogG[5]), g, splat2(kLogG[4]));
    const float2 p67 = __ffma2_rn(splat2(kLogG[7]), g, splat2(kLogG[6]));
    const float2 p03 = __ffma2_rn(p23, g2, p01);
    const float2 p47 = __ffma2_rn(p67, g2, p45);
    const float2 p48 = __ffma2_rn(splat2(kLogG[8]), g4, p47);
    const float2 R = __ffma2_rn(p48, g4, p03);
    const float2 l2m = __ffma2_rn(g2, R, g);
    const float2 ef = make_float2((float)ex, (float)ey);
    return __ffma2_rn(ef, splat2(0x1.05c610p-28f), __ffma2_rn(ef, splat2(-0x1.62e430p+0f), l2m));
}

// half_turn, cos_half and sin_half in both lanes.
struct HalfTurn2 {
    float2 sgn, y, z, f1;
};

__device__ __forceinline__ HalfTurn2 half_turn2(float2 x)
{
    const float2 nf = __fadd2_rn(__ffma2_rn(x, splat2(0.5f), splat2(0x1.8p+23f)), splat2(-0x1.8p+23f));
    HalfTurn2 h;
    h.y = __ffma2_rn(nf, splat2(-2.0f), x);
    h.sgn = __ffma2_rn(__ffma2_rn(nf, splat2(2.0f), splat2(-4.0f)), nf, splat2(1.0f));
    h.z = __fmul2_rn(h.y, h.y);
    h.f1 = __ffma2_rn(make_float2(-h.y.x, -h.y.y), h.y, splat2(1.0f));
    return h;
}

__device__ __forceinline__ float2 cos_half2(const HalfTurn2& h)
{
    const float2 z = h.z;
    const float2 q = __ffma2_rn(
        __ffma2_rn(__ffma2_rn(splat2(kCosQ1[3]), z, splat2(kCosQ1[2])), z, splat2(kCosQ1[1])), z,
        splat2(kCosQ1[0]));
    return __ffma2_rn(__fmul2_rn(h.f1, z), q, h.f1);
}

__device__ __forceinline__ float2 sin_half2(const HalfTurn2& h)
{
    const float2 z = h.z;
    const float2 p = __ffma2_rn(
        __ffma2_rn(__ffma2_rn(__ffma2_rn(splat2(kSinP1[4]), z, splat2(kSinP1[3])), z, splat2(kSinP1[2])),
                   z, splat2(kSinP1[1])),
        z, splat2(kSinP1[0]));
    return __ffma2_rn(h.y, splat2(kSinC0), __fmul2_rn(__fmul2_rn(h.y, z), p));
}

// One particle-step's three normals from m = (-2 ln u1, -2 ln u3) and
// x = (4 u2, 4 u4): g0 = rho1 cos(2 pi u2), g1 = rho1 sin(2 pi u2),
// g2 = rho3 cos(2 pi u4).
__device__ __forceinline__ void box_muller3_x(float2 m2log, float2 x, float& g0, float& g1, float& g2)
{
    const float2 rho = make_float2(sqrt_pos(m2log.x), sqrt_pos(m2log.y));
    const HalfTurn2 h = half_turn2(x);
    const float2 sr = __fmul2_rn(h.sgn, rho);
    const float2 g = __fmul2_rn(sr, cos_half2(h));
    g0 = g.x;
    g2 = g.y;
    g1 = __fmul_rn(sr.x, sin_half(HalfTurn{h.sgn.x, h.y.x, h.z.x, h.f1.x}));
}

// Four raw 32-bit draws -> three normals.
__device__ __forceinline__ void box_muller3_u32(uint32_t r1, uint32_t r2, uint32_t r3, uint32_t r4,
                                                float& g0, float& g1, float& g2)
{
    const float2 u = make_float2(open01_from_u32(r1), open01_from_u32(r3));
    const float2 x = __ffma2_rn(splat2(4.0f), make_float2(mant_from_u32(r2), mant_from_u32(r4)),
                                splat2(-0x1.fffffep+1f));
    box_muller3_x(neg2log2(u), x, g0, g1, g2);
}

// Ran2's four uniforms -> three normals.
__device__ __forceinline__ void box_muller3(float u1, float u2, float u3, float u4, float& g0,
                                            float& g1, float& g2)
{
    box_muller3_x(neg2log2(make_float2(u1, u3)), __fmul2_rn(splat2(4.0f), make_float2(u2, u4)), g0,
                  g1, g2);
}

// Two oscillators side by side (lane j = oscillator j): the pair (rho cos,
// rho sin) and the cosine branch.
__device__ __forceinline__ void box_muller_pair2(float2 m2log, float2 x, float2& gc, float2& gs)
{
    const float2 rho = make_float2(sqrt_pos(m2log.x), sqrt_pos(m2log.y));
    const HalfTurn2 h = half_turn2(x);
    const float2 sr = __fmul2_rn(h.sgn, rho);
    gc = __fmul2_rn(sr, cos_half2(h));
    gs = __fmul2_rn(sr, sin_half2(h));
}

__device__ __forceinline__ float2 box_muller_cos2(float2 m2log, float2 x)
{
    const float2 rho = make_float2(sqrt_pos(m2log.x), sqrt_pos(m2log.y));
    const HalfTurn2 h = half_turn2(x);
    return __fmul2_rn(__fmul2_rn(h.sgn, rho), cos_half2(h));
}

// Two Box-Muller pairs side by side, from draws (r1, r2) and (r3, r4): a =
// box_muller_u32(r1, r2), b = box_muller_u32(r3, r4), bit for bit.
__device__ __forceinline__ void box_muller_2pairs_u32(uint32_t r1, uint32_t r2, uint32_t r3, uint32_t r4,
                                                      float2& a, float2& b)
{
    const float2 u = make_float2(open01_from_u32(r1), open01_from_u32(r3));
    const float2 x = __ffma2_rn(splat2(4.0f), make_float2(mant_from_u32(r2), mant_from_u32(r4)),
                                splat2(-0x1.fffffep+1f));
    float2 gc, gs;
    box_muller_pair2(neg2log2(u), x, gc, gs);
    a = make_float2(gc.x, gs.x);
    b = make_float2(gc.y, gs.y);
}

// The same from Ran2's uniforms: a = box_muller(u1, u2), b = box_muller(u3, u4).
__device__ __forceinline__ void box_muller_2pairs(float u1, float u2, float u3, float u4, float2& a,
                                                  float2& b)
{
    float2 gc, gs;
    box_muller_pair2(neg2log2(make_float2(u1, u3)), __fmul2_rn(splat2(4.0f), make_float2(u2, u4)), gc,
                     gs);
    a = make_float2(gc.x, gs.x);
    b = make_float2(gc.y, gs.y);
}

// Three normals of a particle-step for each of two oscillators from their four
// raw draws r[j][0..3]: g[k] = (normal k of oscillator 0, normal k of
// oscillator 1).
__device__ __forceinline__ void normals3x2_u32(const uint32_t (&r)[2][4], float2 (&g)[3])
{
    const float2 ua = make_float2(open01_from_u32(r[0][0]), open01_from_u32(r[1][0]));
    const float2 ub = make_float2(open01_from_u32(r[0][2]), open01_from_u32(r[1][2]));
    const float2 xa = __ffma2_rn(splat2(4.0f), make_float2(mant_from_u32(r[0][1]), mant_from_u32(r[1][1])),
                                 splat2(-0x1.fffffep+1f));
    const float2 xb = __ffma2_rn(splat2(4.0f), make_float2(mant_from_u32(r[0][3]), mant_from_u32(r[1][3])),
                                 splat2(-0x1.fffffep+1f));
    box_muller_pair2(neg2log2(ua), xa, g[0], g[1]);
    g[2] = box_muller_cos2(neg2log2(ub), xb);
}

// The same from Ran2's uniforms u[j][0..3].
__device__ __forceinline__ void normals3x2_ran2(const float (&u)[2][4], float2 (&g)[3])
{
    const float2 xa = __fmul2_rn(splat2(4.0f), make_float2(u[0][1], u[1][1]));
    const float2 xb = __fmul2_rn(splat2(4.0f), make_float2(u[0][3], u[1][3]));
    box_muller_pair2(neg2log2(make_float2(u[0][0], u[1][0])), xa, g[0], g[1]);
    g[2] = box_muller_cos2(neg2log2(make_float2(u[0][2], u[1][2])), xb);
}

// Three normals of one particle-step from four draws of the generator.
struct TausDraw {
    uint4 y;
    __device__ __forceinline__ void normals3(float& gx, float& gy, float& gz)
    {
        const uint32_t r1 = taus_next(y);
        const uint32_t r2 = taus_next(y);
        const uint32_t r3 = taus_next(y);
        const uint32_t r4 = taus_next(y);
        box_muller3_u32(r1, r2, r3, r4, gx, gy, gz);
    }
};

struct LcgDraw {
    uint32_t x;
    __device__ __forceinline__ void normals3(float& gx, float& gy, float& gz)
    {
        const uint32_t r1 = lcg_next(x);
        const uint32_t r2 = lcg_next(x);
        const uint32_t r3 = lcg_next(x);
        const uint32_t r4 = lcg_next(x);
        box_muller3_u32(r1, r2, r3, r4, gx, gy, gz);
    }
};

struct Ran2Draw {
    Ran2Regs r;
    int32_t* tab;
    int T, tid;
    __device__ __forceinline__ int32_t next()
    {
        int32_t* t = tab;
        const int TT = T, ti = tid;
        return ran2_next(r, [t, TT, ti](int j) -> int32_t& { return t[j * TT + ti]; });
    }
    __device__ __forceinline__ void normals3(float& gx, float& gy, float& gz)
    {
        const float u1 = u01_from_ran2(next());
        const float u2 = u01_from_ran2(next());
        const float u3 = u01_from_ran2(next());
        const float u4 = u01_from_ran2(next());
        box_muller3(u1, u2, u3, u4, gx, gy, gz);
    }
};

// Three normals of a particle-step for each of two oscillators with their own
// generators (lane j = oscillator j); each generator draws its four numbers
// in order, as in draw3.
template <int KIND, bool MUL = false>
__device__ __forceinline__ void draw3x2(TausDraw (&td)[2], LcgDraw (&lc)[2], Ran2Draw (&rd)[2],
                                        float2 (&g)[3])
{
    if (KIND == GBRNG_RAN2) {
        float u[2][4];
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) u[j][q] = u01_from_ran2(rd[j].next());
        normals3x2_ran2(u, g);
    } else {
        uint32_t r[2][4];
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q)
                r[j][q] = KIND == GBRNG_TAUS ? taus_next<MUL>(td[j].y) : lcg_next(lc[j].x);
        normals3x2_u32(r, g);
    }
}

// Three normals of one particle-step from the per-thread generator KIND.
template <int KIND>
__device__ __forceinline__ void draw3(TausDraw& td, LcgDraw& lc, Ran2Draw& rd, float& g0, float& g1,
                                      float& g2)
{
    if (KIND == GBRNG_TAUS)
        td.normals3(g0, g1, g2);
    else if (KIND == GBRNG_LCG)
        lc.normals3(g0, g1, g2);
    else
        rd.normals3(g0, g1, g2);
}

// ------------------------------------------------------------------ LD step
// v' = fma(cva, v, fma(-ckx, x, cs * g)),  x' = fma(cdt, v, x).
__device__ __forceinline__ void em_component(float cdt, float cva, float ckx, float cs, float g,
                                             float& x, float& v)
{
    const float t = __fmaf_rn(-ckx, x, __fmul_rn(cs, g));
    const float vn = __fmaf_rn(cva, v, t);
    x = __fmaf_rn(cdt, v, x);
    v = vn;
}

// Two oscillators' components side by side (lane j = oscillator j), each lane
// em_component; nckx = -(ckm K_j).
__device__ __forceinline__ void em_component2(float2 cdt, float2 cva, float2 nckx, float2 cs, float2 g,
                                              float2& x, float2& v)
{
    const float2 t = __ffma2_rn(nckx, x, __fmul2_rn(cs, g));
    const float2 vn = __ffma2_rn(cva, v, t);
    x = __ffma2_rn(cdt, v, x);
    v = vn;
}

// Energy (m|v|^2 + K|x|^2)/2 of one oscillator with a fixed operation order
// (hK = K/2, hm = m/2), so every kernel accumulates identical values.
__device__ __forceinline__ float energy3(float hK, float hm, float x0, float x1, float x2, float v0,
                                         float v1, float v2)
{
    const float xx = __fmaf_rn(x2, x2, __fmaf_rn(x1, x1, __fmul_rn(x0, x0)));
    const float vv = __fmaf_rn(v2, v2, __fmaf_rn(v1, v1, __fmul_rn(v0, v0)));
    return __fmaf_rn(hK, xx, __fmul_rn(hm, vv));
}

// Kahan-compensated binary32 accumulator.
struct Kahan {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float e)
    {
        const float y = __fsub_rn(e, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Time sum of one oscillator's energy E_t = hK |x_t|^2 + hm |v_t|^2, with hK
// and hm fixed for the oscillator: |x_t|^2 and |v_t|^2 are summed in binary32
// over blocks of at most kEnergyBlock steps, each block is folded into a Kahan
// sum, and the energy sum is formed once, in double, from the two sums.
constexpr int kEnergyBlock = 16;

__device__ __forceinline__ float norm2(float a0, float a1, float a2)
{
    return __fmaf_rn(a2, a2, __fmaf_rn(a1, a1, __fmul_rn(a0, a0)));
}

struct EnergySum {
    Kahan X, V;
    float bx = 0.f, bv = 0.f;
    __device__ __forceinline__ void add(float x0, float x1, float x2, float v0, float v1, float v2)
    {
        bx = __fadd_rn(bx, norm2(x0, x1, x2));
        bv = __fadd_rn(bv, norm2(v0, v1, v2));
    }
    __device__ __forceinline__ void flush()
    {
        X.add(bx);
        V.add(bv);
        bx = bv = 0.f;
    }
    __device__ __forceinline__ double value(float hK, float hm) const
    {
        return (double)hK * X.value() + (double)hm * V.value();
    }
};

// EnergySum of two oscillators, the block sums of |x|^2 and |v|^2 in the two
// lanes (norm2 and the block addition lane by lane).
struct EnergySum2 {
    Kahan X[2], V[2];
    float2 bx = {0.f, 0.f}, bv = {0.f, 0.f};
    __device__ __forceinline__ static float2 norm2x2(const float2 (&a)[3])
    {
        return __ffma2_rn(a[2], a[2], __ffma2_rn(a[1], a[1], __fmul2_rn(a[0], a[0])));
    }
    __device__ __forceinline__ void add(const float2 (&x)[3], const float2 (&v)[3])
    {
        bx = __fadd2_rn(bx, norm2x2(x));
        bv = __fadd2_rn(bv, norm2x2(v));
    }
    __device__ __forceinline__ void flush()
    {
        X[0].add(bx.x), X[1].add(bx.y);
        V[0].add(bv.x), V[1].add(bv.y);
        bx = bv = make_float2(0.f, 0.f);
    }
    __device__ __forceinline__ double value(int j, float hK, float hm) const
    {
        return (double)hK * X[j].value() + (double)hm * V[j].value();
    }
};

// Deterministic block reduction of N doubles per thread (fixed tree order);
// thread 0 receives the block totals in `v`.  smem must hold N*32 doubles.
template <int N>
__device__ __forceinline__ void block_reduce_sum(double (&v)[N], double* smem)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < N; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < N; ++k) smem[k * 32 + warp] = v[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) {
            v[k] = lane < nwarps ? smem[k * 32 + lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
        }
    }
    __syncthreads();
}

// Cheap global-timer read for bounded waits.
__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void red_release_add_u64(uint64_t* p, uint64_t v)
{
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void st_release_u64(uint64_t* p, uint64_t v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p)
{
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint64_t ld_acquire_u64(const uint64_t* p)
{
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_volatile_i32(const int* p)
{
    return *(const volatile int*)p;
}

}  // namespace gb
