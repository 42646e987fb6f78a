"""Fit the polynomial coefficients of the Box-Muller transcendentals used by
the kernels and write them to bm_coeffs.cuh (run from the repository root):

    python paper_1003_1123_gb300/csrc/fit_bm_coeffs.py

The approximations are reduced-range ones:
  * ln(u): u = 2^e m with m in [2/3, 4/3), f = m - 1 (exact), and
    ln(m) = f + f^2 R(f); R is a degree-8 polynomial.
  * sin / cos of 2 pi u, x = 4u (exact), in one of two forms (each generator
    uses one form in all of its kernels):
    - quadrant form: q = rint(x), r = x - q in [-1/2, 1/2] (exact),
      theta = (pi/2) r; sin(theta) = r S(r^2) (degree 3 in r^2),
      cos(theta) = C(r^2) (degree 4 in r^2); the quadrant q rotates (s, c).
    - half-turn form: n = rint(x / 2) in {0, 1, 2}, y = x - 2n in [-1, 1]
      (exact), z = y^2; sin(2 pi u) = (-1)^n sin(pi y / 2) and
      cos(2 pi u) = (-1)^n cos(pi y / 2) with
      sin(pi y / 2) = y c0 + y z P1(z)      (c0 = pi/2 rounded; P1 of degree 4),
      cos(pi y / 2) = (1 - z)(1 + z Q1(z))  (Q1 of degree 3),
      so that no quadrant selection is needed and the zeros of the cosine at
      y = +-1 come from the factor 1 - z, rounded once.
Each polynomial is a least-squares fit in double precision on Chebyshev nodes
of its interval (the half-turn ones weighted by the relative error they cause
in the result), rounded to binary32.  The script then evaluates the binary32
schemes the kernels use (fused multiply-adds emulated in double) on every
input the Taus / LCG / Lagged Fibonacci draws produce (u = (k + 1/2) 2^-23)
and prints the largest error in units in the last place.
"""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
C0 = np.float32(np.pi / 2)


def _R_exact(f):
    f = np.asarray(f, np.float64)
    out = np.empty_like(f)
    small = np.abs(f) < 1e-2
    fs = f[small]
    s = np.zeros_like(fs)
    for k in range(2, 20):
        s += (-1) ** (k + 1) * fs ** (k - 2) / k
    out[small] = s
    fb = f[~small]
    out[~small] = (np.log1p(fb) - fb) / fb ** 2
    return out


def _fit(var, y, deg, w=None):
    V = np.vander(var, deg + 1, increasing=True)
    if w is None:
        w = np.ones_like(var)
    c, *_ = np.linalg.lstsq(V * w[:, None], y * w, rcond=None)
    return c.astype(np.float32)


def _fma32(a, b, c):
    return (np.float64(a) * np.float64(b) + np.float64(c)).astype(np.float32)


def _mul32(a, b):
    return (np.float64(a) * np.float64(b)).astype(np.float32)


def _horner32(c, x):
    r = np.full_like(x, c[-1])
    for cc in c[-2::-1]:
        r = _fma32(r, x, cc)
    return r


def fit_all():
    """Returns (c_log, c_sin_quarter, c_cos_quarter, c_sin_half, c_cos_half)."""
    n = 20001
    k = np.arange(n)
    f = (1 / 3) * np.cos(np.pi * (k + 0.5) / n)
    c_log = _fit(f, _R_exact(f), 8)
    h = np.pi / 2
    r = 0.5 * np.cos(np.pi * (k + 0.5) / (2 * n))
    c_sin_q = _fit(r * r, np.sin(h * r) / r, 3)
    c_cos_q = _fit(r * r, np.cos(h * r), 4)
    m = 40001
    k = np.arange(m)
    y = np.cos(np.pi * (k + 0.5) / (2 * m))          # (0, 1]
    z = y * y
    near1 = np.abs(1 - z) < 1e-9
    Q = np.where(near1, np.pi / 4, np.cos(h * y) / np.where(near1, 1.0, 1 - z))
    P = np.sin(h * y) / y
    c_cos_h = _fit(z, (Q - 1) / z, 3, z / np.abs(Q))
    c_sin_h = _fit(z, (P - np.float64(C0)) / z, 4, z / np.abs(P))
    return c_log, c_sin_q, c_cos_q, c_sin_h, c_cos_h


def sincos_quarter32(x, c_sin, c_cos):
    """The quadrant form in binary32 at x = 4u: (sin, cos) of 2 pi u."""
    q = np.rint(x.astype(np.float64)).astype(np.float32)
    r = (x.astype(np.float64) - q).astype(np.float32)
    z = _mul32(r, r)
    st = _mul32(r, _horner32(c_sin, z))
    z2 = _mul32(z, z)
    ct = _fma32(_fma32(c_cos[4], z2, _fma32(c_cos[3], z, c_cos[2])), z2,
                _fma32(c_cos[1], z, c_cos[0]))
    qi = q.astype(np.int64)
    swap = (qi & 1) == 1
    so, co = np.where(swap, ct, st), np.where(swap, st, ct)
    return np.where(qi & 2, -so, so), np.where((qi + 1) & 2, -co, co)


def sincos_half32(x, c_sin, c_cos):
    """The half-turn form in binary32 at x = 4u: (sin, cos) of 2 pi u."""
    nf = (_fma32(x, np.float32(0.5), np.float32(12582912.0)).astype(np.float64)
          - 12582912.0).astype(np.float32)
    y = _fma32(nf, np.float32(-2), x)
    sgn = _fma32(_fma32(nf, np.float32(2), np.float32(-4)), nf, np.float32(1))
    z = _mul32(y, y)
    f1 = _fma32(-y, y, np.float32(1))
    c = _fma32(_mul32(f1, z), _horner32(c_cos, z), f1)
    s = _fma32(y, C0, _mul32(_mul32(y, z), _horner32(c_sin, z)))
    return _mul32(sgn, s), _mul32(sgn, c)


def _ulp_err(got, exact):
    ulp = np.spacing(np.abs(exact).astype(np.float32)).astype(np.float64)
    return float((np.abs(got.astype(np.float64) - exact) / ulp).max())


def check(c_log, c_sin_q, c_cos_q, c_sin_h, c_cos_h):
    m = np.arange(np.float32(2 / 3).view(np.int32), np.float32(4 / 3).view(np.int32),
                  dtype=np.int32).view(np.float32)
    f = (m - np.float32(1)).astype(np.float32)
    t = (f.astype(np.float64) ** 2).astype(np.float32)
    l32 = _fma32(t, _horner32(c_log, f), f)
    ex = np.log(m.astype(np.float64))
    nz = ex != 0
    e_log = _ulp_err(l32[nz], ex[nz])
    u = (np.arange(2**23, dtype=np.float64) + 0.5) * 2.0**-23   # every u the draws give
    x = (4 * u).astype(np.float32)
    es, ec = np.sin(2 * np.pi * u), np.cos(2 * np.pi * u)
    sq, cq = sincos_quarter32(x, c_sin_q, c_cos_q)
    sh, ch = sincos_half32(x, c_sin_h, c_cos_h)
    return e_log, (_ulp_err(sq, es), _ulp_err(cq, ec)), (_ulp_err(sh, es), _ulp_err(ch, ec))


def _lit(v):
    return f"{float(np.float32(v)).hex()}f /* {float(np.float32(v)):.9g} */"


def main():
    coefs = fit_all()
    e_log, e_q, e_h = check(*coefs)
    c_log, c_sin_q, c_cos_q, c_sin_h, c_cos_h = coefs
    lines = ["// Generated by fit_bm_coeffs.py: least-squares polynomial coefficients of the",
             "// Box-Muller transcendentals (see that script for the reductions).",
             f"// Max error on the draws' input grid: ln(m) {e_log:.2f} ulp; quadrant form sin "
             f"{e_q[0]:.2f}, cos {e_q[1]:.2f} ulp;",
             f"// half-turn form sin {e_h[0]:.2f}, cos {e_h[1]:.2f} ulp.",
             "#pragma once", "", "namespace gb {", "",
             "// c0 = pi/2 rounded: the head of sin(pi y / 2) = y c0 + y z P1(z)",
             f"constexpr float kSinC0 = {_lit(C0)};", ""]
    for name, c in (("kLogR", c_log), ("kSinS", c_sin_q), ("kCosC", c_cos_q),
                    ("kSinP1", c_sin_h), ("kCosQ1", c_cos_h)):
        lines.append(f"// {name}[i]: coefficient of the i-th power")
        lines.append(f"constexpr float {name}[{len(c)}] = {{")
        lines += [f"    {_lit(v)}," for v in c]
        lines.append("};")
        lines.append("")
    lines += ["}  // namespace gb", ""]
    with open(os.path.join(HERE, "bm_coeffs.cuh"), "w") as fh:
        fh.write("\n".join(lines))
    print(f"ln(m) {e_log:.3f} ulp; quadrant sin {e_q[0]:.3f} cos {e_q[1]:.3f} ulp; "
          f"half-turn sin {e_h[0]:.3f} cos {e_h[1]:.3f} ulp")


if __name__ == "__main__":
    main()
