"""The Box-Muller polynomial coefficients the kernels compile in
(csrc/bm_coeffs.cuh) are the ones csrc/fit_bm_coeffs.py fits, and that
script's binary32 emulation of the kernels' evaluation (each fused
multiply-add rounded once) stays within the error bounds the GPU normal tests
rely on: ln(m) within 0.8 ulp on every m of the reduced range, sin and cos of
2 pi u within 1.9 ulp for every u the 32-bit draws give.  Also pins the
half-turn reduction itself: exact, and (-1)^n = (2n - 4) n + 1 for n in
{0, 1, 2}."""
import importlib.util
import os
import re

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_1003_1123_gb300", "csrc")


@pytest.fixture(scope="module")
def fb():
    spec = importlib.util.spec_from_file_location("fit_bm_coeffs",
                                                  os.path.join(CSRC, "fit_bm_coeffs.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def header_arrays():
    text = open(os.path.join(CSRC, "bm_coeffs.cuh")).read()
    out = {}
    for name, body in re.findall(r"constexpr float (\w+)\[\d+\] = \{(.*?)\};", text, re.S):
        out[name] = np.array([float.fromhex(h) for h in re.findall(r"(-?0x[0-9a-f.]+p[-+]\d+)f", body)],
                             np.float32)
    c0 = re.search(r"constexpr float kSinC0 = (-?0x[0-9a-f.]+p[-+]\d+)f", text).group(1)
    out["kSinC0"] = np.float32(float.fromhex(c0))
    return out


def test_header_holds_the_fitted_coefficients(fb):
    c_log, c_sin, c_cos = fb.fit_all()
    h = header_arrays()
    assert np.array_equal(h["kLogR"], c_log)
    assert np.array_equal(h["kSinP1"], c_sin)
    assert np.array_equal(h["kCosQ1"], c_cos)
    assert h["kSinC0"] == fb.C0 == np.float32(np.pi / 2)


def test_transcendental_error_bounds(fb):
    e_log, e_sin, e_cos = fb.check(*fb.fit_all())
    assert e_log <= 0.8
    assert e_sin <= 1.9
    assert e_cos <= 1.9


def test_half_turn_reduction_is_exact_with_the_right_sign(fb):
    # every x = 4u of the 32-bit draws, and Ran2-style uniforms k 2^-31 with
    # fine spacing near the quadrant boundaries
    u32 = (np.arange(0, 2**23, 997, dtype=np.float64) + 0.5) * 2.0**-23
    k = np.concatenate([np.arange(1, 4096), 2**29 + np.arange(-4096, 4096), 2**30 + np.arange(-4096, 4096),
                        3 * 2**29 + np.arange(-4096, 4096), 2**31 - np.arange(100, 4096)])
    uran = (k.astype(np.float32) * np.float32(2.0**-31)).astype(np.float64)
    for u in (u32, uran):
        x = (4 * u).astype(np.float32)
        nf = (fb._fma32(x, np.float32(0.5), np.float32(12582912.0)).astype(np.float64)
              - 12582912.0).astype(np.float32)
        y = fb._fma32(nf, np.float32(-2), x)
        assert np.array_equal(y.astype(np.float64), x.astype(np.float64) - 2 * nf.astype(np.float64))
        assert (np.abs(y) <= 1).all() and set(np.unique(nf)) <= {0.0, 1.0, 2.0}
        sgn = fb._fma32(fb._fma32(nf, np.float32(2), np.float32(-4)), nf, np.float32(1))
        assert np.array_equal(sgn, np.where(nf == 1, -1.0, 1.0).astype(np.float32))
        s32, c32 = fb.sincos_half32(x, *fb.fit_all()[1:])
        ex_s, ex_c = np.sin(2 * np.pi * u), np.cos(2 * np.pi * u)
        assert np.abs(s32 - ex_s).max() < 3e-7 and np.abs(c32 - ex_c).max() < 3e-7
