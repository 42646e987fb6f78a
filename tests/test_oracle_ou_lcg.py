"""Pins of the oracle's Quick and Dirty LCG (Eq. 1) and overdamped 1-D
Langevin run (Eq. 4-5) against facts the mathematics fixes: the LCG's jump-ahead
closed form, its bit periods and full period (Hull-Dobell), and the discrete
Ornstein-Uhlenbeck moments E[R_t] = R0 a^t, Var[R_t] = s^2 (1 - a^2t)/(1 - a^2),
E[R_t R_0] = s^2/(1 - a^2) a^t from a stationary start, plus the paper's
continuous-time curves R0 exp(-t/tau) and (kT/k_sp) exp(-t/tau) at small dt."""
import math

import numpy as np
import pytest

import oracle

A, C_, M = 1664525, 1013904223, 2**32


def lcg_jump(x0: int, n: int) -> int:
    """x_n = a^n x_0 + c (a^n - 1)/(a - 1) mod 2^32, the sum as a geometric
    series evaluated by repeated squaring (no iteration of the recurrence)."""
    an, geo = 1, 0                 # a^n, 1 + a + ... + a^(n-1)
    base, bgeo = A, 1              # a^(2^k), 1 + a + ... + a^(2^k - 1)
    while n:
        if n & 1:
            geo = (geo * base + bgeo) % M
            an = (an * base) % M
        bgeo = (bgeo * base + bgeo) % M
        base = (base * base) % M
        n >>= 1
    return (an * x0 + C_ * geo) % M


@pytest.mark.parametrize("seed", [0, 1, 7, 123456789])
def test_lcg_matches_jump_ahead_closed_form(seed):
    g = oracle.Gen("lcg", seed, 3)
    x0 = [int(v) for v in g.state]
    out = g.fill_u32(3000)
    for s in range(3):
        for n in (1, 2, 17, 999, 1000):
            assert int(out[(n - 1) * 3 + s]) == lcg_jump(x0[s], n)


def test_lcg_low_bits_have_short_periods():
    """m = 2^32 with odd a and c: bit k of x_n has period 2^(k+1) (the flaw
    that makes the LCG a negative control)."""
    x = np.array([2463534242], np.uint32)
    seq = np.array([oracle.lcg_next(x) for _ in range(1 << 13)], np.uint64)
    for k in range(12):
        b = (seq >> np.uint64(k)) & np.uint64(1)
        p = 1 << (k + 1)
        assert np.array_equal(b[p:], b[:-p])
        assert not np.array_equal(b[p // 2:], b[:-(p // 2)])


def test_lcg_full_period():
    """Hull-Dobell: c odd and a - 1 divisible by 4 give period 2^32 from any seed."""
    assert (C_ & 1) and (A - 1) % 4 == 0
    assert oracle.lib().or_lcg_period(12345) == 2**32


def test_lcg_stream_seed_is_first_splitmix_word():
    g = oracle.Gen("lcg", 99, 5)
    for s in range(5):
        assert int(g.state[s]) == oracle.splitmix64(99, 8 * s) & 0xFFFFFFFF


def test_ou_zero_noise_is_geometric_decay():
    n, steps = 64, 5000
    p = oracle.ou_params(k_sp=2.0, xi=3.0, kT=0.0, dt=1e-3)
    R = np.linspace(-5, 5, n).astype(np.float32)
    R0 = R.astype(np.float64).copy()
    mean, _ = oracle.ou_run_f32(oracle.Gen("taus", 1, n), R, p, steps, steps)
    c1 = float(np.float32(2.0 * 1e-3 / 3.0))
    exact = R0 * (1.0 - c1) ** steps
    assert np.abs(R - exact).max() <= steps * 2**-23 * np.abs(R0).max()
    assert mean[0] == pytest.approx(R0.mean(), abs=1e-12)


@pytest.mark.parametrize("kind", ["taus", "ran2", "lagfib"])
def test_ou_mean_and_variance_match_discrete_moments(kind):
    n, steps, every = 20000, 300, 50
    dt, k_sp, xi, kT = 0.01, 1.5, 2.0, 1.0
    p = oracle.ou_params(k_sp=k_sp, xi=xi, kT=kT, dt=dt)
    R = np.full(n, 10.0, np.float32)
    mean, _ = oracle.ou_run_f32(oracle.Gen(kind, 5, n), R, p, steps, every)
    a = 1.0 - k_sp * dt / xi
    s2 = 2.0 * kT * dt / xi
    for r, m in enumerate(mean):
        t = r * every
        var_t = s2 * (1 - a ** (2 * t)) / (1 - a * a)
        assert abs(m - 10.0 * a**t) <= 4.0 * math.sqrt(var_t / n) + 1e-6
    var_t = s2 * (1 - a ** (2 * steps)) / (1 - a * a)
    sample = float(np.var(R.astype(np.float64)))
    assert abs(sample / var_t - 1.0) < 4.0 * math.sqrt(2.0 / n)


def test_ou_stationary_correlation():
    n, steps, every = 20000, 400, 100
    dt = 0.01
    p = oracle.ou_params(k_sp=1.0, xi=1.0, kT=1.0, dt=dt)
    a = 1.0 - dt
    var_eq = 2.0 * dt / (1 - a * a)
    R = (np.random.default_rng(3).standard_normal(n) * math.sqrt(var_eq)).astype(np.float32)
    _, corr = oracle.ou_run_f32(oracle.Gen("taus", 8, n), R, p, steps, every)
    for r, c in enumerate(corr):
        t = r * every
        exp = var_eq * a**t
        sd = var_eq * math.sqrt((1 + a ** (2 * t)) / n)
        assert abs(c - exp) <= 4.0 * sd


def test_ou_paper_curves_at_small_dt():
    """tau = xi/k_sp; with dt/tau = 1e-3 the discrete a^t is exp(-t dt/tau)
    to 5e-4, so the paper's exact curves hold within sampling error."""
    n, steps, every = 20000, 1000, 250
    k_sp, xi, kT, dt = 0.5, 1.0, 2.0, 2e-3
    tau = xi / k_sp
    p = oracle.ou_params(k_sp=k_sp, xi=xi, kT=kT, dt=dt)
    R = np.full(n, 10.0, np.float32)
    mean, _ = oracle.ou_run_f32(oracle.Gen("ran2", 2, n), R, p, steps, every)
    for r, m in enumerate(mean):
        t = r * every * dt
        sd = math.sqrt(kT / k_sp * (1 - math.exp(-2 * t / tau)) / n)
        assert abs(m - 10.0 * math.exp(-t / tau)) <= 4 * sd + 10.0 * 5e-4


def test_lcg_first_outputs_from_zero():
    """From x = 0 the first two words are c = 0x3C6EF35F and a c + c mod 2^32 =
    0x47502932 (the Hybrid Taus LCG word advances the same way)."""
    x = np.zeros(1, np.uint32)
    assert oracle.lcg_next(x) == 0x3C6EF35F
    assert oracle.lcg_next(x) == 0x47502932
    y = np.array([0, 0, 0, 0], np.uint32)
    oracle.taus_next(y)
    assert int(y[3]) == 0x3C6EF35F
