"""Pins of the CPU oracle's Langevin-dynamics path (no GPU): closed forms at
zero noise, the exact covariance of the discrete scheme, run splitting, and the
adjoint against central finite differences."""
import math

import numpy as np
import pytest

import oracle


def _A(K, m, gamma, dt):
    return np.array([[1.0, dt], [-dt * K / m, 1.0 - gamma * dt / m]])


@pytest.mark.parametrize("kind", ["taus", "ran2", "lagfib"])
def test_zero_noise_matches_matrix_power(kind):
    """kT = 0 removes the random force G (Sec. I), so the first-order scheme is
    the linear map s_{t+1} = A s_t per component; A^n s_0 (numpy) pins the
    signs and coefficients of both updates and the use of the old v in x."""
    n, steps = 64, 500
    K, m, gamma, dt = 1.7, 1.3, 0.4, 0.01
    p = oracle.params(K=K, m=m, gamma=gamma, kT=0.0, dt=dt)
    rng = np.random.default_rng(0)
    x0 = rng.standard_normal((n, 3))
    v0 = rng.standard_normal((n, 3))
    x, v = x0.copy(), v0.copy()
    oracle.ld_run_f64(oracle.Gen(kind, 1, n), x, v, p, steps)
    An = np.linalg.matrix_power(_A(K, m, gamma, dt), steps)
    xe = An[0, 0] * x0 + An[0, 1] * v0
    ve = An[1, 0] * x0 + An[1, 1] * v0
    assert np.allclose(x, xe, rtol=1e-11, atol=1e-12)
    assert np.allclose(v, ve, rtol=1e-11, atol=1e-12)
    xf, vf = x0.astype(np.float32), v0.astype(np.float32)
    oracle.ld_run_f32(oracle.Gen(kind, 1, n), xf, vf, p, steps)
    scale = max(np.abs(xe).max(), np.abs(ve).max())
    assert np.abs(xf - xe).max() < 5e-6 * scale and np.abs(vf - ve).max() < 5e-6 * scale


@pytest.mark.parametrize("kind", ["taus", "ran2", "lagfib", "lcg"])
def test_zero_friction_removes_the_noise(kind):
    """gamma = 0 with kT > 0: the random force's amplitude sqrt(2 kT gamma dt)
    (Sec. I) vanishes with the friction, so the FP64 run is the undamped map
    A^n s_0 although kT > 0 (a noise amplitude missing its gamma would fail),
    and the generator still advances by four draws a particle-step."""
    n, steps = 48, 400
    K, m, dt = 0.9, 1.2, 0.02
    p = oracle.params(K=K, m=m, gamma=0.0, kT=3.0, dt=dt)
    rng = np.random.default_rng(3)
    x0 = rng.standard_normal((n, 3))
    v0 = rng.standard_normal((n, 3))
    x, v = x0.copy(), v0.copy()
    g = oracle.Gen(kind, 9, n)
    oracle.ld_run_f64(g, x, v, p, steps)
    An = np.linalg.matrix_power(_A(K, m, 0.0, dt), steps)
    assert np.allclose(x, An[0, 0] * x0 + An[0, 1] * v0, rtol=1e-11, atol=1e-12)
    assert np.allclose(v, An[1, 0] * x0 + An[1, 1] * v0, rtol=1e-11, atol=1e-12)
    ref = oracle.Gen(kind, 9, n)
    ref.fill_u32(4 * n * steps)
    if kind == "lagfib":
        assert np.array_equal(g.ring_in_order(), ref.ring_in_order())
    else:
        assert np.array_equal(g.state, ref.state)


def test_zero_noise_first_order_convergence():
    """The scheme is first order in dt: against the exact underdamped
    oscillator x(t) = e^{-gt/2m}(x0 cos wt + ((v0 + g x0/2m)/w) sin wt), the
    error at fixed t halves when dt halves."""
    K, m, gamma, T = 1.0, 1.0, 0.5, 2.0
    w = math.sqrt(K / m - (gamma / (2 * m)) ** 2)
    x0, v0 = 1.0, 0.0
    exact = math.exp(-gamma * T / (2 * m)) * (
        x0 * math.cos(w * T) + (v0 + gamma * x0 / (2 * m)) / w * math.sin(w * T))
    errs = []
    for dt in [0.02, 0.01, 0.005, 0.0025]:
        x = np.array([[x0, 0, 0]], float)
        v = np.array([[v0, 0, 0]], float)
        oracle.ld_run_f64(oracle.Gen("taus", 1, 1), x, v,
                          oracle.params(K=K, m=m, gamma=gamma, kT=0.0, dt=dt), int(round(T / dt)))
        errs.append(abs(x[0, 0] - exact))
    for a, b in zip(errs, errs[1:]):
        assert 1.8 < a / b < 2.2


def test_em_covariance_closed_form():
    """Stationary covariance of the discrete scheme (m = 1), derived from
    Sigma = A Sigma A^T + Q:  Svv = kT / (1 - g dt/2 - K dt/g + 3K dt^2/4
    - K^2 dt^3/(4g)),  Sxx = Svv (1 - g dt/2 + K dt^2/2)/K,  Sxv = -dt Svv/2;
    also checked against scipy's discrete Lyapunov solver."""
    linalg = pytest.importorskip("scipy.linalg")
    K, g, kT, dt = 1.0, 0.5, 1.0, 0.01
    S = oracle.em_covariance(K, 1.0, g, kT, dt, 40000)
    svv = kT / (1 - g * dt / 2 - K * dt / g + 0.75 * K * dt**2 - K**2 * dt**3 / (4 * g))
    sxx = svv * (1 - g * dt / 2 + K * dt**2 / 2) / K
    assert math.isclose(S[1, 1], svv, rel_tol=1e-9)
    assert math.isclose(S[0, 0], sxx, rel_tol=1e-9)
    assert math.isclose(S[0, 1], -dt * svv / 2, rel_tol=1e-9)
    assert math.isclose(sxx, 1.020434, rel_tol=1e-6) and math.isclose(svv, 1.022940, rel_tol=1e-6)
    A = _A(K, 1.0, g, dt)
    Q = np.diag([0.0, 2 * g * kT * dt])
    assert np.allclose(linalg.solve_discrete_lyapunov(A, Q), S, rtol=1e-9)


@pytest.mark.parametrize("kind", ["taus", "ran2", "lagfib"])
def test_equipartition_discrete(kind):
    """Random force <G G> = 2 kT xi delta (Sec. I) fixes sigma^2 = 2 gamma kT dt:
    starting from x ~ N(0, kT/K), v ~ N(0, kT/m) (the equilibrium draw), the
    sample moments after t steps match the exactly propagated covariance
    within 4 sigma.  A coarse dt = 0.1 makes the discretisation bias (~20%)
    far larger than the tolerance, so a wrong noise amplitude cannot pass."""
    n, steps = 20000, 300
    K, m, g, kT, dt = 1.0, 1.0, 0.5, 1.0, 0.1
    p = oracle.params(K=K, m=m, gamma=g, kT=kT, dt=dt)
    gen = oracle.Gen(kind, 31337, n)
    x, v = oracle.ld_init_eq_f64(gen, n, p)
    for arr, var in ((x, kT / K), (v, kT / m)):
        assert abs(arr.var() - var) < 4 * var * math.sqrt(2 / arr.size)
    oracle.ld_run_f64(gen, x, v, p, steps)
    S = oracle.em_covariance(K, m, g, kT, dt, steps)
    cnt = x.size
    assert abs((x * x).mean() - S[0, 0]) < 4 * S[0, 0] * math.sqrt(2 / cnt)
    assert abs((v * v).mean() - S[1, 1]) < 4 * S[1, 1] * math.sqrt(2 / cnt)
    sd_xv = math.sqrt((S[0, 0] * S[1, 1] + S[0, 1] ** 2) / cnt)
    assert abs((x * v).mean() - S[0, 1]) < 4 * sd_xv
    assert abs(S[0, 0] - kT / K) > 10 * S[0, 0] * math.sqrt(2 / cnt)   # bias resolved


@pytest.mark.parametrize("kind", ["taus", "ran2", "lagfib"])
def test_run_splitting_bit_exact(kind):
    """Generator state carries over between calls (Algorithms 1-3 save the
    state at the end of each step): run(a) then run(b) equals run(a+b)."""
    n = 37
    p = oracle.params()
    g1 = oracle.Gen(kind, 5, n)
    x1, v1 = oracle.ld_init_eq_f32(g1, n, p)
    g2 = g1.copy()
    x2, v2 = x1.copy(), v1.copy()
    oracle.ld_run_f32(g1, x1, v1, p, 70)
    oracle.ld_run_f32(g2, x2, v2, p, 30)
    oracle.ld_run_f32(g2, x2, v2, p, 40)
    assert np.array_equal(x1, x2) and np.array_equal(v1, v2)
    assert np.array_equal(g1.state, g2.state)
    if kind == "lagfib":
        assert g1.pos == g2.pos == 4 * n * (2 + 70)


def test_f32_tracks_f64():
    """The binary32 trajectory stays within ~1e-5 (relative to the rms) of
    the FP64 trajectory driven by the same integer streams."""
    n = 256
    p = oracle.params()
    ga, gb = oracle.Gen("taus", 1234, n), oracle.Gen("taus", 1234, n)
    xf, vf = oracle.ld_init_eq_f32(ga, n, p)
    xd, vd = oracle.ld_init_eq_f64(gb, n, p)
    assert np.abs(xf - xd).max() < 1e-6 * np.abs(xd).max()
    oracle.ld_run_f32(ga, xf, vf, p, 1000)
    oracle.ld_run_f64(gb, xd, vd, p, 1000)
    rms = math.sqrt((xd * xd).mean())
    assert np.abs(xf - xd).max() < 1e-5 * rms


def test_kper_equals_scalar():
    """A per-oscillator K array of equal values reproduces the scalar K."""
    n = 50
    p = oracle.params(K=2.5)
    ga, gb = oracle.Gen("ran2", 8, n), oracle.Gen("ran2", 8, n)
    xa, va = oracle.ld_init_eq_f32(ga, n, p)
    xb, vb = oracle.ld_init_eq_f32(gb, n, p, Kper=np.full(n, 2.5, np.float32))
    oracle.ld_run_f32(ga, xa, va, p, 100)
    oracle.ld_run_f32(gb, xb, vb, p, 100, Kper=np.full(n, 2.5, np.float32))
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)


def _loss_per_osc(kind, seed, n, x0, v0, K, m, g, kT, dt, S, Kper):
    x, v = x0.copy(), v0.copy()
    r = oracle.ld_run_f64(oracle.Gen(kind, seed, n), x, v,
                          oracle.params(K=K, m=m, gamma=g, kT=kT, dt=dt), S, Kper=Kper,
                          per_osc=True)
    return r["loss_per_osc"]


@pytest.mark.parametrize("kind", ["taus", "ran2"])
def test_adjoint_matches_central_differences(kind):
    """Reverse-time adjoint of the trajectory-averaged energy under fixed noise
    versus central finite differences (h = 1e-3 relative) in FP64.  The loss is
    a sum over oscillators, each depending on its own K_i only, so one
    perturbed run gives every dL/dK_i."""
    n, S = 32, 600
    m, g, kT, dt = 1.0, 0.5, 1.0, 0.01
    rng = np.random.default_rng(4)
    Kper = rng.uniform(0.5, 2.0, n)
    x0 = rng.standard_normal((n, 3))
    v0 = rng.standard_normal((n, 3))
    x, v = x0.copy(), v0.copy()
    adj = oracle.ld_adjoint_f64(oracle.Gen(kind, 9, n), x, v,
                                oracle.params(K=1.0, m=m, gamma=g, kT=kT, dt=dt), S, Kper=Kper)
    base = _loss_per_osc(kind, 9, n, x0, v0, 1.0, m, g, kT, dt, S, Kper)
    assert np.allclose(adj["loss_per_osc"], base, rtol=1e-13)
    h = 1e-3
    lp = _loss_per_osc(kind, 9, n, x0, v0, 1.0, m, g, kT, dt, S, Kper * (1 + h))
    lm = _loss_per_osc(kind, 9, n, x0, v0, 1.0, m, g, kT, dt, S, Kper * (1 - h))
    fd_K = (lp - lm) / (2 * h * Kper)
    assert np.allclose(adj["dK"], fd_K, rtol=1e-4, atol=1e-6 * np.abs(fd_K).max())
    for name, idx in (("dgamma", 2), ("dkT", 3)):
        args = [1.0, m, g, kT, dt]
        hp = list(args)
        hm = list(args)
        hp[idx] *= 1 + h
        hm[idx] *= 1 - h
        fp = _loss_per_osc(kind, 9, n, x0, v0, *hp, S, Kper).sum()
        fm = _loss_per_osc(kind, 9, n, x0, v0, *hm, S, Kper).sum()
        fd = (fp - fm) / (2 * h * args[idx])
        assert math.isclose(adj[name], fd, rel_tol=1e-4), (name, adj[name], fd)


def test_adjoint_unbiased_for_exact_gradient():
    """The mean of the pathwise gradient equals d E[L] / d kT computed exactly
    from the covariance recursion (noise enters linearly), within the
    sampling error: a check of the adjoint independent of finite differences."""
    n, S = 4000, 200
    K, m, g, kT, dt = 1.0, 1.0, 0.5, 1.0, 0.02
    rng = np.random.default_rng(5)
    x0 = rng.standard_normal((n, 3)) * math.sqrt(kT / K)
    v0 = rng.standard_normal((n, 3)) * math.sqrt(kT / m)
    adj = oracle.ld_adjoint_f64(oracle.Gen("taus", 21, n), x0.copy(), v0.copy(),
                                oracle.params(K=K, m=m, gamma=g, kT=kT, dt=dt), S)

    def expected_loss(kT_):
        A = _A(K, m, g, dt)
        Q = np.diag([0.0, 2 * g * kT_ * dt / m**2])
        Sig = np.diag([kT / K, kT / m])   # fixed initial ensemble
        tot = 0.0
        for _ in range(S):
            Sig = A @ Sig @ A.T + Q
            tot += 0.5 * m * Sig[1, 1] + 0.5 * K * Sig[0, 0]
        return 3 * n * tot / S

    eps = 1e-4
    d_exact = (expected_loss(kT + eps) - expected_loss(kT - eps)) / (2 * eps)
    # sampling error of the mean over 4000 oscillators is ~0.3%
    assert abs(adj["dkT"] - d_exact) < 0.01 * abs(d_exact)
