"""Reverse-time adjoint on the GPU (ld_backward, through the C ABI) against
the FP64 CPU adjoint of the oracle (itself pinned to central differences),
the system advance it leaves behind, the unbiasedness of the pathwise
gradient at scale, and the torch.autograd wrapper."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1003_1123_gb300 import workloads as W

pytestmark = pytest.mark.gpu
GRAD_RTOL = 1e-4


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1003_1123_gb300 import gbrng
    gbrng.lib()
    return gbrng


def make(G, kind, n, seed, Kper, gamma=0.5, kT=1.0, dt=0.01, m=1.0, start=None):
    """A system on the GPU; start = (x0, v0) float32 arrays, else the
    library's own equilibrium draw."""
    r = G.rng_init(kind, seed, n)
    x = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    v = torch.zeros_like(x)
    kt = torch.from_numpy(np.ascontiguousarray(Kper, np.float32)).cuda()
    s = G.LdSystem(r, x, v, K=1.0, m=m, gamma=gamma, kT=kT, dt=dt, K_per=kt)
    if start is None:
        G.ld_init_equilibrium(s)
    else:
        s.x.copy_(torch.from_numpy(start[0]))
        s.v.copy_(torch.from_numpy(start[1]))
    return s


@pytest.mark.parametrize("kind", ["taus", "ran2"])
@pytest.mark.parametrize("steps,ckpt", [(10**4, 100), (1037, 64), (50, 100), (1, 1)])
def test_adjoint_matches_fp64_oracle(G, kind, steps, ckpt):
    """N = 256 with per-oscillator K: loss, dL/dK_i, dL/dgamma, dL/dkT of the
    binary32 GPU adjoint within 1e-4 of the FP64 adjoint driven by the same
    integer streams (10^4 steps with checkpoints every 100 is the paper-scale
    case; ragged segment counts are covered too)."""
    n = W.ADJOINT["n_check"]
    Kper = W.spring_constants(n, 3, 0.5, 2.0)
    x0, v0 = W.initial_state(n, 17)
    s = make(G, kind, n, 77, Kper, start=(x0, v0))
    r = G.ld_backward(s, steps, ckpt)
    g = oracle.Gen(kind, 77, n)
    ref = oracle.ld_adjoint_f64(g, x0.astype(np.float64), v0.astype(np.float64),
                                oracle.params(K=1.0, m=1.0, gamma=0.5, kT=1.0, dt=0.01),
                                steps, Kper=Kper.astype(np.float64))
    assert math.isclose(r["loss"], ref["loss"], rel_tol=GRAD_RTOL)
    dK = r["dK"].cpu().numpy().astype(np.float64)
    scale = np.abs(ref["dK"]).max()
    assert np.abs(dK - ref["dK"]).max() <= GRAD_RTOL * scale
    for k in ("dgamma", "dkT"):
        assert math.isclose(r[k], ref[k], rel_tol=GRAD_RTOL, abs_tol=1e-6 * abs(ref["loss"])), (
            k, r[k], ref[k])


@pytest.mark.parametrize("kind", ["taus", "ran2"])
@pytest.mark.parametrize("Klo,Khi,gamma,kT,dt", [
    (5.0, 10.0, 2.0, 2.0, 0.005),     # stiff springs, strong friction, hot, the batched dt
    (5.0, 10.0, 2.0, 0.5, 0.01),      # stiff springs, strong friction, cold, coarse step
    (0.1, 0.5, 0.1, 2.0, 0.01),       # soft springs, weak friction
])
def test_adjoint_at_parameter_corners(G, kind, Klo, Khi, gamma, kT, dt):
    """The reverse sweep rebuilds x_t, v_t by inverting the binary32 step
    inside each 100-step segment; across the batched workload's parameter
    range (K up to 10, gamma 0.1 to 2, kT 0.5 to 2, dt 0.005 and 0.01) that
    rebuild stays within the 1e-4 bar of the FP64 adjoint over 5000 steps."""
    n, steps, ckpt = W.ADJOINT["n_check"], 5000, 100
    Kper = W.spring_constants(n, 8, Klo, Khi)
    x0, v0 = W.initial_state(n, 29)
    s = make(G, kind, n, 55, Kper, gamma=gamma, kT=kT, dt=dt, start=(x0, v0))
    r = G.ld_backward(s, steps, ckpt)
    g = oracle.Gen(kind, 55, n)
    ref = oracle.ld_adjoint_f64(g, x0.astype(np.float64), v0.astype(np.float64),
                                oracle.params(K=1.0, m=1.0, gamma=gamma, kT=kT, dt=dt),
                                steps, Kper=Kper.astype(np.float64))
    assert math.isclose(r["loss"], ref["loss"], rel_tol=GRAD_RTOL)
    dK = r["dK"].cpu().numpy().astype(np.float64)
    assert np.abs(dK - ref["dK"]).max() <= GRAD_RTOL * np.abs(ref["dK"]).max()
    for k in ("dgamma", "dkT"):
        assert math.isclose(r[k], ref[k], rel_tol=GRAD_RTOL, abs_tol=1e-6 * abs(ref["loss"])), (
            k, r[k], ref[k])


@pytest.mark.parametrize("kind", ["taus", "ran2"])
def test_backward_advances_like_run(G, kind):
    """After ld_backward the system and its generator are exactly where
    ld_run would have left them."""
    n = 999
    Kper = W.spring_constants(n, 4)
    a = make(G, kind, n, 5, Kper)
    b = make(G, kind, n, 5, Kper)
    G.ld_backward(a, 777, 100)
    st = G.ld_run(b, 777)
    assert torch.equal(a.x, b.x) and torch.equal(a.v, b.v)
    assert G.rng_get_state(a.rng) == G.rng_get_state(b.rng)
    r = G.ld_backward(make(G, kind, n, 5, Kper), 777, 100)
    assert math.isclose(r["loss"], st["energy_time_avg"], rel_tol=1e-6)


def test_adjoint_unbiased_at_scale(G):
    """N = 10^5, 10^4 steps, checkpoints every 100: the pathwise gradients
    summed over all oscillators equal the derivatives of the exactly computed
    E[L] (covariance recursion of the discrete scheme) within 5 standard
    errors estimated from the data.  The 10^5 oscillators run as 20
    independent systems of 5000 (own seeds): dL/dK uses the spread of the
    10^5 per-oscillator dL/dK_i, dL/dgamma and dL/dkT the spread of the 20
    system totals."""
    c = W.ADJOINT
    n, steps, B = c["n"], c["steps"], 20
    nb = n // B
    K, m, gamma, kT, dt = 1.0, 1.0, 0.5, 1.0, 0.01
    S0 = np.diag([kT / K, kT / m])

    def EL(k_, g_, t_, count):
        A = np.array([[1.0, dt], [-dt * k_ / m, 1 - g_ * dt / m]])
        Q = np.diag([0.0, 2 * g_ * t_ * dt / m**2])
        # the equilibrium start is drawn at the unperturbed K and kT
        Sig, tot = S0.copy(), 0.0
        for _ in range(steps):
            Sig = A @ Sig @ A.T + Q
            tot += 0.5 * m * Sig[1, 1] + 0.5 * k_ * Sig[0, 0]
        return 3 * count * tot / steps

    dks, dgs, dts, losses = [], [], [], []
    for b in range(B):
        s = make(G, "taus", nb, c["seed"] + 7919 * b, np.full(nb, K, np.float32), gamma=gamma,
                 kT=kT, dt=dt)
        r = G.ld_backward(s, steps, c["ckpt"])
        dks.append(r["dK"].cpu().numpy().astype(np.float64))
        dgs.append(r["dgamma"])
        dts.append(r["dkT"])
        losses.append(r["loss"])
    e = 1e-5
    d_K = (EL(K + e, gamma, kT, n) - EL(K - e, gamma, kT, n)) / (2 * e)
    d_kT = (EL(K, gamma, kT + e, n) - EL(K, gamma, kT - e, n)) / (2 * e)
    d_g = (EL(K, gamma + e, kT, n) - EL(K, gamma - e, kT, n)) / (2 * e)
    dK_all = np.concatenate(dks)
    se_K = dK_all.std(ddof=1) * math.sqrt(n)
    assert abs(dK_all.sum() - d_K) < 5 * se_K, (dK_all.sum(), d_K, se_K)
    for got, want in ((dts, d_kT), (dgs, d_g), (losses, EL(K, gamma, kT, n))):
        got = np.asarray(got)
        se = got.std(ddof=1) * math.sqrt(B)
        assert se > 0 and abs(got.sum() - want) < 5 * se, (got.sum(), want, se)


def test_autograd_function(G):
    """torch.autograd: gradients of the energy equal ld_backward's, and the
    caller's system is not advanced."""
    from paper_1003_1123_gb300.autograd import langevin_energy
    n = 300
    Kper = W.spring_constants(n, 9)
    s = make(G, "taus", n, 12, Kper)
    x_before = s.x.clone()
    K = torch.from_numpy(Kper).cuda().requires_grad_(True)
    gamma = torch.tensor(0.5, dtype=torch.float64, device="cuda", requires_grad=True)
    kT = torch.tensor(1.0, dtype=torch.float64, device="cuda", requires_grad=True)
    L = langevin_energy(s, 500, K, gamma, kT, ckpt_every=50)
    (2.0 * L).backward()
    assert torch.equal(s.x, x_before)
    ref = G.ld_backward(G.LdSystem(G.rng_clone(s.rng), s.x.clone(), s.v.clone(), K=1.0, m=1.0,
                                   gamma=0.5, kT=1.0, dt=0.01, K_per=K.detach().clone()), 500, 50)
    assert math.isclose(L.item(), ref["loss"], rel_tol=1e-6)
    assert torch.allclose(K.grad, 2 * ref["dK"], rtol=1e-6, atol=0)
    assert math.isclose(gamma.grad.item(), 2 * ref["dgamma"], rel_tol=1e-9)
    assert math.isclose(kT.grad.item(), 2 * ref["dkT"], rel_tol=1e-9)


@pytest.mark.parametrize("kind", ["taus", "ran2"])
@pytest.mark.parametrize("steps,ckpt", [(2000, 100), (1037, 64), (301, 7)])
def test_noise_history_equals_regeneration(G, kind, steps, ckpt):
    """The reverse sweep reading the noise stored by the forward run and the
    one regenerating it segment by segment give identical gradients, loss,
    final state and generator state, bit for bit."""
    n = 777
    Kper = W.spring_constants(n, 5, 0.5, 2.0)
    x0, v0 = W.initial_state(n, 19)
    out = []
    try:
        for limit in (0, 1 << 40):
            G.ld_set_adjoint_history_limit(limit)
            s = make(G, kind, n, 91, Kper, gamma=0.7, kT=1.3, start=(x0, v0))
            r = G.ld_backward(s, steps, ckpt)
            out.append((r["dK"].cpu().numpy().tobytes(), r["loss"], r["dgamma"], r["dkT"],
                        s.x.cpu().numpy().tobytes(), s.v.cpu().numpy().tobytes(),
                        G.rng_get_state(s.rng)))
    finally:
        G.ld_set_adjoint_history_limit(-1)
    assert out[0] == out[1]


def test_history_limit_rejects_bad_values(G):
    with pytest.raises(G.GbrngError):
        G.ld_set_adjoint_history_limit(-2)
    G.ld_set_adjoint_history_limit(-1)


def test_scratch_kept_by_the_handle_across_calls(G):
    """Successive ld_backward calls on one handle (the scratch grows, then is
    reused by smaller calls, on both noise paths) give what a fresh handle
    started from the same state gives."""
    n = 500
    Kper = W.spring_constants(n, 7, 0.5, 2.0)
    x0, v0 = W.initial_state(n, 23)
    s = make(G, "taus", n, 33, Kper, start=(x0, v0))
    try:
        for steps, ckpt, limit in ((200, 50, -1), (1200, 100, -1), (300, 30, 0), (90, 20, -1)):
            G.ld_set_adjoint_history_limit(limit)
            state = G.rng_get_state(s.rng)
            xs, vs = s.x.cpu().numpy().copy(), s.v.cpu().numpy().copy()
            r = G.ld_backward(s, steps, ckpt)
            f = make(G, "taus", n, 33, Kper, start=(xs, vs))
            G.rng_set_state(f.rng, state)
            rf = G.ld_backward(f, steps, ckpt)
            assert torch.equal(r["dK"], rf["dK"])
            assert (r["loss"], r["dgamma"], r["dkT"]) == (rf["loss"], rf["dgamma"], rf["dkT"])
            assert torch.equal(s.x, f.x) and torch.equal(s.v, f.v)
    finally:
        G.ld_set_adjoint_history_limit(-1)
