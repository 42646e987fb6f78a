"""GPU parity of the Quick and Dirty LCG (Eq. 1) and of the overdamped 1-D
run (Eq. 4-5) against the oracle, through the C ABI, and the paper's
Ornstein-Uhlenbeck test (Sec. IV) at its parameters with far fewer steps."""
import math

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1003_1123_gb300 import gbrng
    gbrng.lib()
    return gbrng


def rel(got, exp):
    got = np.asarray(got, np.float64)
    exp = np.asarray(exp, np.float64)
    rms = math.sqrt(float((exp * exp).mean())) or 1.0
    return float((np.abs(got - exp) / np.maximum(np.abs(exp), rms)).max())


@pytest.mark.parametrize("n,count", [(4096, 1 << 20), (1000, 123457), (7, 1001)])
def test_lcg_streams_bit_exact(G, n, count):
    r = G.rng_init("lcg", 77, n)
    got = G.rng_fill_u32(r, count).cpu().numpy().view(np.uint32)
    g = oracle.Gen("lcg", 77, n)
    assert np.array_equal(got, g.fill_u32(count))
    assert G.parse_state(G.rng_get_state(r))[1] == g.state.tobytes()
    u = G.rng_fill_uniform(r, 4096).cpu().numpy()
    assert np.array_equal(u, g.fill_uniform(4096))
    z = G.rng_fill_normal(r, 4096).cpu().numpy()
    zo = g.fill_normal(4096)
    assert np.all(np.abs(z - zo) <= 2e-6 * np.abs(zo) + 1e-7)


def test_lcg_fused_step_matches_oracle(G):
    n, steps = 2048, 500
    r = G.rng_init("lcg", 3, n)
    x = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    s = G.LdSystem(r, x, torch.zeros_like(x))
    G.ld_init_equilibrium(s)
    g = oracle.Gen("lcg", 3, n)
    p = oracle.params()
    xo, vo = oracle.ld_init_eq_f32(g, n, p)
    G.ld_run(s, steps)
    oracle.ld_run_f32(g, xo, vo, p, steps)
    assert rel(s.x.cpu().numpy(), xo) < 1e-5 and rel(s.v.cpu().numpy(), vo) < 1e-5
    assert G.parse_state(G.rng_get_state(r))[1] == g.state.tobytes()


def test_lcg_rejected_where_unsupported(G):
    r = G.rng_init("lcg", 1, 64)
    x = torch.zeros((64, 3), dtype=torch.float32, device="cuda")
    s = G.LdSystem(r, x, torch.zeros_like(x))
    for call in (lambda: G.ld_run_batched([s], 10), lambda: G.ld_backward(s, 10, 5),
                 lambda: G.ld_run_noalloc(s, 10)):
        with pytest.raises(G.GbrngError) as e:
            call()
        assert e.value.code == -1


@pytest.mark.parametrize("kind", ["taus", "ran2", "lcg", "lagfib"])
def test_ou_matches_oracle(G, kind):
    n, steps, every = 3001, 400, 50
    kw = dict(k_sp=1.5, xi=2.0, kT=1.0, dt=0.01)
    R0 = np.linspace(-3, 7, n).astype(np.float32)
    r = G.rng_init(kind, 21, n)
    R = torch.from_numpy(R0.copy()).cuda()
    s = G.OuSystem(r, R, **kw)
    mean, corr = G.ou_run(s, steps, every)
    g = oracle.Gen(kind, 21, n)
    Ro = R0.copy()
    mo, co = oracle.ou_run_f32(g, Ro, oracle.ou_params(**kw), steps, every)
    assert rel(R.cpu().numpy(), Ro) < 1e-5
    assert np.allclose(mean, mo, rtol=1e-5, atol=1e-5 * np.abs(Ro).max())
    assert np.allclose(corr, co, rtol=1e-5, atol=1e-5 * float((R0.astype(float) ** 2).mean()))
    if kind == "lagfib":
        assert G.parse_state(G.rng_get_state(r))[1] == g.ring_in_order().tobytes()
    else:
        assert G.parse_state(G.rng_get_state(r))[1] == g.state.tobytes()
    # continuing without records advances exactly as one longer run
    G.ou_run(s, 37)
    oracle.ou_run_f32(g, Ro, oracle.ou_params(**kw), 37, 37)
    assert rel(R.cpu().numpy(), Ro) < 1e-5


def test_ou_lagfib_several_steps_a_round(G):
    """Lagged Fibonacci overdamped run with three steps a round (Table I row 5,
    2 (ll - sl) = 42068 positions, 2N = 14000): 101 steps with a record every
    7, so rounds end between records and records fall inside rounds; values,
    records and the ring match the oracle."""
    n, steps, every = 7000, 101, 7
    kw = dict(k_sp=1.5, xi=2.0, kT=1.0, dt=0.01)
    R0 = np.linspace(-2, 5, n).astype(np.float32)
    r = G.rng_init_lfg(33, n, lag_row=5)
    R = torch.from_numpy(R0.copy()).cuda()
    mean, corr = G.ou_run(G.OuSystem(r, R, **kw), steps, every)
    g = oracle.Gen("lagfib", 33, n, lag_row=5)
    Ro = R0.copy()
    mo, co = oracle.ou_run_f32(g, Ro, oracle.ou_params(**kw), steps, every)
    assert rel(R.cpu().numpy(), Ro) < 1e-5
    assert np.allclose(mean, mo, rtol=1e-5, atol=1e-5 * np.abs(Ro).max())
    assert np.allclose(corr, co, rtol=1e-5, atol=1e-5 * float((R0.astype(float) ** 2).mean()))
    assert G.parse_state(G.rng_get_state(r))[1] == g.ring_in_order().tobytes()


def test_ou_lagfib_rejects_dependent_rounds(G):
    """A step of 2N positions must fit one round: 2N <= 4 (ll - sl) = 4116 on
    row 0 (the order-4 leap), so N = 2100 is refused."""
    r = G.rng_init_lfg(4, 2100, lag_row=0)
    s = G.OuSystem(r, torch.zeros(2100, dtype=torch.float32, device="cuda"))
    with pytest.raises(G.GbrngError) as e:
        G.ou_run(s, 10, 5)
    assert e.value.code == -5


# The paper's test (Sec. IV): N = 1e4, dt = 1 ps, R0 = 10 nm, k_sp = 0.01 pN/nm,
# T = 300 K, D = 0.25 nm^2/ns, so kT = 4.142 pN nm, xi = kT/D, tau = xi/k_sp =
# 1.66 us.  1e6 steps (0.6 tau) instead of 1e9.
KT = 1.380649e-23 * 300 * 1e21          # pN nm
PAPER = dict(k_sp=0.01, xi=KT / 0.25, kT=KT, dt=1e-3)   # ns
TAU = PAPER["xi"] / PAPER["k_sp"]


@pytest.mark.parametrize("kind", ["taus", "ran2", "lagfib"])
def test_ou_paper_relaxation_and_correlation(G, kind):
    n, steps, every = 10**4, 10**6, 10**5
    var_eq = PAPER["kT"] / PAPER["k_sp"]
    # <R(t)> from R0 = 10 nm against R0 exp(-t/tau)
    r = G.rng_init(kind, 5, n)
    s = G.OuSystem(r, torch.full((n,), 10.0, dtype=torch.float32, device="cuda"), **PAPER)
    mean, _ = G.ou_run(s, steps, every)
    for k, m in enumerate(mean):
        t = k * every * PAPER["dt"]
        sd = math.sqrt(var_eq * (1 - math.exp(-2 * t / TAU)) / n)
        assert abs(m - 10.0 * math.exp(-t / TAU)) <= 4 * sd + 1e-3, (k, m)
    # <R(t)R(0)> from an equilibrium start against (kT/k_sp) exp(-t/tau)
    R0 = np.random.default_rng(11).standard_normal(n) * math.sqrt(var_eq)
    r2 = G.rng_init(kind, 6, n)
    s2 = G.OuSystem(r2, torch.from_numpy(R0.astype(np.float32)).cuda(), **PAPER)
    _, corr = G.ou_run(s2, steps, every)
    for k, c in enumerate(corr):
        e = math.exp(-k * every * PAPER["dt"] / TAU)
        sd = var_eq * math.sqrt((1 + e * e) / n)
        assert abs(c - var_eq * e) <= 4 * sd, (k, c)


@pytest.mark.parametrize("kind", ["taus", "lagfib"])
def test_ou_edge_cases(G, kind):
    """Zero steps record only the entry state; every > n_steps gives one record;
    n_steps = 0 without records leaves R and the generator untouched; bad
    arguments are rejected before any work."""
    n = 300
    r = G.rng_init(kind, 2, n)
    R0 = torch.linspace(-1, 1, n, dtype=torch.float32, device="cuda")
    s = G.OuSystem(r, R0.clone())
    before = G.rng_get_state(r)
    mean, corr = G.ou_run(s, 0, 5)
    assert len(mean) == 1 and mean[0] == pytest.approx(float(R0.double().mean()), abs=1e-12)
    assert corr[0] == pytest.approx(float((R0.double() ** 2).mean()), rel=1e-12)
    assert G.rng_get_state(r) == before and torch.equal(s.R, R0)
    mean, corr = G.ou_run(s, 7, 100)
    assert len(mean) == 1
    with pytest.raises(G.GbrngError):
        G.ou_run(G.OuSystem(r, R0.clone(), k_sp=-1.0), 5, 1)
    with pytest.raises(G.GbrngError):
        G.ou_run(G.OuSystem(r, R0.clone(), dt=0.0), 5, 1)
    small = G.rng_init("taus", 2, 10)
    if kind == "taus":
        with pytest.raises(G.GbrngError):      # fewer streams than particles
            G.ou_run(G.OuSystem(small, R0.clone()), 5, 1)
