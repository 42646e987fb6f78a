"""GPU parity of the fused Langevin-dynamics path against the CPU oracle,
through the C ABI: trajectories after 1000 steps within 1e-5 (relative to the
rms of the oracle's array), generator states bit-exact, statistics, run
splitting, the zero-noise closed form and equipartition."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1003_1123_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TRAJ_TOL = 1e-5      # max |gpu - oracle| / max(|oracle_i|, rms(oracle))
KINDS = ["taus", "ran2", "lagfib"]


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1003_1123_gb300 import gbrng
    gbrng.lib()
    return gbrng


def rel_err(got, exp):
    got = np.asarray(got, np.float64)
    exp = np.asarray(exp, np.float64)
    rms = math.sqrt((exp * exp).mean()) if exp.size else 1.0
    rms = rms or 1.0     # an all-zero expectation is compared absolutely
    return float((np.abs(got - exp) / np.maximum(np.abs(exp), rms)).max()) if exp.size else 0.0


def oracle_state_bytes(g):
    if g.kind == oracle.LAGFIB:
        return g.ring_in_order().tobytes()
    return g.state.tobytes()


def make_pair(G, kind, n, seed, K=1.0, m=1.0, gamma=0.5, kT=1.0, dt=0.01, Kper=None, streams=None):
    streams = streams or n
    r = G.rng_init(kind, seed, streams)
    x = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    v = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    kt = torch.from_numpy(Kper).cuda() if Kper is not None else None
    sysg = G.LdSystem(r, x, v, K=K, m=m, gamma=gamma, kT=kT, dt=dt, K_per=kt)
    g = oracle.Gen(kind, seed, streams)
    p = oracle.params(K=K, m=m, gamma=gamma, kT=kT, dt=dt)
    return sysg, g, p


@pytest.mark.parametrize("kind", KINDS)
def test_small_config_parity(G, kind):
    """Seed 1234, N = 4096, K = m = 1, gamma = 0.5, kT = 1, dt = 0.01, x, v from
    the equilibrium draw, 1000 steps: positions and velocities within 1e-5 of
    the binary32 oracle, generator state bit-exact, statistics within 1e-5."""
    c = W.SMALL
    s, g, p = make_pair(G, kind, c["n"], c["seed"])
    G.ld_init_equilibrium(s)
    x0, v0 = oracle.ld_init_eq_f32(g, c["n"], p)
    assert rel_err(s.x.cpu().numpy(), x0) < 1e-6 and rel_err(s.v.cpu().numpy(), v0) < 1e-6
    st = G.ld_run(s, c["steps"])
    ost = oracle.ld_run_f32(g, x0, v0, p, c["steps"])
    ex, ev = rel_err(s.x.cpu().numpy(), x0), rel_err(s.v.cpu().numpy(), v0)
    assert ex < TRAJ_TOL and ev < TRAJ_TOL, (ex, ev)
    assert G.parse_state(G.rng_get_state(s.rng))[1] == oracle_state_bytes(g)
    for k in ("sum_x2", "sum_v2", "energy_time_avg"):
        assert math.isclose(st[k], ost[k], rel_tol=1e-5), (k, st[k], ost[k])
    assert abs(st["sum_xv"] - ost["sum_xv"]) < 1e-5 * math.sqrt(ost["sum_x2"] * ost["sum_v2"])
    assert st["steps"] == c["steps"]
    # the FP64 oracle driven by the same integer streams, for the record
    g64 = oracle.Gen(kind, c["seed"], c["n"])
    xd, vd = oracle.ld_init_eq_f64(g64, c["n"], p)
    oracle.ld_run_f64(g64, xd, vd, p, c["steps"])
    assert rel_err(s.x.cpu().numpy(), xd) < 1e-4


@pytest.mark.parametrize("kind", KINDS)
def test_ragged_n_and_per_oscillator_K(G, kind):
    """An odd oscillator count, more streams than oscillators, K per
    oscillator, a start state from outside the library."""
    n = 1237
    Kper = W.spring_constants(n, 5)
    s, g, p = make_pair(G, kind, n, 8, gamma=0.9, kT=1.7, dt=0.02, Kper=Kper,
                        streams=n if kind == "lagfib" else n + 50)
    x0, v0 = W.initial_state(n, 6)
    s.x.copy_(torch.from_numpy(x0))
    s.v.copy_(torch.from_numpy(v0))
    G.ld_run(s, 257, stats=False)
    oracle.ld_run_f32(g, x0, v0, p, 257, Kper=Kper)
    assert rel_err(s.x.cpu().numpy(), x0) < TRAJ_TOL and rel_err(s.v.cpu().numpy(), v0) < TRAJ_TOL
    assert G.parse_state(G.rng_get_state(s.rng))[1] == oracle_state_bytes(g)


@pytest.mark.parametrize("kind", KINDS)
def test_run_splitting_bit_exact(G, kind):
    """ld_run(300) then ld_run(700) equals ld_run(1000) bit for bit."""
    n = 3000
    a, _, _ = make_pair(G, kind, n, 21)
    b, _, _ = make_pair(G, kind, n, 21)
    G.ld_init_equilibrium(a)
    G.ld_init_equilibrium(b)
    G.ld_run(a, 1000, stats=False)
    G.ld_run(b, 300, stats=False)
    G.ld_run(b, 700, stats=False)
    assert torch.equal(a.x, b.x) and torch.equal(a.v, b.v)
    assert G.rng_get_state(a.rng) == G.rng_get_state(b.rng)


@pytest.mark.parametrize("kind", KINDS)
def test_zero_noise_closed_form(G, kind):
    """kT = 0: the binary32 GPU trajectory follows A^n s0 (FP64 numpy)."""
    n, steps = 2000, 800
    K, m, gamma, dt = 1.3, 1.1, 0.3, 0.01
    s, _, _ = make_pair(G, kind, n, 2, K=K, m=m, gamma=gamma, kT=0.0, dt=dt)
    x0, v0 = W.initial_state(n, 3)
    s.x.copy_(torch.from_numpy(x0))
    s.v.copy_(torch.from_numpy(v0))
    G.ld_run(s, steps, stats=False)
    A = np.array([[1.0, dt], [-dt * K / m, 1 - gamma * dt / m]])
    An = np.linalg.matrix_power(A, steps)
    xe = An[0, 0] * x0.astype(np.float64) + An[0, 1] * v0
    ve = An[1, 0] * x0.astype(np.float64) + An[1, 1] * v0
    scale = max(np.abs(xe).max(), np.abs(ve).max())
    assert np.abs(s.x.cpu().numpy() - xe).max() < 5e-6 * scale
    assert np.abs(s.v.cpu().numpy() - ve).max() < 5e-6 * scale


@pytest.mark.parametrize("kind", KINDS + ["lcg"])
def test_zero_friction_is_noise_free(G, kind):
    """gamma = 0, a degenerate case of the Langevin equation (Sec. I): the
    random force's amplitude sqrt(2 gamma kT dt) is zero, so the trajectory is
    the deterministic Euler map whatever the draws -- bit-identical to the
    binary32 oracle and within binary32 rounding of A^n s0 (FP64) -- while
    the generator still advances by four draws a step."""
    n, steps = 1500, 600
    K, m, dt = 0.7, 1.3, 0.02
    s, g, p = make_pair(G, kind, n, 4, K=K, m=m, gamma=0.0, kT=2.0, dt=dt)
    x0, v0 = W.initial_state(n, 5)
    s.x.copy_(torch.from_numpy(x0))
    s.v.copy_(torch.from_numpy(v0))
    G.ld_run(s, steps, stats=False)
    xo, vo = x0.copy(), v0.copy()
    oracle.ld_run_f32(g, xo, vo, p, steps)
    assert np.array_equal(s.x.cpu().numpy(), xo) and np.array_equal(s.v.cpu().numpy(), vo)
    assert G.parse_state(G.rng_get_state(s.rng))[1] == oracle_state_bytes(g)
    A = np.array([[1.0, dt], [-dt * K / m, 1.0]])
    An = np.linalg.matrix_power(A, steps)
    xe = An[0, 0] * x0.astype(np.float64) + An[0, 1] * v0
    ve = An[1, 0] * x0.astype(np.float64) + An[1, 1] * v0
    scale = max(np.abs(xe).max(), np.abs(ve).max())
    assert np.abs(xo - xe).max() < 5e-6 * scale and np.abs(vo - ve).max() < 5e-6 * scale


@pytest.mark.parametrize("kind", KINDS)
def test_equipartition_large(G, kind):
    """N = 10^6 from the equilibrium draw, 2000 steps: <x^2>, <v^2> match the
    exactly propagated covariance of the discrete scheme within 3 sigma."""
    n, steps = 10**6, 2000
    K, m, gamma, kT, dt = 1.0, 1.0, 0.5, 1.0, 0.01
    s, _, _ = make_pair(G, kind, n, 31, K=K, m=m, gamma=gamma, kT=kT, dt=dt)
    G.ld_init_equilibrium(s)
    st = G.ld_run(s, steps)
    S = oracle.em_covariance(K, m, gamma, kT, dt, steps)
    cnt = 3 * n
    assert abs(st["sum_x2"] / cnt - S[0, 0]) < 3 * S[0, 0] * math.sqrt(2 / cnt)
    assert abs(st["sum_v2"] / cnt - S[1, 1]) < 3 * S[1, 1] * math.sqrt(2 / cnt)


@pytest.mark.parametrize("kind", ["taus", "ran2"])
def test_large_config_sampled_parity(G, kind):
    """N = 10^6 oscillators, 10^4 steps in one launch: 48 sampled oscillators
    recomputed by the oracle from their own streams match within 1e-5."""
    c = W.LARGE
    n, steps = c["n"], c["steps"]
    s, g, p = make_pair(G, kind, n, c["seed"])
    G.ld_init_equilibrium(s)
    x0 = s.x.cpu().numpy().copy()
    v0 = s.v.cpu().numpy().copy()
    state0 = g.state.copy()
    # advance the oracle streams past the two equilibrium draw-steps
    G.ld_run(s, steps, stats=False)
    picks = np.unique(np.concatenate([[0, 1, n - 1], np.random.default_rng(1).integers(0, n, 45)]))
    sub = oracle.Gen(kind, c["seed"], len(picks))
    sub.state[:] = state0[picks]
    xs, vs = oracle.ld_init_eq_f32(sub, len(picks), p)
    assert rel_err(xs, x0[picks]) < 1e-6
    oracle.ld_run_f32(sub, xs, vs, p, steps)
    ref = np.sqrt((xs.astype(np.float64) ** 2).mean())
    gx = s.x.cpu().numpy()[picks]
    assert np.abs(gx - xs).max() / max(ref, 1e-30) < TRAJ_TOL


def test_lagfib_large_n_parity(G):
    """N = 10^6 threads on the last Table I row, 60 steps (2.4e8 shared
    values, ~120 dependency rounds): full trajectories vs the oracle."""
    n, steps = 10**6, 60
    s, g, p = make_pair(G, "lagfib", n, 404)
    G.ld_init_equilibrium(s)
    x0, v0 = oracle.ld_init_eq_f32(g, n, p)
    st = G.ld_run(s, steps)
    ost = oracle.ld_run_f32(g, x0, v0, p, steps)
    assert rel_err(s.x.cpu().numpy(), x0) < TRAJ_TOL and rel_err(s.v.cpu().numpy(), v0) < TRAJ_TOL
    assert math.isclose(st["energy_time_avg"], ost["energy_time_avg"], rel_tol=1e-5)
    assert G.parse_state(G.rng_get_state(s.rng))[1] == oracle_state_bytes(g)


def test_lagfib_streamed_rounds_large_n(G):
    """N = 2.5e6 on the last Table I row (4N = 2.5 rounds a step, rounds
    straddling step boundaries, two rounds within N oscillator-steps so the
    x, v copies for the next round are issued before the barrier), per-
    oscillator K: full trajectories and generator state vs the oracle."""
    n = 2_500_001
    Kper = W.spring_constants(n, 9)
    r = G.rng_init("lagfib", 515, n)
    x = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    s = G.LdSystem(r, x, torch.zeros_like(x), K_per=torch.from_numpy(Kper).cuda())
    g = oracle.Gen("lagfib", 515, n)
    p = oracle.params()
    G.ld_init_equilibrium(s)
    xo, vo = oracle.ld_init_eq_f32(g, n, p, Kper=Kper)
    for steps in (1, 3):
        st = G.ld_run(s, steps)
        ost = oracle.ld_run_f32(g, xo, vo, p, steps, Kper=Kper)
        assert rel_err(s.x.cpu().numpy(), xo) < TRAJ_TOL and rel_err(s.v.cpu().numpy(), vo) < TRAJ_TOL
        assert math.isclose(st["energy_time_avg"], ost["energy_time_avg"], rel_tol=1e-5)
    assert G.parse_state(G.rng_get_state(s.rng))[1] == oracle_state_bytes(g)


@pytest.mark.parametrize("row,n,init", [
    (0, 200, True),      # 4N <= D: one round per step from position 0 on
    (3, 4096, True),     # D < 4N <= 2D, after the first ll positions: one round per step
    (3, 4096, False),    # same, but the run starts below ll with 4N > D
    (0, 1000, True),     # 4N > 2D: several rounds per step
    (2, 3001, True),     # ragged N, 4N between D and 2D
    (0, 4099, True),     # ~8 rounds a step: x, v copies for the next round cross the barrier
    (1, 2000, False),    # ~3 rounds a step from position 0, copies cross the barrier
])
def test_lagfib_rows_and_round_shapes(G, row, n, init):
    """The shared Lagged Fibonacci sequence drives the fused step for every
    relation of 4N to the lags (Sec. III.C requires ll - sl > 4N for its own
    one-step-per-launch scheme; here every relation is exact): trajectories
    within the tolerance, generator state bit-exact, per-oscillator K."""
    Kper = W.spring_constants(n, row)
    r = G.rng_init_lfg(11 + row, n, lag_row=row)
    x = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    v = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    s = G.LdSystem(r, x, v, K_per=torch.from_numpy(Kper).cuda())
    g = oracle.Gen("lagfib", 11 + row, n, lag_row=row)
    p = oracle.params()
    if init:
        G.ld_init_equilibrium(s)
        xo, vo = oracle.ld_init_eq_f32(g, n, p, Kper=Kper)
    else:
        xo = np.zeros((n, 3), np.float32)
        vo = np.zeros((n, 3), np.float32)
    for steps in (1, 99, 150):
        G.ld_run(s, steps)
        oracle.ld_run_f32(g, xo, vo, p, steps, Kper=Kper)
        assert G.parse_state(G.rng_get_state(s.rng))[1] == oracle_state_bytes(g)
        ex, ev = rel_err(s.x.cpu().numpy(), xo), rel_err(s.v.cpu().numpy(), vo)
        assert ex < TRAJ_TOL and ev < TRAJ_TOL, (steps, ex, ev)


def test_lagfib_timeout_reported_without_fault(G):
    """A chunk whose CTA never publishes (test hook: a flag nothing sets)
    makes every dependent wait run out after the limit; the kernel records
    GBRNG_ETIMEOUT and returns, and the context stays usable."""
    n = 10**5
    s, _, _ = make_pair(G, "lagfib", n, 5)
    G.rng_set_wait_limit_ns(200_000_000)
    G.gbrng_test_stall_chunk(3)
    try:
        with pytest.raises(G.GbrngError) as e:
            G.ld_run(s, 50, stats=False)
        assert e.value.code == -4
    finally:
        G.gbrng_test_stall_chunk(-1)
        G.rng_set_wait_limit_ns(2_000_000_000)
    torch.cuda.synchronize()
    r = G.rng_init("taus", 1, 10)
    assert G.rng_fill_u32(r, 100).numel() == 100
    r2 = G.rng_init("lagfib", 1, 100)
    assert G.rng_fill_u32(r2, 10**6).numel() == 10**6


@pytest.mark.parametrize("path", ["resident", "resident_dataflow", "fill", "fill_narrow_rounds", "ou"])
def test_lagfib_timeouts_on_every_cooperative_kernel(G, path):
    """The stall hook (one CTA never arrives at the grid barrier, or never
    publishes its steps to the CTAs that wait on it) ends the resident-state
    fused kernel in both of its synchronisation modes, the fill rounds (per-CTA
    waits where a round fills the grid, the grid barrier on Table I row 0's
    narrow rounds) and the overdamped run with GBRNG_ETIMEOUT after the wait
    limit; the context stays usable."""
    # 1e6 oscillators: one step a round, so the resident kernel waits per CTA
    n = 10**6 if path == "resident_dataflow" else 10**5
    r = G.rng_init("lagfib", 9, n)
    x = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    s = G.LdSystem(r, x, torch.zeros_like(x))
    G.ld_init_equilibrium(s)
    G.rng_fill_u32(r, 4 * 10**6)
    G.rng_set_wait_limit_ns(200_000_000)
    G.gbrng_test_stall_chunk(5)
    try:
        with pytest.raises(G.GbrngError) as e:
            if path.startswith("resident"):
                # a round holds up to 4 (ll - sl) / 4N = 20 steps of 1e5 oscillators
                G.ld_run(s, 100, stats=False)
            elif path == "fill":
                G.rng_fill_uniform(r, 32 * 10**6)
            elif path == "fill_narrow_rounds":
                G.rng_fill_uniform(G.rng_init_lfg(9, 1000, 0), 10**6)
            else:
                # 1e6 particles: two steps a round (2 (ll - sl) / 2N), so the
                # run takes a grid barrier every second step
                ro = G.rng_init("lagfib", 9, 10**6)
                G.ou_run(G.OuSystem(ro, torch.zeros(10**6, dtype=torch.float32, device="cuda")),
                         50, 10)
        assert e.value.code == -4
    finally:
        G.gbrng_test_stall_chunk(-1)
        G.rng_set_wait_limit_ns(2_000_000_000)
    torch.cuda.synchronize()
    r2 = G.rng_init("lagfib", 1, 100)
    assert G.rng_fill_u32(r2, 10**6).numel() == 10**6


def test_zero_steps_and_empty(G):
    s, _, _ = make_pair(G, "taus", 100, 1)
    G.ld_init_equilibrium(s)
    st = G.ld_run(s, 0)
    xx = (s.x.double() ** 2).sum().item()
    assert st["steps"] == 0 and math.isclose(st["sum_x2"], xx, rel_tol=1e-12)
    s2, _, _ = make_pair(G, "lagfib", 100, 1)
    G.ld_init_equilibrium(s2)
    st2 = G.ld_run(s2, 0)
    assert math.isclose(st2["sum_x2"], (s2.x.double() ** 2).sum().item(), rel_tol=1e-12)


@pytest.mark.parametrize("kind", ["taus", "ran2", "lagfib", "lcg"])
def test_runs_are_bit_reproducible(G, kind):
    """Two identical runs give identical trajectories, generator states and
    statistics (fixed-order reductions, no atomics in any sum)."""
    out = []
    for _ in range(2):
        r = G.rng_init(kind, 606, 3000)
        x = torch.zeros((3000, 3), dtype=torch.float32, device="cuda")
        s = G.LdSystem(r, x, torch.zeros_like(x))
        G.ld_init_equilibrium(s)
        st = G.ld_run(s, 250)
        out.append((s.x.cpu().numpy().tobytes(), s.v.cpu().numpy().tobytes(),
                    G.rng_get_state(r), st))
    assert out[0][:3] == out[1][:3]
    assert out[0][3] == out[1][3]


def test_allocation_failure_reports_enomem(G):
    """A generator larger than the device reports GBRNG_ENOMEM (no fault), and
    the context stays usable."""
    with pytest.raises(G.GbrngError) as e:
        G.rng_init("taus", 1, 2 * 10**10)      # 320 GB of state, more than the device holds
    assert e.value.code == -2
    r = G.rng_init("taus", 1, 100)
    assert G.rng_fill_u32(r, 1000).numel() == 1000


@pytest.mark.parametrize("kind,n", [("taus", 200_001), ("lcg", 200_001), ("ran2", 250_001)])
def test_two_oscillators_a_thread_odd_n(G, kind, n):
    """Odd N with enough oscillators for two a thread (Ran2's wave is larger:
    its tables and registers allow fewer warps a SM): the last pair has no
    second oscillator; full trajectories within the tolerance of the binary32
    oracle, generator states bit-exact, per-oscillator K."""
    steps = 60
    Kper = W.spring_constants(n, 41)
    s, g, p = make_pair(G, kind, n, 52, Kper=Kper)
    G.ld_init_equilibrium(s)
    xo, vo = oracle.ld_init_eq_f32(g, n, p, Kper=Kper)
    st = G.ld_run(s, steps)
    ost = oracle.ld_run_f32(g, xo, vo, p, steps, Kper=Kper)
    assert rel_err(s.x.cpu().numpy(), xo) < TRAJ_TOL and rel_err(s.v.cpu().numpy(), vo) < TRAJ_TOL
    assert math.isclose(st["energy_time_avg"], ost["energy_time_avg"], rel_tol=1e-5)
    assert math.isclose(st["sum_x2"], ost["sum_x2"], rel_tol=1e-5)
    assert G.parse_state(G.rng_get_state(s.rng))[1] == oracle_state_bytes(g)
