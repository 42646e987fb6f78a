"""The leap order of the Lagged Fibonacci schedule (Sec. III.C, Algorithm 3 in
the leap form x_p = sum_j C(k, j) x_{p - (k-j) ll - j (ll - sl)}) changes only
how many lag reads a value costs and how many positions a barrier round
holds: orders 1, 2 and 4 give the oracle's serial sequence bit for bit in the
fills, the fused step (general and resident-state kernels), the paper form
and the overdamped run, from a fresh seed and from a restored state (whose
backward extension to x_{p-K ll}, K the ring's highest order, is rebuilt on
the host)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1003_1123_gb300 import workloads as W

pytestmark = pytest.mark.gpu
ORDERS = [1, 2, 4]
TRAJ_TOL = 1e-5


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1003_1123_gb300 import gbrng
    gbrng.lib()
    yield gbrng
    gbrng.gbrng_set_lfg_order(0)


@pytest.fixture
def order(G, request):
    G.gbrng_set_lfg_order(request.param)
    yield request.param
    G.gbrng_set_lfg_order(0)


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def rel_err(got, exp):
    got = np.asarray(got, np.float64)
    exp = np.asarray(exp, np.float64)
    rms = float(np.sqrt((exp * exp).mean())) or 1.0
    return float((np.abs(got - exp) / np.maximum(np.abs(exp), rms)).max())


@pytest.mark.parametrize("order", ORDERS, indirect=True)
@pytest.mark.parametrize("row", [0, 2, 6, 9])
def test_fill_every_order(G, order, row):
    """Raw fills over many rounds and a ragged split, then a restored state
    continued by the same order."""
    sl, ll = oracle.lfg_table(row)
    n = min(5 * ll + 777, 3 * 10**6)
    r = G.rng_init_lfg(21 + row, 50, row)
    g = oracle.Gen("lagfib", 21 + row, 50, lag_row=row)
    a = n // 3 + 5
    got = np.concatenate([u32(G.rng_fill_u32(r, a)), u32(G.rng_fill_u32(r, n - a))])
    assert np.array_equal(got, g.fill_u32(n))
    blob = G.rng_get_state(r)
    assert G.parse_state(blob)[1] == g.ring_in_order().tobytes()
    r2 = G.rng_init_lfg(999, 50, row)
    G.rng_set_state(r2, blob)
    m = 2 * ll + 333
    assert np.array_equal(u32(G.rng_fill_u32(r2, m)), g.fill_u32(m))


@pytest.mark.parametrize("order", ORDERS, indirect=True)
@pytest.mark.parametrize("row,n", [(0, 200), (0, 1000), (3, 4096), (2, 3001), (9, 10**6)])
def test_fused_every_order(G, order, row, n):
    """The fused step (equilibrium start, then 1 and 37 steps) for several
    relations of 4N to the lags; at 10^6 oscillators order 4 takes the
    resident-state kernel with two steps a round."""
    Kper = W.spring_constants(n, 40 + row)
    r = G.rng_init_lfg(31 + row, n, lag_row=row)
    x = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    s = G.LdSystem(r, x, torch.zeros_like(x), K_per=torch.from_numpy(Kper).cuda())
    g = oracle.Gen("lagfib", 31 + row, n, lag_row=row)
    p = oracle.params()
    G.ld_init_equilibrium(s)
    xo, vo = oracle.ld_init_eq_f32(g, n, p, Kper=Kper)
    for steps in (1, 37):
        G.ld_run(s, steps)
        oracle.ld_run_f32(g, xo, vo, p, steps, Kper=Kper)
        assert G.parse_state(G.rng_get_state(r))[1] == g.ring_in_order().tobytes()
        assert rel_err(s.x.cpu().numpy(), xo) < TRAJ_TOL
        assert rel_err(s.v.cpu().numpy(), vo) < TRAJ_TOL


@pytest.mark.parametrize("order", ORDERS, indirect=True)
def test_paper_form_and_overdamped_every_order(G, order):
    """One launch per step and the overdamped run (one grid round a step),
    where the order bounds the largest N a step may hold."""
    row, n = 3, 1000
    r = G.rng_init_lfg(8, n, lag_row=row)
    x = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    s = G.LdSystem(r, x, torch.zeros_like(x))
    g = oracle.Gen("lagfib", 8, n, lag_row=row)
    p = oracle.params()
    G.ld_init_equilibrium(s)
    xo, vo = oracle.ld_init_eq_f32(g, n, p)
    G.ld_run_stepwise(s, 25)
    oracle.ld_run_f32(g, xo, vo, p, 25)
    assert rel_err(s.x.cpu().numpy(), xo) < TRAJ_TOL
    assert G.parse_state(G.rng_get_state(r))[1] == g.ring_in_order().tobytes()
    R = torch.full((n,), 10.0, dtype=torch.float32, device="cuda")
    ou = G.OuSystem(r, R, k_sp=0.01, xi=1.0, kT=4.1, dt=1.0)
    G.ou_run(ou, 40, every=10)
    Ro = np.full(n, 10.0, np.float32)
    oracle.ou_run_f32(g, Ro, oracle.ou_params(k_sp=0.01, xi=1.0, kT=4.1, dt=1.0), 40, 10)
    assert rel_err(R.cpu().numpy(), Ro) < TRAJ_TOL
    assert G.parse_state(G.rng_get_state(r))[1] == g.ring_in_order().tobytes()


def test_order_setting_rejects_other_values(G):
    for bad in (3, 5, -1):
        with pytest.raises(G.GbrngError) as e:
            G.gbrng_set_lfg_order(bad)
        assert e.value.code == -1
    G.gbrng_set_lfg_order(0)


def test_state_blob_moves_between_ring_orders(G):
    """A state blob holds the last ll values only, so it moves between a
    handle whose ring serves order 4 and one that serves order 2 (each rebuilds
    its own backward extension); both continue the oracle's sequence."""
    row, n = 5, 300
    sl, ll = oracle.lfg_table(row)
    g = oracle.Gen("lagfib", 61, n, lag_row=row)
    try:
        G.gbrng_set_lfg_order(4)
        r4 = G.rng_init_lfg(61, n, row)
        a = 3 * ll + 11
        assert np.array_equal(u32(G.rng_fill_u32(r4, a)), g.fill_u32(a))   # order 4
        G.gbrng_set_lfg_order(0)
        r2 = G.rng_init_lfg(62, n, row)
        G.rng_set_state(r2, G.rng_get_state(r4))
        b = 4 * ll + 5
        assert np.array_equal(u32(G.rng_fill_u32(r2, b)), g.fill_u32(b))
        G.gbrng_set_lfg_order(4)
        G.rng_set_state(r4, G.rng_get_state(r2))
        assert np.array_equal(u32(G.rng_fill_u32(r4, b)), g.fill_u32(b))
    finally:
        G.gbrng_set_lfg_order(0)
