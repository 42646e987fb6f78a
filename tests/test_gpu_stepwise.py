"""The paper-form run (one launch per step, state through global memory)
against the persistent kernels and the oracle: x, v and generator states bit
for bit equal to ld_run's, statistics within 1e-5, the lag condition of the
one-step-per-launch scheme enforced for the Lagged Fibonacci generator."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1003_1123_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1003_1123_gb300 import gbrng
    gbrng.lib()
    return gbrng


def pair(G, kind, n, seed, row=None, kper=False):
    out = []
    for _ in range(2):
        r = G.rng_init_lfg(seed, n, lag_row=row) if row is not None else G.rng_init(kind, seed, n)
        x = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
        v = torch.zeros_like(x)
        kp = torch.from_numpy(W.spring_constants(n, seed)).cuda() if kper else None
        s = G.LdSystem(r, x, v, K_per=kp)
        G.ld_init_equilibrium(s)
        out.append(s)
    return out


@pytest.mark.parametrize("kind,n,row", [("taus", 5000, None), ("ran2", 3001, None), ("lcg", 999, None),
                                        ("lagfib", 4096, None), ("lagfib", 600, 3),
                                        ("lagfib", 100, 0)])
def test_stepwise_equals_persistent(G, kind, n, row):
    a, b = pair(G, kind, n, 31, row=row, kper=True)
    for steps in (1, 57, 200):
        sa = G.ld_run(a, steps)
        sb = G.ld_run_stepwise(b, steps)
        assert torch.equal(a.x, b.x) and torch.equal(a.v, b.v)
        assert G.rng_get_state(a.rng) == G.rng_get_state(b.rng)
        for k in ("sum_x2", "sum_v2", "sum_xv", "energy_time_avg"):
            assert math.isclose(sa[k], sb[k], rel_tol=1e-5, abs_tol=1e-9), (k, sa[k], sb[k])
        assert sb["steps"] == steps


def test_stepwise_matches_oracle(G):
    c = W.SMALL
    r = G.rng_init("taus", c["seed"], c["n"])
    x = torch.zeros((c["n"], 3), dtype=torch.float32, device="cuda")
    v = torch.zeros_like(x)
    s = G.LdSystem(r, x, v)
    G.ld_init_equilibrium(s)
    g = oracle.Gen("taus", c["seed"], c["n"])
    p = oracle.params()
    xo, vo = oracle.ld_init_eq_f32(g, c["n"], p)
    st = G.ld_run_stepwise(s, 300)
    ost = oracle.ld_run_f32(g, xo, vo, p, 300)
    rms = math.sqrt(float((xo.astype(np.float64) ** 2).mean()))
    assert np.abs(s.x.cpu().numpy() - xo).max() / rms < 1e-5
    assert math.isclose(st["energy_time_avg"], ost["energy_time_avg"], rel_tol=1e-5)


def test_stepwise_lagfib_rejects_dependent_steps(G):
    """Row 0 has ll - sl = 1029: 4N = 4800 > 4(ll - sl) cannot run one step per launch."""
    r = G.rng_init_lfg(5, 1200, lag_row=0)
    x = torch.zeros((1200, 3), dtype=torch.float32, device="cuda")
    s = G.LdSystem(r, x, torch.zeros_like(x))
    before = G.rng_get_state(r)
    with pytest.raises(G.GbrngError) as e:
        G.ld_run_stepwise(s, 10)
    assert e.value.code == -5
    assert G.rng_get_state(r) == before
    G.ld_run(s, 10)      # the round schedule of ld_run has no such limit
