"""The large workload: 10^8 independent 3-D oscillators (x, v 2.4 GB; Ran2
state 14 GB), 1000 steps, K = gamma = kT = 1, dt = 0.01, for every generator.
Sampled oscillators of the per-thread generators are recomputed by the oracle
from their own streams; the shared Lagged Fibonacci sequence is compared with
the oracle on every oscillator over the run's first two steps (4e8 values of
the sequence, about 100 barrier rounds a step); every generator's ensemble
moments match the exactly propagated covariance of the discrete scheme within
3 sigma."""
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


@pytest.mark.parametrize("kind", ["taus", "ran2", "lagfib"])
def test_hundred_million_oscillators(G, kind):
    c = W.HUGE
    n, steps = c["n"], c["steps"]
    p = dict(K=c["K"], m=c["m"], gamma=c["gamma"], kT=c["kT"], dt=c["dt"])
    r = G.rng_init(kind, c["seed"], n)
    x = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    v = torch.zeros_like(x)
    s = G.LdSystem(r, x, v, **p)
    G.ld_init_equilibrium(s)
    picks = np.array([0, 1, 12345678, n // 2, n - 2, n - 1])
    if kind == "lagfib":
        # every oscillator over the first two steps, from the state the
        # equilibrium start left: the oracle continues the sequence from the
        # library's portable state (the last ll values, in order)
        hd, ring = G.parse_state(G.rng_get_state(r))
        sl, ll = G.rng_lfg_lags(hd["lag_row"])
        g = oracle.Gen.custom_lfg(c["seed"], sl, ll,
                                  ring=np.frombuffer(ring, dtype=np.uint32))
        xs, vs = x.cpu().numpy(), v.cpu().numpy()
        G.ld_run(s, 2, stats=False)
        oracle.ld_run_f32(g, xs, vs, oracle.params(**p), 2)
        for got, exp in ((x, xs), (v, vs)):
            exp64 = exp.astype(np.float64)
            rms = float(np.sqrt((exp64 * exp64).mean()))
            err = np.abs(got.cpu().numpy().astype(np.float64) - exp64) / np.maximum(
                np.abs(exp64), rms)
            assert float(err.max()) <= 1e-5
        assert G.parse_state(G.rng_get_state(r))[1] == g.ring_in_order().tobytes()
        del xs, vs, g
        steps -= 2
    st = G.ld_run(s, steps)
    if kind != "lagfib":
        # streams are counter-seeded: the oracle seeds just the sampled ones
        sub = oracle.Gen.streams(kind, c["seed"], picks)
        po = oracle.params(**p)
        xs, vs = oracle.ld_init_eq_f32(sub, len(picks), po)
        oracle.ld_run_f32(sub, xs, vs, po, steps)
        got = x[torch.as_tensor(picks, device="cuda")].cpu().numpy()
        ref = max(float(np.sqrt((xs.astype(np.float64) ** 2).mean())), 1e-30)
        assert np.abs(got - xs).max() / ref < 1e-5
    S = oracle.em_covariance(p["K"], p["m"], p["gamma"], p["kT"], p["dt"], steps)
    cnt = 3 * n
    assert abs(st["sum_x2"] / cnt - S[0, 0]) < 3 * S[0, 0] * math.sqrt(2 / cnt)
    assert abs(st["sum_v2"] / cnt - S[1, 1]) < 3 * S[1, 1] * math.sqrt(2 / cnt)
    sd_xv = math.sqrt((S[0, 0] * S[1, 1] + S[0, 1] ** 2) / cnt)
    assert abs(st["sum_xv"] / cnt - S[0, 1]) < 3 * sd_xv
