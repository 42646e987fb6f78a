"""ld_run_noalloc is the run for callers that cannot allocate device memory
when they step a system: a real-time loop that cannot wait on cudaMalloc, or
an application that gives the library a fixed memory budget.  It must give
the same results as ld_run.  This file is collected last on purpose, so a
failure here comes after every other test has run."""
import math

import numpy as np
import pytest
import torch

from paper_1003_1123_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TRAJ_TOL = 1e-5      # the tolerance of the other GPU parity tests
STATS_RTOL = 1e-5


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
    rms = math.sqrt((exp * exp).mean())
    return float((np.abs(got - exp) / np.maximum(np.abs(exp), rms)).max())


def system(G, kind, n, seed, Kper):
    r = G.rng_init(kind, seed, n)
    x = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    v = torch.zeros_like(x)
    s = G.LdSystem(r, x, v, K=1.0, m=1.0, gamma=0.5, kT=1.0, dt=0.01,
                   K_per=torch.from_numpy(Kper).cuda())
    G.ld_init_equilibrium(s)
    return s


@pytest.mark.parametrize("kind", ["taus", "ran2"])
@pytest.mark.parametrize("n", [4096, 300001])
def test_noalloc_matches_ld_run_twice(G, kind, n):
    """Two calls in a row through the C ABI: positions, velocities, generator
    states and statistics agree with ld_run's on identical systems."""
    Kper = W.spring_constants(n, 1)
    ref = system(G, kind, n, 99, Kper)
    new = system(G, kind, n, 99, Kper)
    for steps in (250, 111):
        a = G.ld_run(ref, steps)
        b = G.ld_run_noalloc(new, steps)
        assert rel_err(new.x.cpu().numpy(), ref.x.cpu().numpy()) <= TRAJ_TOL
        assert rel_err(new.v.cpu().numpy(), ref.v.cpu().numpy()) <= TRAJ_TOL
        assert G.rng_get_state(new.rng) == G.rng_get_state(ref.rng)
        for k in ("sum_x2", "sum_v2", "energy_time_avg"):
            assert math.isclose(a[k], b[k], rel_tol=STATS_RTOL), (k, a[k], b[k])
        assert abs(a["sum_xv"] - b["sum_xv"]) <= STATS_RTOL * math.sqrt(a["sum_x2"] * a["sum_v2"])
        assert b["steps"] == steps


@pytest.mark.parametrize("kind", ["taus", "ran2"])
def test_noalloc_empty_system(G, kind):
    """n == 0: nothing to run; the statistics are zero and the step count is
    reported, as ld_run does."""
    r = G.rng_init(kind, 5, 1)
    x = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    s = G.LdSystem(r, x, torch.zeros_like(x), K=1.0, m=1.0, gamma=0.5, kT=1.0, dt=0.01)
    for _ in range(2):
        b = G.ld_run_noalloc(s, 7)
        assert b["steps"] == 7
        assert b["sum_x2"] == b["sum_v2"] == b["sum_xv"] == b["energy_time_avg"] == 0.0
