"""Seeded synthetic workloads shaped like the paper's tests (Sec. IV: N
independent 3-D harmonic oscillators in a thermostat, 10^3-10^4 steps).

This module only draws workload parameters with numpy's PCG64; it contains
none of the method's arithmetic and is shared by the tests, the oracle legs
and the GPU runs.
"""
from __future__ import annotations

import numpy as np

# Parity configuration: Hybrid Taus, seed 1234, 4096 oscillators, 1000 steps,
# plus the raw 2^20-number stream of the same generator.
SMALL = dict(seed=1234, n=4096, K=1.0, m=1.0, gamma=0.5, kT=1.0, dt=0.01, steps=1000,
             raw_n=2**20)

# Throughput configuration: 10^6 oscillators, 10^4 fused steps per generator,
# fills of 2^30 numbers.
LARGE = dict(seed=2024, n=10**6, K=1.0, m=1.0, gamma=0.5, kT=1.0, dt=0.01, steps=10**4,
             fill_n=2**30)

# Differentiation: 10^5 oscillators, per-oscillator K = 1, 10^4 steps,
# checkpoints every 100 steps; FP64 comparison at 256 oscillators.
ADJOINT = dict(seed=77, n=10**5, K=1.0, m=1.0, gamma=0.5, kT=1.0, dt=0.01, steps=10**4,
               ckpt=100, n_check=256)

# Large system: 10^8 oscillators, 1000 steps.
HUGE = dict(seed=99, n=10**8, K=1.0, m=1.0, gamma=1.0, kT=1.0, dt=0.01, steps=1000)


def batched_systems(n_sys: int = 512, seed: int = 1234, n_lo: float = 1e2, n_hi: float = 1e5):
    """Parameters of independent systems: N log-uniform in [n_lo, n_hi],
    K log-uniform in [0.1, 10], gamma uniform in [0.1, 2], kT uniform in
    [0.5, 2], dt = 0.005, one generator seed per system."""
    rng = np.random.default_rng(seed)
    n = np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), n_sys)).astype(np.int64)
    K = np.exp(rng.uniform(np.log(0.1), np.log(10.0), n_sys))
    gamma = rng.uniform(0.1, 2.0, n_sys)
    kT = rng.uniform(0.5, 2.0, n_sys)
    seeds = rng.integers(0, 2**63, n_sys, dtype=np.int64)
    return [dict(n=int(n[i]), K=float(K[i]), m=1.0, gamma=float(gamma[i]), kT=float(kT[i]),
                 dt=0.005, seed=int(seeds[i])) for i in range(n_sys)]


def spring_constants(n: int, seed: int, lo: float = 0.5, hi: float = 2.0) -> np.ndarray:
    """Per-oscillator spring constants, uniform in [lo, hi] (float32)."""
    return np.random.default_rng(seed).uniform(lo, hi, n).astype(np.float32)


def initial_state(n: int, seed: int, scale_x: float = 1.0, scale_v: float = 1.0):
    """Gaussian positions and velocities (float32 [n, 3]) for tests that start
    from a given state instead of the equilibrium draw."""
    r = np.random.default_rng(seed)
    x = (r.standard_normal((n, 3)) * scale_x).astype(np.float32)
    v = (r.standard_normal((n, 3)) * scale_v).astype(np.float32)
    return x, v
