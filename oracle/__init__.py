"""CPU oracle for the on-the-fly RNG + Langevin-dynamics hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  It shares no code with the CUDA library: the arithmetic lives
in ``gbrng_oracle.c`` (plain serial C, built with ``-ffp-contract=off``), and
this module only marshals numpy arrays into it.

Every function follows the paper it cites in ``gbrng_oracle.c``:
Algorithm 1 (Hybrid Taus), Algorithm 2 (Ran2), Algorithm 3 and Table I
(additive Lagged Fibonacci), the Box-Muller transform (Sec. II.A), the
Euler-Maruyama Langevin step (Sec. I and Eq. 5) and its reverse-time adjoint.
``em_covariance`` propagates the exact covariance of the discrete scheme.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gbrng_oracle.c")
_HDR = os.path.join(_HERE, "gbrng_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

TAUS, RAN2, LAGFIB, LCG = 0, 1, 2, 3
KIND_NAMES = {"taus": TAUS, "ran2": RAN2, "lagfib": LAGFIB, "lfg": LAGFIB, "lcg": LCG}


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (plain gcc, no GPU)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class _OuParams(C.Structure):
    _fields_ = [("k_sp", C.c_double), ("xi", C.c_double), ("kT", C.c_double), ("dt", C.c_double)]


class _Gen(C.Structure):
    _fields_ = [("kind", C.c_int32), ("ll", C.c_int32), ("sl", C.c_int32),
                ("n_streams", C.c_int64), ("pos", C.c_int64), ("state", C.c_void_p)]


class _Params(C.Structure):
    _fields_ = [("K", C.c_double), ("m", C.c_double), ("gamma", C.c_double),
                ("kT", C.c_double), ("dt", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            u64, i64, i32, u32 = C.c_uint64, C.c_int64, C.c_int32, C.c_uint32
            vp, dp, fp = C.c_void_p, C.POINTER(C.c_double), C.c_void_p
            G = C.POINTER(_Gen)
            sig = {
                "or_splitmix64": (u64, [u64, u64]),
                "or_taus_seed": (None, [u64, i64, vp]),
                "or_ran2_seed": (None, [u64, i64, vp]),
                "or_lfg_seed": (None, [u64, i32, vp]),
                "or_lcg_seed": (None, [u64, i64, vp]),
                "or_lcg_next": (u32, [vp]),
                "or_ou_run_f32": (C.c_int, [G, i64, _OuParams, vp, i64, i64, vp, vp]),
                "or_seed_streams": (None, [C.c_int, u64, vp, i64, vp]),
                "or_lfg_table": (C.c_int, [C.c_int, C.POINTER(i32), C.POINTER(i32)]),
                "or_lfg_default_row": (C.c_int, [i64]),
                "or_taus_next": (u32, [vp]),
                "or_taus_component": (u32, [u32, C.c_int]),
                "or_ran2_schrage": (i32, [i32, C.c_int]),
                "or_ran2_next": (i32, [vp]),
                "or_lfg_next": (u32, [G]),
                "or_u01_f32": (C.c_float, [u32]),
                "or_open01": (C.c_double, [u32]),
                "or_ran2_u01_f32": (C.c_float, [i32]),
                "or_ran2_u01_f64": (C.c_double, [i32]),
                "or_box_muller_f32": (None, [C.c_float, C.c_float, C.POINTER(C.c_float),
                                             C.POINTER(C.c_float)]),
                "or_box_muller_f64": (None, [C.c_double, C.c_double, dp, dp]),
                "or_fill_u32": (C.c_int, [G, i64, vp]),
                "or_fill_uniform": (C.c_int, [G, i64, vp]),
                "or_fill_normal": (C.c_int, [G, i64, vp]),
                "or_ld_init_eq_f32": (C.c_int, [G, i64, fp, _Params, vp, vp]),
                "or_ld_run_f32": (C.c_int, [G, i64, fp, _Params, vp, vp, i64, vp]),
                "or_ld_init_eq_f64": (C.c_int, [G, i64, fp, _Params, vp, vp]),
                "or_ld_run_f64": (C.c_int, [G, i64, fp, _Params, vp, vp, i64, vp, vp]),
                "or_ld_adjoint_f64": (C.c_int, [G, i64, fp, _Params, vp, vp, i64, vp, vp,
                                                dp, dp]),
                "or_taus_component_period": (u64, [C.c_int, u32]),
                "or_lcg_period": (u64, [u32]),
                "or_gf2_trinomial_irreducible": (C.c_int, [i32, i32]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------- generators
def lfg_table(row: int):
    sl, ll = C.c_int32(), C.c_int32()
    if lib().or_lfg_table(row, C.byref(sl), C.byref(ll)) != 0:
        raise ValueError(f"no Table I row {row}")
    return sl.value, ll.value


def lfg_default_row(n_threads: int) -> int:
    return lib().or_lfg_default_row(n_threads)


class Gen:
    """A generator bundle: ``n`` independent streams (Taus, Ran2) or the one
    shared Lagged Fibonacci sequence used by ``n`` threads per step."""

    def __init__(self, kind, seed: int, n: int, lag_row: int | None = None):
        self.kind = KIND_NAMES[kind] if isinstance(kind, str) else int(kind)
        self.seed = int(seed)
        self.n = int(n)
        L = lib()
        g = _Gen()
        g.kind, g.n_streams, g.pos = self.kind, self.n, 0
        if self.kind == TAUS:
            self.state = np.zeros((self.n, 4), np.uint32)
            L.or_taus_seed(self.seed, self.n, _ptr(self.state))
        elif self.kind == RAN2:
            self.state = np.zeros((self.n, 35), np.int32)
            L.or_ran2_seed(self.seed, self.n, _ptr(self.state))
        elif self.kind == LCG:
            self.state = np.zeros(self.n, np.uint32)
            L.or_lcg_seed(self.seed, self.n, _ptr(self.state))
        else:
            self.row = lfg_default_row(self.n) if lag_row is None or lag_row < 0 else lag_row
            sl, ll = lfg_table(self.row)
            g.sl, g.ll = sl, ll
            self.state = np.zeros(ll, np.uint32)
            L.or_lfg_seed(self.seed, ll, _ptr(self.state))
        g.state = self.state.ctypes.data
        self._g = g

    @classmethod
    def custom_lfg(cls, seed: int, sl: int, ll: int, ring=None) -> "Gen":
        """Lagged Fibonacci with arbitrary lags (tiny-lag pins); ring word w holds
        x_{w-ll}.  Seeds as the Table I rows do unless ``ring`` is given."""
        g = cls.__new__(cls)
        g.kind, g.seed, g.n, g.row = LAGFIB, int(seed), 1, -1
        if ring is None:
            g.state = np.zeros(ll, np.uint32)
            lib().or_lfg_seed(g.seed, ll, _ptr(g.state))
        else:
            g.state = np.ascontiguousarray(ring, dtype=np.uint32).copy()
        s = _Gen()
        s.kind, s.sl, s.ll, s.n_streams, s.pos = LAGFIB, sl, ll, 1, 0
        s.state = g.state.ctypes.data
        g._g = s
        return g

    @classmethod
    def streams(cls, kind, seed: int, indices) -> "Gen":
        """Per-thread generator holding only the streams with the given indices
        of a larger generator (stream s is seeded from counters 8s + k)."""
        k = KIND_NAMES[kind] if isinstance(kind, str) else int(kind)
        idx = np.ascontiguousarray(indices, dtype=np.int64)
        g = cls.__new__(cls)
        g.kind, g.seed, g.n = k, int(seed), len(idx)
        if k == LCG:
            g.state = np.zeros(len(idx), np.uint32)
        else:
            g.state = np.zeros((len(idx), 4 if k == TAUS else 35),
                               np.uint32 if k == TAUS else np.int32)
        lib().or_seed_streams(k, g.seed, _ptr(idx), len(idx), _ptr(g.state))
        s = _Gen()
        s.kind, s.n_streams, s.pos = k, len(idx), 0
        s.state = g.state.ctypes.data
        g._g = s
        return g

    @property
    def ref(self):
        return C.byref(self._g)

    @property
    def pos(self) -> int:
        return self._g.pos

    @property
    def lags(self):
        return self._g.sl, self._g.ll

    def ring_in_order(self) -> np.ndarray:
        """Lagged Fibonacci: the last ll values x_{pos-ll} .. x_{pos-1}."""
        ll, p = self._g.ll, self._g.pos
        idx = (np.arange(p - ll, p, dtype=np.int64)) % ll
        return self.state[idx].copy()

    def copy(self) -> "Gen":
        other = Gen.__new__(Gen)
        other.kind, other.seed, other.n = self.kind, self.seed, self.n
        if hasattr(self, "row"):
            other.row = self.row
        other.state = self.state.copy()
        g = _Gen()
        g.kind, g.ll, g.sl = self._g.kind, self._g.ll, self._g.sl
        g.n_streams, g.pos = self._g.n_streams, self._g.pos
        g.state = other.state.ctypes.data
        other._g = g
        return other

    # ---- fills
    def fill_u32(self, n: int) -> np.ndarray:
        out = np.zeros(n, np.uint32)
        assert lib().or_fill_u32(self.ref, n, _ptr(out)) == 0
        return out

    def fill_uniform(self, n: int) -> np.ndarray:
        out = np.zeros(n, np.float32)
        assert lib().or_fill_uniform(self.ref, n, _ptr(out)) == 0
        return out

    def fill_normal(self, n: int) -> np.ndarray:
        out = np.zeros(n, np.float32)
        if lib().or_fill_normal(self.ref, n, _ptr(out)) != 0:
            raise ValueError("n must be even and non-negative")
        return out


def splitmix64(seed: int, idx: int) -> int:
    return lib().or_splitmix64(seed, idx)


def taus_next(y: np.ndarray) -> int:
    assert y.dtype == np.uint32 and y.shape == (4,) and y.flags.c_contiguous
    return lib().or_taus_next(_ptr(y))


def taus_component(y: int, which: int) -> int:
    return lib().or_taus_component(y, which)


def ran2_schrage(x: int, which: int) -> int:
    return lib().or_ran2_schrage(x, which)


def ran2_next(st: np.ndarray) -> int:
    assert st.dtype == np.int32 and st.shape == (35,) and st.flags.c_contiguous
    return lib().or_ran2_next(_ptr(st))


def u01_f32(raw: int) -> float:
    return lib().or_u01_f32(raw)


def open01(raw: int) -> float:
    return lib().or_open01(raw)


def ran2_u01_f32(iy: int) -> float:
    return lib().or_ran2_u01_f32(iy)


def box_muller_f32(u1: float, u2: float):
    a, b = C.c_float(), C.c_float()
    lib().or_box_muller_f32(u1, u2, C.byref(a), C.byref(b))
    return a.value, b.value


def box_muller_f64(u1: float, u2: float):
    a, b = C.c_double(), C.c_double()
    lib().or_box_muller_f64(u1, u2, C.byref(a), C.byref(b))
    return a.value, b.value


# --------------------------------------------------------- Langevin dynamics
def params(K=1.0, m=1.0, gamma=0.5, kT=1.0, dt=0.01) -> _Params:
    return _Params(float(K), float(m), float(gamma), float(kT), float(dt))


def _kper(Kper, dtype):
    if Kper is None:
        return None
    return np.ascontiguousarray(Kper, dtype=dtype)


def ld_init_eq_f32(gen: Gen, n: int, p: _Params, Kper=None):
    x = np.zeros((n, 3), np.float32)
    v = np.zeros((n, 3), np.float32)
    k = _kper(Kper, np.float32)
    assert lib().or_ld_init_eq_f32(gen.ref, n, _ptr(k), p, _ptr(x), _ptr(v)) == 0
    return x, v


def ld_run_f32(gen: Gen, x: np.ndarray, v: np.ndarray, p: _Params, n_steps: int, Kper=None):
    """Advance x, v (float32 [n,3], in place) by n_steps; returns the stats
    dict (sum_x2, sum_v2, sum_xv, energy_time_avg, steps)."""
    assert x.dtype == np.float32 and v.dtype == np.float32
    assert x.flags.c_contiguous and v.flags.c_contiguous
    st = np.zeros(5, np.float64)
    k = _kper(Kper, np.float32)
    assert lib().or_ld_run_f32(gen.ref, x.shape[0], _ptr(k), p, _ptr(x), _ptr(v), n_steps,
                               _ptr(st)) == 0
    return _stats(st)


def ld_init_eq_f64(gen: Gen, n: int, p: _Params, Kper=None):
    x = np.zeros((n, 3), np.float64)
    v = np.zeros((n, 3), np.float64)
    k = _kper(Kper, np.float64)
    assert lib().or_ld_init_eq_f64(gen.ref, n, _ptr(k), p, _ptr(x), _ptr(v)) == 0
    return x, v


def ld_run_f64(gen: Gen, x: np.ndarray, v: np.ndarray, p: _Params, n_steps: int, Kper=None,
               per_osc: bool = False):
    assert x.dtype == np.float64 and v.dtype == np.float64
    st = np.zeros(5, np.float64)
    lp = np.zeros(x.shape[0], np.float64) if per_osc else None
    k = _kper(Kper, np.float64)
    assert lib().or_ld_run_f64(gen.ref, x.shape[0], _ptr(k), p, _ptr(x), _ptr(v), n_steps,
                               _ptr(st), _ptr(lp)) == 0
    out = _stats(st)
    if per_osc:
        out["loss_per_osc"] = lp
    return out


def ld_adjoint_f64(gen: Gen, x: np.ndarray, v: np.ndarray, p: _Params, n_steps: int,
                   Kper=None):
    """Reverse-time adjoint (FP64).  Returns dict with loss (sum of the
    per-oscillator time-averaged energies), loss_per_osc, dK, dgamma, dkT;
    x and v are advanced in place."""
    n = x.shape[0]
    lp = np.zeros(n, np.float64)
    dK = np.zeros(n, np.float64)
    dg, dk = C.c_double(), C.c_double()
    k = _kper(Kper, np.float64)
    rc = lib().or_ld_adjoint_f64(gen.ref, n, _ptr(k), p, _ptr(x), _ptr(v), n_steps, _ptr(lp),
                                 _ptr(dK), C.byref(dg), C.byref(dk))
    if rc != 0:
        raise ValueError(f"or_ld_adjoint_f64 failed ({rc})")
    return {"loss": float(lp.sum()), "loss_per_osc": lp, "dK": dK, "dgamma": dg.value,
            "dkT": dk.value}


def _stats(st):
    return {"sum_x2": st[0], "sum_v2": st[1], "sum_xv": st[2], "energy_time_avg": st[3],
            "steps": int(st[4])}


def em_covariance(K, m, gamma, kT, dt, n_steps, sigma0=None):
    """Exact covariance of one component of the discrete Euler-Maruyama scheme:
    Sigma_{t+1} = A Sigma_t A^T + Q with A = [[1, dt], [-dt K/m, 1 - gamma dt/m]]
    and Q = diag(0, 2 gamma kT dt / m^2), from Sigma_0 (default the continuous
    equilibrium diag(kT/K, kT/m)).  Returns the 2x2 matrix after n_steps."""
    A = np.array([[1.0, dt], [-dt * K / m, 1.0 - gamma * dt / m]])
    Q = np.array([[0.0, 0.0], [0.0, 2.0 * gamma * kT * dt / m ** 2]])
    S = np.diag([kT / K, kT / m]) if sigma0 is None else np.array(sigma0, float)
    for _ in range(int(n_steps)):
        S = A @ S @ A.T + Q
    return S


# --------------------------------------------------------------------- pins
def taus_component_period(which: int, seed: int) -> int:
    return lib().or_taus_component_period(which, seed)


def lcg_period(seed: int) -> int:
    return lib().or_lcg_period(seed)


def gf2_trinomial_irreducible(ll: int, k: int) -> bool:
    r = lib().or_gf2_trinomial_irreducible(ll, k)
    if r < 0:
        raise ValueError("bad trinomial")
    return bool(r)


# ------------------------------------------------------- overdamped 1-D run
def ou_params(k_sp=1.0, xi=1.0, kT=1.0, dt=0.01) -> _OuParams:
    return _OuParams(float(k_sp), float(xi), float(kT), float(dt))


def ou_run_f32(gen: Gen, R: np.ndarray, p: _OuParams, n_steps: int, every: int):
    """Advance the float32 positions R (in place) by n_steps of Eq. 5; returns
    (mean, corr) at records r = 0 .. n_steps // every (after r * every steps)."""
    assert R.dtype == np.float32 and R.flags.c_contiguous
    n_rec = n_steps // every + 1
    mean = np.zeros(n_rec, np.float64)
    corr = np.zeros(n_rec, np.float64)
    assert lib().or_ou_run_f32(gen.ref, len(R), p, _ptr(R), n_steps, every, _ptr(mean),
                               _ptr(corr)) == 0
    return mean, corr


def lcg_next(x: np.ndarray) -> int:
    """One step of the Quick and Dirty LCG on x (uint32[1], in place)."""
    return lib().or_lcg_next(_ptr(x))
