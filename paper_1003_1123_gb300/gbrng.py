"""Python binding of the C ABI in include/gbrng.h (argument marshalling only).

Every function here has the name of the C entry point it calls.  Device
memory comes from torch tensors (their data pointers are passed through);
streams are torch's current CUDA stream unless one is given.  Every step of
the computation runs in libgbrng.so: there is no Python or CPU fallback, and
a missing library raises at import of the first call.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

from . import build as _build

TAUS, RAN2, LAGFIB, LCG = 0, 1, 2, 3
_KINDS = {"taus": TAUS, "ran2": RAN2, "lagfib": LAGFIB, "lfg": LAGFIB, "lcg": LCG}
_STATUS = {0: "GBRNG_OK", -1: "GBRNG_EINVAL", -2: "GBRNG_ENOMEM", -3: "GBRNG_ECUDA",
           -4: "GBRNG_ETIMEOUT", -5: "GBRNG_ELAGS", -6: "GBRNG_ESTATE"}

_lock = threading.Lock()
_lib = None


class GbrngError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


class LdSystemC(C.Structure):
    _fields_ = [("n", C.c_int64), ("x", C.c_void_p), ("v", C.c_void_p), ("K_per", C.c_void_p),
                ("K", C.c_double), ("m", C.c_double), ("gamma", C.c_double), ("kT", C.c_double),
                ("dt", C.c_double), ("rng", C.c_void_p)]


class OuSystemC(C.Structure):
    _fields_ = [("n", C.c_int64), ("R", C.c_void_p), ("k_sp", C.c_double), ("xi", C.c_double),
                ("kT", C.c_double), ("dt", C.c_double), ("rng", C.c_void_p)]


class LdStatsC(C.Structure):
    _fields_ = [("sum_x2", C.c_double), ("sum_v2", C.c_double), ("sum_xv", C.c_double),
                ("energy_time_avg", C.c_double), ("steps", C.c_int64)]


class StateHeaderC(C.Structure):
    _fields_ = [("magic", C.c_uint32), ("version", C.c_uint32), ("kind", C.c_int32),
                ("lag_row", C.c_int32), ("n_streams", C.c_int64), ("position", C.c_int64),
                ("payload_bytes", C.c_uint64)]


# Exported symbols and their argument types (also used by the ABI tests).
SIGNATURES = {
    "rng_init": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_uint64, C.c_int64, C.c_void_p]),
    "rng_init_lfg": (C.c_int, [C.POINTER(C.c_void_p), C.c_uint64, C.c_int64, C.c_int,
                               C.c_void_p]),
    "rng_destroy": (C.c_int, [C.c_void_p]),
    "rng_clone": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.c_void_p]),
    "rng_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int64),
                           C.POINTER(C.c_int), C.POINTER(C.c_int64)]),
    "rng_lfg_lags": (C.c_int, [C.c_int, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "rng_lfg_default_row": (C.c_int, [C.c_int64]),
    "rng_fill_u32": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "rng_fill_uniform": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "rng_fill_normal": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "rng_state_bytes": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    "rng_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "rng_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "rng_set_wait_limit_ns": (C.c_int, [C.c_uint64]),
    "gbrng_test_stall_chunk": (C.c_int, [C.c_int64]),
    "gbrng_set_lfg_order": (C.c_int, [C.c_int]),
    "ld_init_equilibrium": (C.c_int, [C.POINTER(LdSystemC), C.c_void_p]),
    "ld_run": (C.c_int, [C.POINTER(LdSystemC), C.c_int64, C.POINTER(LdStatsC), C.c_void_p]),
    "ld_run_stepwise": (C.c_int, [C.POINTER(LdSystemC), C.c_int64, C.POINTER(LdStatsC),
                                  C.c_void_p]),
    "ou_run": (C.c_int, [C.POINTER(OuSystemC), C.c_int64, C.c_int64, C.c_void_p, C.c_void_p,
                         C.c_void_p]),
    "ld_run_batched": (C.c_int, [C.POINTER(LdSystemC), C.c_int, C.c_int64,
                                 C.POINTER(C.c_int), C.POINTER(LdStatsC), C.c_void_p]),
    "ld_batched_tune": (C.c_int, [C.POINTER(LdSystemC), C.c_int, C.POINTER(C.c_int)]),
    "ld_backward": (C.c_int, [C.POINTER(LdSystemC), C.c_int64, C.c_int, C.c_void_p,
                              C.POINTER(C.c_double), C.POINTER(C.c_double),
                              C.POINTER(C.c_double), C.c_void_p]),
    "ld_run_noalloc": (C.c_int, [C.POINTER(LdSystemC), C.c_int64, C.POINTER(LdStatsC),
                                 C.c_void_p]),
    "ld_set_adjoint_history_limit": (C.c_int, [C.c_int64]),
    "gbrng_last_error": (C.c_char_p, []),
}


def library_path() -> str:
    return _build.LIB


def lib() -> C.CDLL:
    """Load libgbrng.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def gbrng_last_error() -> str:
    return lib().gbrng_last_error().decode(errors="replace")


def _check(rc: int):
    if rc != 0:
        raise GbrngError(rc, gbrng_last_error())


def _stream(stream):
    if stream is None:
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


# ----------------------------------------------------------------- handles
class Rng:
    """Owns one gbrng_t handle; destroyed with the object."""

    def __init__(self, handle: int, kind: int):
        self.handle = C.c_void_p(handle)
        self.kind = kind

    def __del__(self):
        if getattr(self, "handle", None) and self.handle.value and _lib is not None:
            _lib.rng_destroy(self.handle)
            self.handle = C.c_void_p(None)

    def info(self):
        return rng_info(self)


def rng_init(kind, seed: int, n_streams: int, stream=None) -> Rng:
    k = _KINDS[kind] if isinstance(kind, str) else int(kind)
    h = C.c_void_p()
    _check(lib().rng_init(C.byref(h), k, seed & (2**64 - 1), n_streams, _stream(stream)))
    return Rng(h.value, k)


def rng_init_lfg(seed: int, n_threads: int, lag_row: int = -1, stream=None) -> Rng:
    h = C.c_void_p()
    _check(lib().rng_init_lfg(C.byref(h), seed & (2**64 - 1), n_threads, lag_row,
                              _stream(stream)))
    return Rng(h.value, LAGFIB)


def rng_destroy(rng: Rng):
    if rng.handle.value:
        _check(lib().rng_destroy(rng.handle))
        rng.handle = C.c_void_p(None)


def rng_clone(rng: Rng, stream=None) -> Rng:
    h = C.c_void_p()
    _check(lib().rng_clone(rng.handle, C.byref(h), _stream(stream)))
    return Rng(h.value, rng.kind)


def rng_info(rng: Rng) -> dict:
    k, n, row, pos = C.c_int(), C.c_int64(), C.c_int(), C.c_int64()
    _check(lib().rng_info(rng.handle, C.byref(k), C.byref(n), C.byref(row), C.byref(pos)))
    return {"kind": k.value, "n_streams": n.value, "lag_row": row.value, "position": pos.value}


def rng_lfg_lags(row: int):
    sl, ll = C.c_int32(), C.c_int32()
    _check(lib().rng_lfg_lags(row, C.byref(sl), C.byref(ll)))
    return sl.value, ll.value


def rng_lfg_default_row(n_threads: int) -> int:
    r = lib().rng_lfg_default_row(n_threads)
    if r < 0:
        _check(r)
    return r


def _out(out, n, dtype, device):
    if out is None:
        out = torch.empty(n, dtype=dtype, device=device)
    assert out.is_cuda and out.is_contiguous() and out.dtype == dtype and out.numel() >= n
    return out


def rng_fill_u32(rng: Rng, n: int, out=None, stream=None, device="cuda"):
    """n raw draws; returned as an int32 tensor holding the uint32 bit patterns."""
    out = _out(out, n, torch.int32, device)
    _check(lib().rng_fill_u32(rng.handle, _ptr(out), n, _stream(stream)))
    return out


def rng_fill_uniform(rng: Rng, n: int, out=None, stream=None, device="cuda"):
    out = _out(out, n, torch.float32, device)
    _check(lib().rng_fill_uniform(rng.handle, _ptr(out), n, _stream(stream)))
    return out


def rng_fill_normal(rng: Rng, n: int, out=None, stream=None, device="cuda"):
    out = _out(out, n, torch.float32, device)
    _check(lib().rng_fill_normal(rng.handle, _ptr(out), n, _stream(stream)))
    return out


def rng_state_bytes(rng: Rng) -> int:
    b = C.c_size_t()
    _check(lib().rng_state_bytes(rng.handle, C.byref(b)))
    return b.value


def rng_get_state(rng: Rng) -> bytes:
    n = rng_state_bytes(rng)
    buf = C.create_string_buffer(n)
    _check(lib().rng_get_state(rng.handle, buf, n))
    return buf.raw


def rng_set_state(rng: Rng, blob: bytes):
    buf = C.create_string_buffer(bytes(blob), len(blob))
    _check(lib().rng_set_state(rng.handle, buf, len(blob)))


def rng_set_wait_limit_ns(ns: int):
    _check(lib().rng_set_wait_limit_ns(ns))


def ld_set_adjoint_history_limit(nbytes: int):
    """Largest noise history ld_backward keeps (bytes; 0 always regenerates,
    -1 half the free device memory)."""
    _check(lib().ld_set_adjoint_history_limit(nbytes))


def gbrng_set_lfg_order(k: int):
    """Leap order of every Lagged Fibonacci launch (1, 2 or 4; 0 = each
    launch's own choice).  Every order gives the same sequence."""
    _check(lib().gbrng_set_lfg_order(k))


def gbrng_test_stall_chunk(chunk: int):
    _check(lib().gbrng_test_stall_chunk(chunk))


def parse_state(blob: bytes):
    """Split a state blob into (header dict, payload bytes)."""
    h = StateHeaderC.from_buffer_copy(blob[:C.sizeof(StateHeaderC)])
    hd = {f: getattr(h, f) for f, _ in StateHeaderC._fields_}
    return hd, blob[C.sizeof(StateHeaderC):]


# -------------------------------------------------------- Langevin systems
class LdSystem:
    """One system of n 3-D oscillators: x, v are float32 [n, 3] CUDA tensors."""

    def __init__(self, rng: Rng, x: torch.Tensor, v: torch.Tensor, K=1.0, m=1.0, gamma=0.5,
                 kT=1.0, dt=0.01, K_per: torch.Tensor | None = None):
        for t in (x, v):
            assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
            assert t.dim() == 2 and t.shape[1] == 3
        assert x.shape == v.shape
        if K_per is not None:
            assert K_per.is_cuda and K_per.dtype == torch.float32 and K_per.is_contiguous()
            assert K_per.numel() == x.shape[0]
        self.rng, self.x, self.v, self.K_per = rng, x, v, K_per
        self.K, self.m, self.gamma, self.kT, self.dt = float(K), float(m), float(gamma), float(
            kT), float(dt)

    @property
    def n(self) -> int:
        return self.x.shape[0]

    def c_struct(self) -> LdSystemC:
        return LdSystemC(self.n, self.x.data_ptr(), self.v.data_ptr(),
                         self.K_per.data_ptr() if self.K_per is not None else None, self.K,
                         self.m, self.gamma, self.kT, self.dt, self.rng.handle.value)


def _stats(s: LdStatsC) -> dict:
    return {"sum_x2": s.sum_x2, "sum_v2": s.sum_v2, "sum_xv": s.sum_xv,
            "energy_time_avg": s.energy_time_avg, "steps": s.steps}


def ld_init_equilibrium(system: LdSystem, stream=None):
    cs = system.c_struct()
    _check(lib().ld_init_equilibrium(C.byref(cs), _stream(stream)))


def ld_run(system: LdSystem, n_steps: int, stats: bool = True, stream=None):
    cs = system.c_struct()
    st = LdStatsC()
    _check(lib().ld_run(C.byref(cs), n_steps, C.byref(st) if stats else None, _stream(stream)))
    return _stats(st) if stats else None


def ld_run_stepwise(system: LdSystem, n_steps: int, stats: bool = True, stream=None):
    """The paper form of ld_run: one kernel launch per step, state through
    global memory (same results as ld_run)."""
    cs = system.c_struct()
    st = LdStatsC()
    _check(lib().ld_run_stepwise(C.byref(cs), n_steps, C.byref(st) if stats else None,
                                 _stream(stream)))
    return _stats(st) if stats else None


def ld_run_noalloc(system: LdSystem, n_steps: int, stats: bool = True, stream=None):
    """ld_run without any device allocation (per-thread generators); see the C
    header for who needs it and what it shares."""
    cs = system.c_struct()
    st = LdStatsC()
    _check(lib().ld_run_noalloc(C.byref(cs), n_steps, C.byref(st) if stats else None,
                                _stream(stream)))
    return _stats(st) if stats else None


def ld_run_batched(systems, n_steps: int, tune=None, stats: bool = True, stream=None):
    arr = (LdSystemC * len(systems))(*[s.c_struct() for s in systems])
    out = (LdStatsC * len(systems))()
    tn = (C.c_int * 3)(*tune) if tune is not None else None
    _check(lib().ld_run_batched(arr, len(systems), n_steps, tn, out if stats else None,
                                _stream(stream)))
    return [_stats(s) for s in out] if stats else None


def ld_batched_tune(systems):
    """The autotuned (T, K, steps per launch) of these systems' shape."""
    arr = (LdSystemC * len(systems))(*[s.c_struct() for s in systems])
    out = (C.c_int * 3)()
    _check(lib().ld_batched_tune(arr, len(systems), out))
    return tuple(out)


def ld_backward(system: LdSystem, n_steps: int, ckpt_every: int = 100, dK: torch.Tensor = None,
                stream=None):
    """Returns dict(loss, dgamma, dkT, dK) (dK a float32 CUDA tensor [n])."""
    if dK is None:
        dK = torch.empty(system.n, dtype=torch.float32, device=system.x.device)
    cs = system.c_struct()
    dg, dk, loss = C.c_double(), C.c_double(), C.c_double()
    _check(lib().ld_backward(C.byref(cs), n_steps, ckpt_every, _ptr(dK), C.byref(dg),
                             C.byref(dk), C.byref(loss), _stream(stream)))
    return {"loss": loss.value, "dgamma": dg.value, "dkT": dk.value, "dK": dK}


# ------------------------------------------------------ overdamped 1-D runs
class OuSystem:
    """n 1-D particles (Eq. 4-5): R is a float32 [n] CUDA tensor."""

    def __init__(self, rng: Rng, R: torch.Tensor, k_sp=1.0, xi=1.0, kT=1.0, dt=0.01):
        assert R.is_cuda and R.dtype == torch.float32 and R.is_contiguous() and R.dim() == 1
        self.rng, self.R = rng, R
        self.k_sp, self.xi, self.kT, self.dt = float(k_sp), float(xi), float(kT), float(dt)

    def c_struct(self) -> OuSystemC:
        return OuSystemC(self.R.numel(), self.R.data_ptr(), self.k_sp, self.xi, self.kT, self.dt,
                         self.rng.handle)


def ou_run(system: OuSystem, n_steps: int, every: int = 0, stream=None):
    """Advance by n_steps; with every >= 1 returns (mean, corr) numpy arrays of
    n_steps // every + 1 records (<R(t)> and <R(t)R(0)>), else None."""
    import numpy as np
    cs = system.c_struct()
    if every:
        n_rec = n_steps // every + 1
        mean = np.zeros(n_rec, np.float64)
        corr = np.zeros(n_rec, np.float64)
        _check(lib().ou_run(C.byref(cs), n_steps, every, mean.ctypes.data, corr.ctypes.data,
                            _stream(stream)))
        return mean, corr
    _check(lib().ou_run(C.byref(cs), n_steps, 1, None, None, _stream(stream)))
    return None
