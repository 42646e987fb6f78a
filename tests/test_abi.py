"""The C ABI library builds, loads and exports every entry point that
include/gbrng.h declares; host-only entry points (Table I, argument checks)
behave as documented.  No GPU is touched."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbrng.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\([^;]*\)\s*;", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def G():
    from paper_1003_1123_gb300 import gbrng
    gbrng.lib()
    return gbrng


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["rng_init", "rng_fill_uniform", "rng_fill_normal", "ld_run", "ld_run_batched",
                 "ld_backward", "rng_get_state", "gbrng_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol(G):
    lib = G.lib()
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_declared()) <= set(G.SIGNATURES)


def test_library_is_sm103a_only():
    """The build passes one -gencode: compute_103a / sm_103a."""
    from paper_1003_1123_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_lfg_table_via_abi(G, oracle_lib):
    """Table I lags (row 4 read as sl = 13470) and the default-row rule agree
    with the oracle's own table."""
    for row in range(10):
        assert G.rng_lfg_lags(row) == oracle_lib.lfg_table(row)
    for n in [1, 100, 256, 257, 300, 1000, 2460, 2461, 4096, 5000, 10**5, 10**6, 10**8]:
        assert G.rng_lfg_default_row(n) == oracle_lib.lfg_default_row(n)
    with pytest.raises(G.GbrngError) as e:
        G.rng_lfg_lags(10)
    assert e.value.code == -5


def test_invalid_arguments_rejected_before_any_device_work(G):
    lib = G.lib()
    h = C.c_void_p()
    assert lib.rng_init(C.byref(h), 7, 1, 10, None) == -1
    assert "kind" in G.gbrng_last_error()
    assert lib.rng_init(C.byref(h), 0, 1, 0, None) == -1
    assert lib.rng_init(None, 0, 1, 10, None) == -1
    assert lib.rng_init_lfg(C.byref(h), 1, 10, 11, None) == -5
    assert lib.ld_run(None, 10, None, None) == -1
    assert lib.ld_run_noalloc(None, 10, None, None) == -1
    assert lib.gbrng_set_lfg_order(3) == -1
    assert lib.gbrng_set_lfg_order(0) == 0
    assert lib.rng_fill_u32(None, None, 10, None) == -1
    assert lib.rng_set_wait_limit_ns(0) == -1
    assert lib.rng_set_wait_limit_ns(2_000_000_000) == 0
    assert lib.ld_set_adjoint_history_limit(-2) == -1
    assert "history limit" in G.gbrng_last_error()
    assert lib.ld_set_adjoint_history_limit(0) == 0
    assert lib.ld_set_adjoint_history_limit(-1) == 0
    assert lib.ld_backward(None, 10, 100, None, None, None, None, None) == -1
