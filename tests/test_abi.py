"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports
every entry point that include/sldm.h declares (no compute without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "sldm.h")).read()
    return sorted(set(re.findall(r"^(?:int|void)\s+(sldm_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2106_06184_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("sldm_mesh_create", "sldm_stack_create", "sldm_assemble", "sldm_apply", "sldm_solve"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2106_06184_gb300 import sldm
    assert set(declared_symbols()) <= set(sldm.EXPORTS)


def test_last_error_is_callable_without_gpu(lib):
    buf = ctypes.create_string_buffer(64)
    lib.sldm_last_error(buf, ctypes.c_size_t(64))
    assert isinstance(buf.value, bytes)


def test_port_sparams_is_host_math_matching_the_oracle(lib):
    """sldm_port_sparams needs no GPU: S from Y against the oracle's formula,
    the singular case and invalid arguments."""
    import numpy as np

    from oracle import ports as PT
    from paper_2106_06184_gb300 import sldm
    rng = np.random.default_rng(3)
    for n in (1, 2, 5):
        Y = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / 50.0
        Y = Y + Y.T                     # reciprocal
        assert np.allclose(sldm.sparams(Y, 50.0), PT.s_matrix(Y, 50.0), rtol=1e-12, atol=1e-12)
    with pytest.raises(sldm.SldmError):
        sldm.sparams(-np.eye(1) / 50.0, 50.0)
    with pytest.raises(sldm.SldmError):
        sldm.sparams(np.eye(2), -1.0)


def test_host_bookkeeping_calls_without_gpu(lib):
    """Timers, launch counter, device-memory budget and fault injection are host
    bookkeeping: they answer without a GPU and reject invalid arguments."""
    c = ctypes
    u, t, n = c.c_double(-1), c.c_double(-1), c.c_int64(-1)
    assert lib.sldm_timers_reset() == 0
    assert lib.sldm_timer_units(b"gemv_main", c.byref(u)) == 0 and u.value == 0.0
    assert lib.sldm_timer_units(None, c.byref(u)) == -1
    assert lib.sldm_timer_get(b"no_such_timer", c.byref(t), c.byref(n)) == 0 and (t.value, n.value) == (0.0, 0)
    buf = c.create_string_buffer(16)
    assert lib.sldm_timer_names(buf, c.c_size_t(16)) == 0 and buf.value == b""
    assert lib.sldm_launch_count(None) == -1
    assert lib.sldm_launch_count(c.byref(n)) == 0 and n.value >= 0
    assert lib.sldm_set_device_budget(c.c_int64(-1)) == -1
    assert lib.sldm_set_device_budget(c.c_int64(0)) == 0
    assert lib.sldm_device_bytes(None) == -1
    assert lib.sldm_device_bytes(c.byref(n)) == 0 and n.value == 0
    assert lib.sldm_test_inject(99, 1) == -1 and lib.sldm_test_inject(1, -1) == -1
    assert lib.sldm_test_inject(1, 0) == 0
    assert lib.sldm_set_tc_policy(0) == 0 and lib.sldm_set_tc_policy(34) == -1
