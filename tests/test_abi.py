"""The C ABI library builds for sm_103a, loads without a GPU and exports every
function include/crk.h declares; host-side argument checks need no device."""
import ctypes as C

import pytest

from paper_2511_21921_gb300 import _lib as L


def test_library_exports_every_header_symbol():
    lib = L.load()
    names = L.header_symbols()
    assert len(names) >= 12
    for nm in names:
        assert hasattr(lib, nm), nm
    assert set(names) == set(L._SIGS), "binding and header disagree"


def test_status_strings_and_defaults():
    for code in range(9):
        assert L.crk_status_string(code)
    p = L.crk_params_default()
    assert abs(p.gamma - 5.0 / 3.0) < 1e-15 and p.Cl == 2.0 and p.Cq == 1.0
    assert p.precision == L.CRK_MIXED32 and p.limiter == 1 and p.relax_dt == 0.0


def test_argument_errors_are_synchronous():
    lib = L.load()
    p = L.crk_params_default()
    h = C.c_void_p()
    assert lib.crk_plan_create(None, 10, 1, C.byref(h)) == L.CRK_EINVAL
    bad = L.crk_params_default()
    bad.gamma = 1.0
    assert lib.crk_plan_create(C.byref(bad), 10, 1, C.byref(h)) == L.CRK_EINVAL
    bad = L.crk_params_default()
    bad.precision = 7
    assert lib.crk_plan_create(C.byref(bad), 10, 1, C.byref(h)) == L.CRK_EINVAL
    assert lib.crk_plan_create(C.byref(p), -1, 1, C.byref(h)) == L.CRK_EINVAL
    assert lib.crk_plan_create(C.byref(p), 10, 0, C.byref(h)) == L.CRK_EINVAL
    b = C.c_size_t()
    assert lib.crk_workspace_size(None, 10, 1, C.byref(b)) == L.CRK_EINVAL
    assert lib.crk_moments(None, None, None, None, None, None) == L.CRK_EINVAL
    assert lib.crk_rates(None, None, None, None, None, None, None, None, None) == L.CRK_EINVAL


def test_copy_argument_errors():
    """crk_copy rejects bad arguments before any CUDA call; zero bytes is a no-op."""
    lib = L.load()
    assert lib.crk_copy(None, None, None, 0) == L.CRK_OK
    assert lib.crk_copy(None, None, C.c_void_p(0x1000), 16) == L.CRK_EINVAL
    assert lib.crk_copy(None, C.c_void_p(0x1000), None, 16) == L.CRK_EINVAL
    # overlapping ranges
    assert lib.crk_copy(None, C.c_void_p(0x1008), C.c_void_p(0x1000), 16) == L.CRK_EINVAL
