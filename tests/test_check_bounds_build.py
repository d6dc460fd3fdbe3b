"""Host-side checks of the bounds-checked debug build (no GPU needed).

The debug build (compiled with SSM_CHECK_BOUNDS, libssm_check.so) stands in for a
memory checker: its kernels check the indices they take from data against the
arrays they address and report SSM_EBOUNDS instead of touching memory outside an
array.  Here: both builds compile and export the same entry points; the flag that
tells them apart; the status string; and the test hook ssm_opts.inject, which only
the debug build accepts and only where the planted index stays inside the padded
arrays -- all checked before any GPU call.
"""
import ctypes
import os

import pytest

from tests.test_abi import _declared_functions

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libs():
    from paper_2105_09688_gb300 import build as B
    import paper_2105_09688_gb300 as S
    rel = ctypes.CDLL(B.build())
    chk = ctypes.CDLL(B.build(check_bounds=True))
    for L in (rel, chk):
        L.ssm_build_flags.restype = ctypes.c_int
        L.ssm_status_str.restype = ctypes.c_char_p
        L.ssm_status_str.argtypes = [ctypes.c_int]
        L.ssm_opts_default.argtypes = [ctypes.POINTER(S.ssm_opts)]
        L.ssm_create.restype = ctypes.c_int
        L.ssm_create.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                 ctypes.c_uint64, ctypes.POINTER(S.ssm_opts), ctypes.POINTER(ctypes.c_void_p)]
    return S, rel, chk


def test_both_builds_export_every_declared_symbol(libs):
    _, rel, chk = libs
    for n in _declared_functions():
        assert hasattr(rel, n) and hasattr(chk, n), n


def test_build_flag_tells_the_builds_apart(libs):
    S, rel, chk = libs
    assert rel.ssm_build_flags() == 0
    assert chk.ssm_build_flags() == S.SSM_BUILD_CHECK_BOUNDS
    for L in (rel, chk):
        assert L.ssm_status_str(S.SSM_EBOUNDS).decode().startswith("SSM_EBOUNDS")


def _create(S, L, d, N, coef, **opt):
    o = S.ssm_opts()
    L.ssm_opts_default(ctypes.byref(o))
    for k, v in opt.items():
        setattr(o, k, v)
    out = ctypes.c_void_p()
    return L.ssm_create(d, N, 2.0 ** -8, 1.0, coef, 0, ctypes.byref(o), ctypes.byref(out))


def test_inject_hook_is_rejected_where_it_is_not_safe(libs):
    """Release build: any nonzero inject.  Debug build: values other than 1, sets
    other than the coupled ones, step 1 against mu^Y, or N a multiple of 128 (no
    padding past particle N)."""
    S, rel, chk = libs
    assert _create(S, rel, 3, 33, S.SSM_COEF_COUPLED3D, inject=1) == S.SSM_EINVAL
    assert _create(S, chk, 3, 33, S.SSM_COEF_COUPLED3D, inject=2) == S.SSM_EINVAL
    assert _create(S, chk, 3, 128, S.SSM_COEF_COUPLED3D, inject=1) == S.SSM_EINVAL
    assert _create(S, chk, 3, 33, S.SSM_COEF_COUPLED3D, inject=1, measure_y=1) == S.SSM_EINVAL
    assert _create(S, chk, 1, 33, S.SSM_COEF_CUBIC1D_GAUSS, inject=1) == S.SSM_EINVAL
