"""Host-side checks of the C ABI library (no GPU needed): it builds, loads, and exports
every function include/bem.h declares."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2210_08580_gb300 import bem, build
    if not os.path.exists(bem.LIB_PATH):
        build.build_library()
    import ctypes
    return ctypes.CDLL(bem.LIB_PATH)


def _declared():
    src = open(os.path.join(ROOT, "include", "bem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:bem_status|void|const char\*)\s+(\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_six_calls():
    names = _declared()
    for n in ("bem_assemble", "filter_apply", "compress_compact", "factor", "solve_many", "solve_backward"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2210_08580_gb300 import bem
    names = _declared()
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(bem.EXPORTS)


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2210_08580_gb300 import bem
    with pytest.raises(RuntimeError):
        bem._lib = None
        bem.load_library(str(tmp_path / "missing.so"))
    bem._lib = None


def test_batch_solve_refuses_bad_arguments_before_any_device_work(lib):
    """bem_solve_batch and its stall check validate their host arrays first: null arrays, a
    null handle, nprob outside [1, 65536] and a stall limit outside [1, 10000] ms return
    BEM_E_INVALID (1) without touching a device."""
    import ctypes
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    f = lib.bem_solve_batch
    f.argtypes = [ctypes.POINTER(vp), i64, ctypes.POINTER(vp), ctypes.POINTER(i64),
                  ctypes.POINTER(vp), ctypes.POINTER(i64), ctypes.POINTER(i64)]
    f.restype = ctypes.c_int
    g = lib.bem_solve_batch_stall_check
    g.argtypes = f.argtypes + [ctypes.c_int]
    g.restype = ctypes.c_int
    one = (i64 * 1)(16)
    ptrs = (vp * 1)(None)
    assert f(None, 1, ptrs, one, ptrs, one, one) == 1
    assert f(ptrs, 1, ptrs, one, ptrs, one, one) == 1          # a null handle
    assert f(ptrs, 0, ptrs, one, ptrs, one, one) == 1
    assert f(ptrs, 65537, ptrs, one, ptrs, one, one) == 1
    assert f(ptrs, 1, None, one, ptrs, one, one) == 1
    assert g(ptrs, 1, ptrs, one, ptrs, one, one, 0) == 1
    assert g(ptrs, 1, ptrs, one, ptrs, one, one, 10001) == 1
