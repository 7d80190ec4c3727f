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
