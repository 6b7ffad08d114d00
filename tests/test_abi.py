"""The C ABI library builds for sm_103a, loads, and exports every entry point that
include/dvm.h declares; the Python binding names the same functions.  No compute calls
(no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dvm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dvm_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1912_04582_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("dvm_create", "dvm_set_bc", "dvm_init_maxwellian", "dvm_init_f", "dvm_step",
                 "dvm_moments", "dvm_solve", "dvm_get_f", "dvm_save", "dvm_load",
                 "dvm_destroy", "dvm_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib_path):
    from paper_1912_04582_gb300 import _native, api
    names = _declared()
    assert set(names) <= set(_native.SIGNATURES), set(names) - set(_native.SIGNATURES)
    for n in names:
        assert hasattr(api, n), n


def test_library_is_built_for_sm_103a(lib_path):
    from paper_1912_04582_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
    assert os.path.getsize(lib_path) > 100_000


def test_missing_library_fails_loudly(tmp_path):
    from paper_1912_04582_gb300 import _native
    with pytest.raises(RuntimeError):
        _native.load(str(tmp_path / "nope.so"))
