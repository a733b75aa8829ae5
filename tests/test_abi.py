"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/nsli.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT
from paper_2003_09956_gb300 import _build, nsli


def declared_functions():
    text = open(os.path.join(ROOT, "include", "nsli.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nsli_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(_build.LIB_PATH):
        _build.build()
    return ctypes.CDLL(_build.LIB_PATH)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["nsli_create", "nsli_update_b", "nsli_iterate", "nsli_solve",
                     "nsli_residual_max", "nsli_destroy"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    assert sorted(set(nsli.EXPORTS)) == [n for n in declared_functions() if n in nsli.EXPORTS]
    missing = [n for n in declared_functions() if n not in nsli.EXPORTS]
    assert missing == [], missing


def test_strerror_without_gpu(lib):
    lib.nsli_strerror.restype = ctypes.c_char_p
    assert lib.nsli_strerror(0) == b"ok"
    assert b"zero row" in lib.nsli_strerror(-2)


def test_argument_errors_need_no_gpu(lib):
    h = ctypes.c_void_p()
    # NULL output handle and invalid sizes are rejected before any CUDA call
    assert lib.nsli_create(None, 1, 1, 1, 1, None, 1, None, None, None, None, None) == -1
    assert lib.nsli_create(ctypes.byref(h), 0, 1, 1, 1, None, 1, None, None, None, None, None) == -1
    assert h.value is None


def test_library_links_no_torch():
    """The boundary takes plain pointers: the library's dynamic dependencies
    (the NEEDED entries that readelf prints) name no libtorch or libc10."""
    import shutil
    import subprocess

    if not os.path.exists(_build.LIB_PATH):
        _build.build()
    readelf = shutil.which("readelf")
    if readelf is None:
        pytest.skip("readelf is not installed")
    out = subprocess.run([readelf, "-d", _build.LIB_PATH], check=True, capture_output=True,
                         text=True).stdout
    needed = re.findall(r"\(NEEDED\)\s+Shared library: \[([^\]]+)\]", out)
    assert needed, out
    assert not [n for n in needed if "torch" in n or "c10" in n], needed
