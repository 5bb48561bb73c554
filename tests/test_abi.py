"""The C ABI: the shared library builds, loads without a GPU, and exports
exactly the entry points include/ccorr.h declares (no compute calls)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "ccorr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return set(re.findall(r"^\s*(?:cc_status|const char\*)\s+(cc_\w+)\s*\(", text, flags=re.M))


@pytest.fixture(scope="module")
def libpath():
    from paper_2309_03308_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = header_functions()
    assert {"cc_create", "cc_load_field", "cc_eval_pairs", "cc_all_pairs"} <= names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    missing = header_functions() - exported
    assert not missing, missing
    lib = ctypes.CDLL(libpath)
    for name in header_functions():
        assert getattr(lib, name) is not None


def test_binding_declares_every_symbol(libpath):
    from paper_2309_03308_gb300 import _lib
    assert set(_lib.SIGNATURES) == header_functions()
    lib = _lib.load(libpath)
    assert lib.cc_last_error(None) == b"null context"


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2309_03308_gb300 import _lib
    with pytest.raises(RuntimeError):
        ctypes_lib = _lib._lib
        _lib._lib = None
        try:
            _lib.load(str(tmp_path / "missing.so"))
        finally:
            _lib._lib = ctypes_lib


def test_create_rejects_bad_device(libpath):
    from paper_2309_03308_gb300 import _lib
    lib = _lib.load(libpath)
    h = ctypes.c_void_p()
    assert lib.cc_create(-1, None, ctypes.byref(h)) == _lib.CC_ERR_INVALID_ARG
