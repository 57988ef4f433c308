"""Host-side checks of the C ABI: the library builds, loads, and exports every
function that include/*.h declares.  No compute call is made (no GPU here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(dqmc_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2003_05286_gb300 import build as b
    b.build()
    return ctypes.CDLL(b.lib_path())


def test_header_declares_the_paper_calls():
    names = _declared()
    for n in ("dqmc_greens", "dqmc_greens_tdisplaced", "dqmc_logdet", "dqmc_logdet_grad"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header():
    from paper_2003_05286_gb300 import _abi
    assert set(_abi.SIGNATURES) == set(_declared())


def test_status_string_and_arg_checks(lib):
    lib.dqmc_status_string.restype = ctypes.c_char_p
    assert lib.dqmc_status_string(0) == b"ok"
    assert lib.dqmc_status_string(1) == b"invalid argument"
    # NULL handle is rejected before any CUDA call
    lib.dqmc_greens.restype = ctypes.c_int
    rc = lib.dqmc_greens(None, 1, 4, 4, None, ctypes.c_double(0.1), None, 1, None, None, None, None)
    assert rc == 1
    lib.dqmc_destroy.restype = ctypes.c_int
    assert lib.dqmc_destroy(None) == 1


def test_product_path_has_no_cpu_fallback():
    """The package must not import the oracle or any CPU implementation."""
    pkg = os.path.join(ROOT, "paper_2003_05286_gb300")
    for f in glob.glob(os.path.join(pkg, "*.py")):
        src = open(f).read()
        assert "oracle" not in src.replace("oracle`", ""), f
        assert "numpy.linalg" not in src and "scipy" not in src, f


def test_fp64_rate_rejects_bad_arguments(lib):
    """Argument checks run before any CUDA call (no GPU needed)."""
    f = lib.dqmc_selftest_fp64_rate
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                  ctypes.POINTER(ctypes.c_double)]
    tf = ctypes.c_double()
    assert f(None, 0, 100, None, None) == 1                 # NULL result pointer
    assert f(None, 3, 100, ctypes.byref(tf), None) == 1     # unknown kind
    assert f(None, 0, 0, ctypes.byref(tf), None) == 1       # no iterations


@pytest.fixture(scope="module")
def dlib():
    from paper_2003_05286_gb300 import build as b
    b.build(debug=True)
    return ctypes.CDLL(b.lib_path(debug=True))


def test_debug_library_exports_the_same_calls(lib, dlib):
    """The debug variant (-DDQMC_DEBUG) is the same C ABI: every declared
    symbol, and it reports itself as the debug build."""
    missing = [n for n in _declared() if not hasattr(dlib, n)]
    assert not missing, missing
    lib.dqmc_is_debug_build.restype = ctypes.c_int
    dlib.dqmc_is_debug_build.restype = ctypes.c_int
    assert lib.dqmc_is_debug_build() == 0 and dlib.dqmc_is_debug_build() == 1


def test_debug_read_in_release_library(lib):
    """Argument checks and the release answer come before any CUDA call."""
    f = lib.dqmc_debug_read
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_int),
                  ctypes.POINTER(ctypes.c_int)]
    fn, ln, val = ctypes.c_char_p(), ctypes.c_int(), ctypes.c_int()
    assert f(0, None, ctypes.byref(ln), ctypes.byref(val)) == 1
    assert f(0, ctypes.byref(fn), ctypes.byref(ln), ctypes.byref(val)) == 7   # UNSUPPORTED
    s = lib.dqmc_selftest_check
    s.restype = ctypes.c_int
    s.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    fired = ctypes.c_int()
    assert s(None, None, ctypes.byref(val)) == 1
    assert s(None, ctypes.byref(fired), ctypes.byref(val)) == 7


def test_memory_limit_rejects_bad_arguments(lib):
    f = lib.dqmc_set_memory_limit
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_longlong]
    assert f(None, 0) == 1
    lib.dqmc_device_bytes.restype = ctypes.c_longlong
    lib.dqmc_device_bytes.argtypes = [ctypes.c_void_p]
    assert lib.dqmc_device_bytes(None) == -1


def test_tune_mode_parsing(monkeypatch):
    """The tuner's mode switch is host logic (no GPU needed)."""
    from paper_2003_05286_gb300 import tune
    for v, want in (("", "on"), ("on", "on"), ("FORCE", "force"), (" off ", "off")):
        monkeypatch.setenv("DQMC_TUNE", v)
        assert tune.tune_mode() == want
    monkeypatch.delenv("DQMC_TUNE")
    assert tune.tune_mode() == "on"
    monkeypatch.setenv("DQMC_TUNE", "x")
    with pytest.raises(ValueError):
        tune.tune_mode()
