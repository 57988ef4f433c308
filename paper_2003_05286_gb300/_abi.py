"""ctypes declarations of the C ABI in include/dqmc.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

DQMC_OK = 0
STATUS_STRINGS = {
    0: "ok", 1: "invalid argument", 2: "CUDA runtime or launch failure",
    3: "device workspace allocation failed", 4: "non-finite value", 5: "singular pivot",
    6: "bounded device wait gave up", 7: "unsupported configuration",
    8: "problem needs more device scratch than the fixed array holds",
    9: "a device-side check of the debug build failed",
}
STATUS_BITS = {
    "NONFINITE_INPUT": 1 << 0, "NONFINITE_SCALE": 1 << 1, "SINGULAR": 1 << 2,
    "NONFINITE_OUTPUT": 1 << 3, "BAD_K": 1 << 4, "TIMEOUT": 1 << 5, "NOT_CONVERGED": 1 << 6,
}
CHAIN_FP64 = 0
CHAIN_BF16X3 = 3
PTR_DEVICE = 0
PTR_HOST = 1
FOLD_SEQUENTIAL, FOLD_TREE, FOLD_AUTO = 0, 1, 2
INV_LOH, INV_PLAIN = 0, 1
DECOMP_QR, DECOMP_JACOBI = 0, 1


class DqmcDesc(C.Structure):
    _fields_ = [("N", C.c_int), ("M", C.c_int), ("k", C.c_int), ("K_id", C.c_int),
                ("off_V", C.c_longlong), ("off_G", C.c_longlong)]


class DqmcInstance(C.Structure):
    _fields_ = [("N", C.c_int), ("M", C.c_int), ("k", C.c_int), ("pad", C.c_int),
                ("dtau", C.c_double), ("off_K", C.c_longlong), ("off_V", C.c_longlong),
                ("off_G", C.c_longlong)]


_P = C.c_void_p
_I = C.c_int
_D = C.c_double

# name -> (restype, argtypes)
SIGNATURES = {
    "dqmc_create": (_I, [C.POINTER(_P)]),
    "dqmc_destroy": (_I, [_P]),
    "dqmc_set_stream": (_I, [_P, _P]),
    "dqmc_set_pointer_mode": (_I, [_P, _I]),
    "dqmc_set_chain_precision": (_I, [_P, _I]),
    "dqmc_set_gemm_tile": (_I, [_P, _I]),
    "dqmc_set_chain_fold": (_I, [_P, _I]),
    "dqmc_set_inversion_scheme": (_I, [_P, _I]),
    "dqmc_set_decomposition": (_I, [_P, _I]),
    "dqmc_last_launch_count": (C.c_longlong, [_P]),
    "dqmc_workspace_bytes": (C.c_longlong, [_P]),
    "dqmc_device_bytes": (C.c_longlong, [_P]),
    "dqmc_set_memory_limit": (C.c_int, [_P, C.c_longlong]),
    "dqmc_status_string": (C.c_char_p, [_I]),
    "dqmc_profile_enable": (_I, [_P, _I]),
    "dqmc_profile_reset": (_I, [_P]),
    "dqmc_profile_read": (_I, [_P, _I, C.POINTER(C.c_double), C.POINTER(C.c_longlong),
                               C.POINTER(C.c_double)]),
    "dqmc_greens": (_I, [_P, _I, _I, _I, _P, _D, _P, _I, _P, _P, _P, _P]),
    "dqmc_logdet": (_I, [_P, _I, _I, _I, _P, _D, _P, _I, _P, _P, _P]),
    "dqmc_greens_tdisplaced": (_I, [_P, _I, _I, _I, _P, _D, _P, _I, _P, _P, _P]),
    "dqmc_greens_tdisplaced_ex": (_I, [_P, _I, _I, _I, _P, _D, _P, _I, _P, _P, _P, _P]),
    "dqmc_greens_tdisplaced_all": (_I, [_P, _I, _I, _I, _P, _D, _P, _I, _P, _P, _P, _P]),
    "dqmc_greens_tdisplaced_from": (_I, [_P, _I, _I, _I, _P, _D, _P, _I, _P, _I, _P, _P, _P, _P]),
    "dqmc_logdet_grad": (_I, [_P, _I, _I, _I, _P, _D, _P, _I, _P, _P, _P, _P]),
    "dqmc_greens_ragged": (_I, [_P, _I, C.POINTER(DqmcInstance), _P, _P, _P, _P, _P, _P]),
    "dqmc_greens_noalloc": (_I, [_P, _I, _I, _I, _P, _D, _P, _I, _P, _P, _P, _P]),
    "dqmc_selftest_wait_timeout": (_I, [_P, _P]),
    "dqmc_selftest_fp64_rate": (_I, [_P, _I, _I, C.POINTER(_D), C.POINTER(_D)]),
    "dqmc_is_debug_build": (_I, []),
    "dqmc_debug_read": (_I, [_I, C.POINTER(C.c_char_p), C.POINTER(_I), C.POINTER(_I)]),
    "dqmc_selftest_check": (_I, [_P, C.POINTER(_I), C.POINTER(_I)]),
    "dqmc_register_K": (_I, [_P, _I, _P, _D, C.POINTER(_I)]),
    "dqmc_greens_batched": (_I, [_P, _I, _P, _P, _P, _P, _P, _P]),
    "dqmc_set_graph_mode": (_I, [_P, _I]),
    "dqmc_greens_tdisplaced_ragged": (_I, [_P, _I, C.POINTER(DqmcInstance), _P, _P, _P, _P, _P]),
    "dqmc_greens_tdisplaced_ragged_ex": (_I, [_P, _I, C.POINTER(DqmcInstance), _P, _P, _P, _P, _P,
                                              _P]),
    "dqmc_logdet_grad_ragged": (_I, [_P, _I, C.POINTER(DqmcInstance), _P, _P, _P, _P, _P, _P]),
}

_lib = None


def debug_requested() -> bool:
    """True when the environment asks for the debug library (DQMC_DEBUG set, not 0)."""
    return os.environ.get("DQMC_DEBUG", "0") not in ("", "0")


def load(path: str | None = None):
    """Loads the in-tree shared library; raises if it has not been built.

    With DQMC_DEBUG=1 in the environment the debug library (device-side checks,
    include/dqmc.h) is loaded instead."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.lib_path(debug=debug_requested())
    if not os.path.exists(path):
        raise RuntimeError(
            f"CUDA library not built ({path} missing): run "
            "`python -c 'import __graft_entry__ as g; g.build()'` first")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(rc: int, what: str) -> None:
    if rc != DQMC_OK:
        raise RuntimeError(f"{what} failed: {STATUS_STRINGS.get(rc, rc)} (code {rc})")
