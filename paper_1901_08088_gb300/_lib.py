"""ctypes binding of ``libqbvh.so`` (C ABI in include/qbvh.h).

Argument marshalling only: every step of the neighbor search runs in the CUDA
kernels of the library.  There is no CPU fallback; if the library has not been
built, loading fails with an error that says how to build it.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libqbvh.so")

QBVH_OK = 0
QBVH_ERR_INVALID_ARG = 1
QBVH_ERR_OUT_OF_BOX = 2
QBVH_ERR_BAD_TYPE = 3
QBVH_ERR_CUTOFF_TOO_LARGE = 4
QBVH_ERR_OVERFLOW = 5
QBVH_ERR_DEVICE_TIMEOUT = 6
QBVH_ERR_CUDA = 7
QBVH_ERR_OOM = 8
QBVH_ERR_NOT_BUILT = 9
QBVH_ERR_INTERNAL = 10

QBVH_OPT_BUNDLE = 1
QBVH_OPT_QUERY_BLOCK = 2
QBVH_OPT_CANDIDATES = 3
QBVH_OPT_TRAVERSAL = 4
QBVH_OPT_NODE_FORMAT = 5
QBVH_OPT_LJ_LANES = 6
QBVH_OPT_LJ_ZORDER = 7
QBVH_OPT_METHOD = 8
QBVH_OPT_GRID_LANES = 9
QBVH_OPT_WARP_PARTICLES = 10
QBVH_OPT_TYPE_TREES = 11
QBVH_OPT_FUSED_LJ = 12
QBVH_OPT_PERSISTENT = 13

_lock = threading.Lock()
_lib = None

P = C.c_void_p
I = C.c_int
F = C.c_float
D = C.c_double
PP = C.POINTER(C.c_void_p)
PI = C.POINTER(C.c_int)

# name -> (restype, argtypes); names are the C entry points
SIGNATURES = {
    "qbvh_strerror": (C.c_char_p, [I]),
    "qbvh_create": (I, [PP, I]),
    "qbvh_destroy": (I, [P]),
    "qbvh_set_option": (I, [P, I, I]),
    "qbvh_get_option": (I, [P, I, PI]),
    "qbvh_build": (I, [P, P, I, F, I, P]),
    "qbvh_build_f64": (I, [P, P, I, D, I, P]),
    "qbvh_build_batched": (I, [P, P, I, I, P, P, I, P]),
    "qbvh_query": (I, [P, P, I, I, P]),
    "qbvh_query_async": (I, [P, P, I, P]),
    "qbvh_query_status": (I, [P, PI]),
    "qbvh_query_lj_async": (I, [P, P, P, I, P, P, P, P, P, P, P, P, P]),
    "nlist_get": (I, [P, PP, PP, PI, PI]),
    "qbvh_tree_get": (I, [P, PP, PP, PP, PP, PP, PI]),
    "qbvh_lj_forward": (I, [P, P, P, P, P, P, P, P, P, P, P]),
    "qbvh_lj_backward": (I, [P, P, P, P, P, P, P, P, P]),
    "qbvh_pack_positions": (I, [P, P, I, P, P]),
    "qbvh_lj_forward_noalloc": (I, [P, I, F, I, P, P, I, P, P, P, P, P, P, P, P, P, P]),
    "qbvh_selftest_wait_timeout": (I, [I, P]),
}


class QBVHError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        self.code = int(code)
        msg = lib().qbvh_strerror(self.code).decode()
        super().__init__(f"{where}: {msg} (code {self.code})" if where else f"{msg} (code {self.code})")


def lib():
    """Load libqbvh.so once; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with "
                    "`python -m paper_1901_08088_gb300.build_lib` (the CUDA path has no CPU fallback)")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(code: int, where: str = "") -> int:
    if code != QBVH_OK:
        raise QBVHError(code, where)
    return code
