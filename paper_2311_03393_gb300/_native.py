"""ctypes loader for libtsketch.so: the C ABI declared in include/tsketch.h.

No fallback exists: if the library is missing or fails to load, every call
raises.  Build it with `python -m paper_2311_03393_gb300.build` (or the
repository's build entry point).
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtsketch.so")

TSK_OK = 0
STATUS_NAMES = {
    0: "TSK_OK", 1: "TSK_ERR_INVALID_ARG", 2: "TSK_ERR_CUDA", 3: "TSK_ERR_OOM",
    4: "TSK_ERR_UNSUPPORTED", 5: "TSK_ERR_TIMEOUT", 6: "TSK_ERR_NONFINITE",
}
TSK_F32, TSK_F64 = 0, 1
TSK_SKETCH_BF16, TSK_SKETCH_FP32, TSK_SKETCH_FP64 = 0, 1, 2
TSK_MP_FP32, TSK_MP_FP64 = 0, 1
TSK_PROF_MP_DIAG, TSK_PROF_SKETCH, TSK_PROF_DIMS = 0, 1, 2

# name -> (restype, argtypes), mirroring include/tsketch.h
_P = C.c_void_p
_I32 = C.c_int32
_I64 = C.c_int64
SIGNATURES = {
    "tsk_create": (_I32, [C.POINTER(_P), _I32, _P]),
    "tsk_set_stream": (_I32, [_P, _P]),
    "tsk_destroy": (None, [_P]),
    "tsk_last_error": (C.c_char_p, [_P]),
    "tsk_reserve": (_I32, [_P, C.c_size_t]),
    "tsk_mp_workspace_bytes": (_I32, [_P, _I32, _P, _I32, C.POINTER(C.c_size_t)]),
    "tsk_sync": (_I32, [_P, C.c_double]),
    "tsk_selftest_timeout": (_I32, [_P]),
    "tsk_set_tile_rows": (_I32, [_P, _I32]),
    "tsk_launch_count": (_I64, [_P]),
    "tsk_profile_enable": (_I32, [_P, _I32]),
    "tsk_profile_read": (_I32, [_P, _I32, C.POINTER(C.c_double), C.POINTER(_I64)]),
    "ts_sketch_build": (_I32, [_P, _P, _I32, _I32, _P, _I32, _P, _I32, _I32, _P, _P]),
    "ts_sketch_update_dims": (_I32, [_P, _P, _P, _I32, _I32, _P, _I32, _P, _P, _I32, _I32, _P, _P]),
    "mp_selfjoin": (_I32, [_P, _P, _I32, _I32, _P, _P, _I32, _I32, _I32, _P, _P]),
    "discord_topk": (_I32, [_P, _P, _I32, _P, _I32, _P, _I32, _I32, _I32, _I32, _P, _P, _P, _P]),
    "mp_backward": (_I32, [_P, _P, _P, _P, _P, _I32, _P, _I32, _P, _P, _P, _I32, _P, _I32, _I32, _I32, _P, _P]),
    "ts_sketch_point_update": (_I32, [_P, _P, _P, _I32, _I32, _P, _I32, _P, _I32, _I32, _P, _I32, _P, _P, _P, _P]),
    "mp_abjoin": (_I32, [_P, _P, _P, _I32, _I32, _P, _P, _I32, _I32, _P, _P, _P, _P]),
    "dimension_detection": (_I32, [_P, _P, _I32, _I32, _P, _I32, _P, _I32, _I32, _I32, _I32, _P, _P, _P, _P, _P,
                                   _P, _P, _P, _P, _P]),
    "mp_selfjoin_static": (_I32, [_P, _I32, _I32, _I32, _P, _P, _P]),
    "mp_selfjoin_update": (_I32, [_P, _P, _I32, _P, _I32, _I32, _P, _P, _I32, _P, _P]),
}

_lib = None


class TskError(RuntimeError):
    """A libtsketch call returned a non-zero tsk_status."""

    def __init__(self, status: int, where: str, message: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")


def lib() -> C.CDLL:
    """Load libtsketch.so once; raise if it is not there."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build the CUDA library first "
                "(python -m paper_2311_03393_gb300.build)")
        h = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(h, name)
            fn.restype = res
            fn.argtypes = args
        _lib = h
    return _lib


def exported_symbols() -> list:
    """The C entry points this binding expects the library to export."""
    return list(SIGNATURES)


def check(status: int, ctx, where: str) -> None:
    if status != TSK_OK:
        msg = lib().tsk_last_error(ctx) if ctx else b""
        raise TskError(status, where, (msg or b"").decode(errors="replace"))
