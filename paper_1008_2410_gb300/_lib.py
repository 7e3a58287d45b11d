"""ctypes loader of the C ABI in ``include/fmm2d.h`` (library ``_build/libfmm2d.so``).

Argument marshalling only: every step of an evaluation runs in the CUDA library. Loading fails loudly (an
ImportError naming the missing file) when the library has not been built; there is no other code path.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("FMM2D_LIB") or os.path.join(HERE, "_build", "libfmm2d.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "fmm2d.h")

FMM_OK, FMM_EINVAL, FMM_ENOMEM, FMM_ECUDA, FMM_ETIMEOUT, FMM_EINTERNAL = range(6)
FMM_FP64, FMM_MIXED = 0, 1

_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.c_double
_I = ctypes.c_int

SIGNATURES = {
    "fmm_create": (_I, [_I, _I, _D, ctypes.POINTER(_P)]),
    "fmm_destroy": (_I, [_P]),
    "fmm_set_domain": (_I, [_P, _D, _D, _D]),
    "fmm_clear_domain": (_I, [_P]),
    "fmm_set_precision": (_I, [_P, _I]),
    "fmm_set_coarse_level": (_I, [_P, _I]),
    "fmm_set_m2l_engine": (_I, [_P, _I]),
    "fmm_get_m2l_engine": (_I, [_P]),
    "fmm_set_adaptive": (_I, [_P, _I]),
    "fmm_get_adaptive": (_I, [_P]),
    "fmm_suggest_depth": (_I, [_I64, _D, _D, _D, _D]),
    "fmm_set_params": (_I, [_P, _I, _I, _D]),
    "fmm_set_stream": (_I, [_P, _P]),
    "fmm_set_graph": (_I, [_P, _I]),
    "fmm_set_p2p_tile": (_I, [_P, _I, _I]),
    "fmm_set_far_tail": (_I, [_P, _I]),
    "fmm_velocity": (_I, [_P, _I64, _P, _P, _P, _P, _P]),
    "fmm_velocity_host": (_I, [_P, _I64, _P, _P, _P, _P, _P]),
    "fmm_velocity_near": (_I, [_P, _I64, _P, _P, _P, _P, _P]),
    "fmm_velocity_far": (_I, [_P, _I64, _P, _P, _P, _P, _P]),
    "fmm_velocity_adjoint": (_I, [_P, _I64, _P, _P, _P, _P, _P, _P, _P, _P]),
    "fmm_velocity_batched": (_I, [_P, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "fmm_advect": (_I, [_P, _I64, _P, _P, _P, _D, _I, _I]),
    "fmm_sync": (_I, [_P]),
    "fmm_selftest_timeout": (_I, [_P, _I]),
    "fmm_set_adjoint_precision": (_I, [_P, _I]),
    "fmm_level_multipoles": (_I, [_P, _I64, _P, _P, _P, _I, _P, _P]),
    "fmm_velocity_level": (_I, [_P, _I64, _P, _P, _P, _I, _P, _P, _P, _P]),
    "fmm_set_timing": (_I, [_P, _I]),
    "fmm_stage_times": (_I, [_P, ctypes.POINTER(ctypes.c_float), _I]),
    "fmm_set_count_pairs": (_I, [_P, _I]),
    "fmm_last_pair_count": (_I64, [_P]),
    "fmm_kernel_launches": (_I64, [_P]),
    "fmm_autotune": (_I, [_P, _I64, _P, _P, _P, _P, _P, _I, _I]),
    "fmm_autotune_p": (_I, [_P, _I64, _P, _P, _P, _D, _I, _I, ctypes.POINTER(_D)]),
    "fmm_autotune_batched": (_I, [_P, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "fmm_get_params": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_D), ctypes.POINTER(_I),
                            ctypes.POINTER(_I)]),
    "fmm_probe_peaks": (_I, [ctypes.POINTER(_D), _I]),
    "fmm_velocity_noalloc": (_I, [_I, _I, _D, _I, _P, _I64, _P, _P, _P, _P, _P, _P]),
    "fmm_status_string": (ctypes.c_char_p, [_I]),
    "fmm_last_error": (ctypes.c_char_p, [_P]),
}


def header_functions() -> list[str]:
    """Names of the functions declared in include/fmm2d.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fmm_[a-z0-9_]+)\s*\(", text)))


def load() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA library {LIB_PATH} is missing: build it with paper_1008_2410_gb300.build.build()")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def probe_peaks() -> dict:
    """Measured FP32 / FP64 FMA TFLOP/s, SFU (ex2 + rcp) rate and TF32 MMA issue cycles of the current device."""
    lib = load()
    buf = (_D * 6)()
    st = lib.fmm_probe_peaks(buf, 6)
    if st != FMM_OK:
        raise FMMError(st, lib.fmm_status_string(st).decode())
    return {"fp32_tflops": buf[0], "fp64_tflops": buf[1], "sfu_tops": buf[2], "sms": int(buf[3]),
            "tf32_mma_cycles_n48": buf[4], "tf32_mma_cycles_n256": buf[5]}


class FMMError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"[{status}] {message}")
        self.status = status


def check(status: int, handle=None) -> None:
    if status != FMM_OK:
        lib = load()
        msg = lib.fmm_last_error(handle).decode() if handle else ""
        if not msg:
            msg = lib.fmm_status_string(status).decode()
        raise FMMError(status, msg)
