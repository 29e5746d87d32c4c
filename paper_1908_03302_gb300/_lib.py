"""ctypes binding of ``libfft_gb300.so`` (declarations in ``include/fft_gb300.h``).

Argument marshalling only: every step of the computation runs in the library's CUDA
kernels. Device vectors are passed as raw pointers (``tensor.data_ptr()``) together with
the current CUDA stream of PyTorch. If the library is missing the import of any function
here raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _buildlib as _build

_lock = threading.Lock()
_lib = None

FFT_OK = 0
FFT_ERR_ARG = -1
FFT_ERR_CUDA = -2
FFT_ERR_OOM = -3
FFT_ERR_BREAKDOWN = -4
FFT_ERR_TIMEOUT = -5
FFT_ERR_STATE = -6

FFT_DT_STABLE = 0
FFT_DT_NAIVE = 1
FFT_DT_FP64 = 2

_STATUS_NAMES = {
    FFT_ERR_ARG: "FFT_ERR_ARG", FFT_ERR_CUDA: "FFT_ERR_CUDA", FFT_ERR_OOM: "FFT_ERR_OOM",
    FFT_ERR_BREAKDOWN: "FFT_ERR_BREAKDOWN", FFT_ERR_TIMEOUT: "FFT_ERR_TIMEOUT",
    FFT_ERR_STATE: "FFT_ERR_STATE",
}


class FFTError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class fft_spectrum(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("f_center_hz", ctypes.c_double), ("f_sigma_hz", ctypes.c_double),
                ("omega", ctypes.c_void_p), ("weight", ctypes.c_void_p), ("n_omega", ctypes.c_int32)]


class fft_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("h", ctypes.c_double), ("origin", ctypes.c_double * 3)]


class fft_tune_info_t(ctypes.Structure):
    _fields_ = [("items_per_cta", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("ms_J", ctypes.c_double),
                ("ms_JT", ctypes.c_double), ("n_tried", ctypes.c_int32)]


class fft_geom_info_t(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("n_vox", ctypes.c_int64), ("n_entries", ctypes.c_int64),
                ("n_items", ctypes.c_int64), ("support_evals", ctypes.c_int64),
                ("scratch_bytes", ctypes.c_int64), ("dt_mode", ctypes.c_int32),
                ("evaluated_evals", ctypes.c_int64), ("phi_terms", ctypes.c_int32),
                ("psf_tc_mma_flops", ctypes.c_double), ("psf_tc_entries", ctypes.c_double)]


# (name, restype, argtypes) for every function declared in include/fft_gb300.h
_VP, _I32, _I64, _D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
SIGNATURES = {
    "fft_table_build": (ctypes.c_int, [ctypes.POINTER(fft_spectrum), _I32, _D, _VP, ctypes.POINTER(_VP)]),
    "fft_table_destroy": (None, [_VP]),
    "fft_trig_build": (ctypes.c_int, [ctypes.POINTER(fft_spectrum), _D, _I32, _VP, _VP, _VP, ctypes.POINTER(_VP)]),
    "fft_geom_create": (ctypes.c_int, [_VP, _I32, _VP, _I64, _VP, ctypes.POINTER(fft_grid), _D, _VP, _I32,
                                       _I32, ctypes.POINTER(_VP)]),
    "fft_geom_destroy": (None, [_VP]),
    "fft_geom_info": (ctypes.c_int, [_VP, ctypes.POINTER(fft_geom_info_t)]),
    "fft_geom_autotune": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(fft_tune_info_t)]),
    "fft_J_apply": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "fft_JT_apply": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "fft_coverage": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "fft_J_apply_batch": (ctypes.c_int, [_VP, _VP, _I32, _VP, _VP]),
    "fft_JT_apply_batch": (ctypes.c_int, [_VP, _VP, _I32, _VP, _VP]),
    "fft_J2d_apply": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "fft_JT2d_apply": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "fft_hessian_lowrank": (ctypes.c_int, [_VP, _VP, _I32, _I32, _I32, _D, _VP, _VP, _VP]),
    "fft_lowrank_diag": (ctypes.c_int, [_VP, _VP, _VP, _I32, _D, _VP, _VP, _VP]),
    "fft_frob2": (ctypes.c_int, [_VP, ctypes.POINTER(_D)]),
    "fft_cg_solve": (ctypes.c_int, [_VP, _VP, _D, _I32, _VP, _VP, _VP]),
    "fft_cg_status": (ctypes.c_int, [_VP, _VP]),
    "fft_cg_continue": (ctypes.c_int, [_VP, _I32, _VP, _VP, _VP]),
    "fft_cg_state_bytes": (ctypes.c_int, [_VP, ctypes.POINTER(_I64)]),
    "fft_cg_save": (ctypes.c_int, [_VP, _VP, _I64, _VP]),
    "fft_cg_load": (ctypes.c_int, [_VP, _VP, _I64, _VP]),
    "fft_psf_batch": (ctypes.c_int, [_VP, _VP, _I32, _VP, _I32, _VP, _I32, _VP, _VP]),
    "fft_psf_noalloc": (ctypes.c_int, [_VP, _I64, _VP, _I32, _VP, _VP]),
    "fft_psf_row_groups": (ctypes.c_int, [_I64, _VP, _I32, _VP, _VP, _VP, ctypes.POINTER(_I32)]),
    "fft_tc_selftest": (ctypes.c_int, [_I32, _I32, ctypes.POINTER(_D)]),
    "fft_last_error": (ctypes.c_char_p, []),
}


def lib_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = True):
    """Load the library (building it first if it is missing or stale and nvcc is present)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB_PATH
            if build_if_missing and not _build.up_to_date():
                _build.build()
            if not os.path.exists(path):
                raise ImportError(f"CUDA library {path} is missing; run build() first")
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(status: int) -> None:
    if status != FFT_OK:
        msg = load().fft_last_error()
        raise FFTError(status, msg.decode() if msg else "")
