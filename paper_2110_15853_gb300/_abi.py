"""ctypes declarations of the chfsi C ABI (include/chfsi.h).

Argument marshalling only: every computation happens in libchfsi.so on the GPU.
Loading fails loudly if the library has not been built; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libchfsi.so")

CHFSI_OK = 0
CHFSI_ERR_ARG = 1
CHFSI_ERR_BOUNDS = 2
CHFSI_ERR_PATTERN = 3
CHFSI_ERR_CHOL = 4
CHFSI_ERR_NONFINITE = 5
CHFSI_ERR_CUDA = 6
CHFSI_ERR_TIMEOUT = 7
CHFSI_ERR_NOMEM = 8
CHFSI_ERR_UNSUPPORTED = 9

CHFSI_CSR = 0
CHFSI_BSR = 1
CHFSI_HYBRID = 2
CHFSI_SPLIT = 3

CHFSI_F64 = 0
CHFSI_F32 = 1
CHFSI_BF16_F32ACC = 2
CHFSI_F32X2 = 3
CHFSI_F64_OZAKI = 4
CHFSI_F40_OZAKI = 5

CHFSI_OP_TN = 0
CHFSI_OP_NN = 1
CHFSI_GEMM_SYMMETRIC = 1
CHFSI_GEMM_B_UPPER = 2

_i32, _i64, _dbl, _vp, _sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t


class chfsi_csr(ctypes.Structure):
    _fields_ = [("n_rows", _i64), ("nnz", _i64), ("row_ptr", _vp), ("col", _vp), ("val", _vp)]


class chfsi_bsr(ctypes.Structure):
    _fields_ = [("n_block_rows", _i64), ("n_blocks", _i64), ("bdim", _i32), ("brow_ptr", _vp), ("bcol", _vp),
                ("val", _vp)]


class chfsi_split(ctypes.Structure):
    _fields_ = [("n_rows", _i64), ("block", _i32), ("diag", _vp), ("off", chfsi_csr)]


class chfsi_matrix(ctypes.Structure):
    _fields_ = [("kind", _i32), ("csr", chfsi_csr), ("bsr", chfsi_bsr), ("split", chfsi_split)]


class chfsi_schedule(ctypes.Structure):
    _fields_ = [("m", _i32), ("step_prec", ctypes.POINTER(_i32))]


_MP = ctypes.POINTER(chfsi_matrix)
_SP = ctypes.POINTER(chfsi_schedule)
_SZP = ctypes.POINTER(_sz)
_DP = ctypes.POINTER(_dbl)

# name -> (restype, argtypes)
SIGNATURES = {
    "chfsi_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "chfsi_version": (ctypes.c_int, []),
    "chfsi_filter_workspace_size": (ctypes.c_int, [_MP, _i64, _i32, _SP, _SZP]),
    "chfsi_filter": (ctypes.c_int, [_MP, _vp, _i64, _vp, _i64, _i64, _i32, _dbl, _dbl, _dbl, _SP, _vp, _sz, _vp]),
    "chfsi_filter_backward_workspace_size": (ctypes.c_int, [_MP, _i64, _i32, _i32, _SZP]),
    "chfsi_filter_backward": (ctypes.c_int, [_MP, _vp, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _i32, _dbl, _dbl,
                                             _dbl, _i32, _vp, _sz, _vp]),
    "chfsi_filter_backward_ex_workspace_size": (ctypes.c_int, [_MP, _i64, _i32, _i32, _i32, _SZP]),
    "chfsi_filter_backward_ex": (ctypes.c_int, [_MP, _vp, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _i32, _dbl, _dbl,
                                                _dbl, _i32, _i32, _vp, _sz, _vp]),
    "chfsi_rayleigh_ritz_workspace_size": (ctypes.c_int, [_MP, _i64, _i32, _SZP]),
    "chfsi_rayleigh_ritz": (ctypes.c_int, [_MP, _vp, _i64, _i64, _vp, _i64, _vp, _i32, _vp, _sz, _vp]),
    "chfsi_rayleigh_ritz_ex_workspace_size": (ctypes.c_int, [_MP, _i64, _i32, _i32, _SZP]),
    "chfsi_rayleigh_ritz_ex": (ctypes.c_int, [_MP, _vp, _i64, _i64, _vp, _i64, _vp, _i32, _i32, _vp, _sz, _vp]),
    "chfsi_lanczos_workspace_size": (ctypes.c_int, [_MP, _i32, _SZP]),
    "chfsi_lanczos_bounds": (ctypes.c_int, [_MP, _i32, _vp, _i64, _DP, _DP, _DP, _vp, _sz, _vp]),
    "chfsi_read_status": (ctypes.c_int, [_vp, _vp]),
    "chfsi_clear_status": (ctypes.c_int, [_vp, _vp]),
    "chfsi_kernel_launches": (ctypes.c_ulonglong, []),
    "chfsi_set_pipeline_wait_limit": (ctypes.c_int, [ctypes.c_uint64]),
    "chfsi_measure_pipe_peak": (ctypes.c_int, [_i32, _DP, _vp]),
    "chfsi_eigh_workspace_size": (ctypes.c_int, [_i64, _SZP]),
    "chfsi_eigh": (ctypes.c_int, [_vp, _i64, _i64, _vp, _vp, _i64, _vp, _sz, _vp]),
    "chfsi_ozaki_gemm_workspace_size": (ctypes.c_int, [_i32, _i64, _i64, _i64, _i32, _SZP]),
    "chfsi_ozaki_gemm": (ctypes.c_int, [_i32, _vp, _i64, _vp, _i64, _vp, _i64, _i64, _i64, _i64, _i32, _vp, _sz,
                                        _vp]),
    "chfsi_filter_noalloc": (ctypes.c_int, [_MP, _vp, _i64, _vp, _i64, _i64, _i32, _dbl, _dbl, _dbl, _SP, _vp]),
    "chfsi_filter_noalloc_read_status": (ctypes.c_int, [_vp]),
}

_lib = None


class ChfsiError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: chfsi status {code} ({status_string(code)})")


def load():
    """Load libchfsi.so (built in-tree); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"libchfsi.so not found at {LIB_PATH}; build it with "
                "`python -m paper_2110_15853_gb300.build` (nvcc, sm_103a)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def status_string(code: int) -> str:
    try:
        return load().chfsi_status_string(int(code)).decode()
    except ImportError:
        return "library not loaded"


def check(code: int, where: str) -> None:
    if code != CHFSI_OK:
        raise ChfsiError(code, where)
