"""ctypes declarations of librom's C ABI (include/rom.h). Marshalling only."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librom.so")

ROM_OK, ROM_EINVAL, ROM_ENOMEM, ROM_ECUDA, ROM_ENOCONV, ROM_ENONFINITE, ROM_ETIMEOUT, ROM_ESTATE = range(8)

EXPORTED = [
    "rom_init", "rom_step", "rom_update_basis", "rom_state", "rom_load_state", "rom_samples",
    "rom_info", "rom_destroy", "rom_status_string", "rom_fom_rhs_dev", "rom_fom_step_dev",
    "rom_isvd_update_dev", "rom_profile", "rom_profile_read", "rom_fom_step_noalloc_dev",
    "rom_batch_init", "rom_batch_step", "rom_batch_state", "rom_batch_info", "rom_batch_layout",
    "rom_batch_profile", "rom_batch_profile_read", "rom_batch_destroy", "rom_batch_work",
    "rom_debug_set_wait_limit", "rom_adjoint", "rom_batch_fom_work",
]


class RomConfigC(ctypes.Structure):
    _fields_ = [
        ("problem", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("n_cells", ctypes.c_int64),
        ("n_var", ctypes.c_int32),
        ("r", ctypes.c_int32),
        ("n_s", ctypes.c_int32),
        ("w_init", ctypes.c_int32),
        ("z", ctypes.c_int32),
        ("newton_max", ctypes.c_int32),
        ("dt", ctypes.c_double),
        ("nu", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("lambda_", ctypes.c_double),
        ("newton_tol", ctypes.c_double),
        ("rank_tol", ctypes.c_double),
        ("projection", ctypes.c_int32),
        ("update_rule", ctypes.c_int32),
        ("window", ctypes.c_int32),
        ("time_scheme", ctypes.c_int32),
        ("learning_rate", ctypes.c_double),
    ]


class RomError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {status_string(code)} ({code})")


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load librom.so; there is no fallback if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"librom.so not found at {path}; build it with "
                          "python -m paper_2605_28684_gb300.build")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    D = ctypes.POINTER(ctypes.c_double)
    I32P = ctypes.POINTER(ctypes.c_int32)
    lib.rom_init.argtypes = [ctypes.POINTER(RomConfigC), D, P, ctypes.POINTER(P)]
    lib.rom_step.argtypes = [P, ctypes.c_int64]
    lib.rom_update_basis.argtypes = [P, D]
    lib.rom_state.argtypes = [P, D, D, D, D, D, ctypes.POINTER(ctypes.c_int64)]
    lib.rom_load_state.argtypes = [P, D, D, D, D, ctypes.c_int64]
    lib.rom_samples.argtypes = [P, I32P]
    lib.rom_info.argtypes = [P, I32P, I32P, I32P]
    lib.rom_destroy.argtypes = [P]
    lib.rom_destroy.restype = None
    lib.rom_status_string.argtypes = [ctypes.c_int]
    lib.rom_status_string.restype = ctypes.c_char_p
    lib.rom_fom_rhs_dev.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                    P, P, P]
    lib.rom_fom_step_dev.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_int32, P, P, I32P, P]
    lib.rom_fom_step_noalloc_dev.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_int32, P, P, I32P, P]
    lib.rom_isvd_update_dev.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                                        ctypes.c_double, P, P, P, D, P]
    lib.rom_debug_set_wait_limit.argtypes = [ctypes.c_int64]
    lib.rom_adjoint.argtypes = [ctypes.POINTER(RomConfigC), D, D, ctypes.c_int64, ctypes.c_int32, P,
                                D, D, D, D]
    lib.rom_profile.argtypes = [P, ctypes.c_int32]
    lib.rom_profile_read.argtypes = [P, D, ctypes.POINTER(ctypes.c_int64)]
    I64P = ctypes.POINTER(ctypes.c_int64)
    lib.rom_batch_init.argtypes = [ctypes.POINTER(RomConfigC), ctypes.POINTER(D), ctypes.c_int32, P,
                                   ctypes.POINTER(P)]
    lib.rom_batch_step.argtypes = [P, ctypes.c_int64]
    lib.rom_batch_state.argtypes = [P, ctypes.c_int32, D, D, D, D, D, I64P]
    lib.rom_batch_info.argtypes = [P, ctypes.c_int32, I32P, I32P, I32P]
    lib.rom_batch_layout.argtypes = [P, I64P, I64P, I32P, I32P, I32P, I32P]
    lib.rom_batch_profile.argtypes = [P, ctypes.c_int32]
    lib.rom_batch_profile_read.argtypes = [P, D, I64P]
    lib.rom_batch_work.argtypes = [P, I64P, D]
    lib.rom_batch_fom_work.argtypes = [P, I64P, D]
    lib.rom_batch_destroy.argtypes = [P]
    lib.rom_batch_destroy.restype = None
    for name in ["rom_batch_init", "rom_batch_step", "rom_batch_state", "rom_batch_info",
                 "rom_batch_layout", "rom_batch_profile", "rom_batch_profile_read", "rom_batch_work",
                 "rom_batch_fom_work", "rom_fom_step_noalloc_dev", "rom_profile", "rom_profile_read", "rom_init", "rom_step", "rom_update_basis", "rom_state", "rom_load_state",
                 "rom_samples", "rom_info", "rom_fom_rhs_dev", "rom_fom_step_dev",
                 "rom_isvd_update_dev", "rom_debug_set_wait_limit", "rom_adjoint"]:
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def status_string(code: int) -> str:
    return load().rom_status_string(code).decode()


def check(code: int, what: str):
    if code != ROM_OK:
        raise RomError(code, what)
