"""ctypes binding of libssa.so: the C ABI of include/ssa.h, same names.

Argument marshalling only -- every computation runs in the library's CUDA
kernels.  Loading fails loudly when the library is missing: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

SSA_OK, SSA_EINVAL, SSA_EEMPTY, SSA_ERANK, SSA_ENOMEM = 0, -1, -2, -3, -4
SSA_ENOTCONV, SSA_ETIMEOUT, SSA_ECUDA, SSA_ESTATE, SSA_EUNSUPPORTED = -5, -6, -7, -8, -9
SSA_1D, SSA_MSSA, SSA_2D = 0, 1, 2
SSA_F32, SSA_F64 = 0, 1
SSA_PREC_FP32FFT_FP64REORTH, SSA_PREC_FP64 = 0, 1

EXPORTS = [
    "ssa_embed", "ssa_embed_batch", "ssa_decompose", "ssa_decompose_batch", "ssa_continue", "ssa_get_info", "ssa_get_sigma",
    "ssa_get_vectors", "ssa_reconstruct", "ssa_reconstruct_batch", "ssa_wcor", "ssa_forecast", "ssa_forecast_vector", "ssa_forecast_row", "ssa_get_shape", "ssa_matvec",
    "ssa_synchronize", "ssa_destroy", "ssa_strerror", "ssa_last_error", "ssa_version",
    "ssa_profile_enable", "ssa_profile_reset", "ssa_profile_read", "ssa_kernel_launches",
    "ssa_matvec_series_noalloc", "ssa_noalloc_last_error", "ssa_autotune", "ssa_plans_export", "ssa_plans_import",
    "ssa_server_create", "ssa_server_submit", "ssa_server_step", "ssa_server_stats", "ssa_server_finished", "ssa_server_take",
    "ssa_server_clock", "ssa_server_destroy",
]
PHASES = ["shapes", "spectrum", "matvec", "short", "long", "ritz", "recon"]


class ssa_input(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dtype", C.c_int32), ("on_device", C.c_int32),
                ("n_series", C.c_int32), ("data", C.c_void_p), ("n", C.c_int64),
                ("lengths", C.POINTER(C.c_int64)), ("nx", C.c_int64), ("ny", C.c_int64),
                ("mask", C.c_void_p)]


class ssa_window(C.Structure):
    _fields_ = [("L", C.c_int64), ("lx", C.c_int64), ("ly", C.c_int64), ("wmask", C.c_void_p)]


class ssa_params(C.Structure):
    _fields_ = [("rank", C.c_int32), ("krylov_dim", C.c_int32), ("max_restarts", C.c_int32),
                ("prec", C.c_int32), ("tol", C.c_double), ("seed", C.c_uint64)]


class ssa_info(C.Structure):
    _fields_ = [("L", C.c_int64), ("K", C.c_int64), ("nx", C.c_int64), ("ny", C.c_int64),
                ("n_channels", C.c_int32), ("rank", C.c_int32), ("krylov_dim", C.c_int32),
                ("restarts", C.c_int32), ("converged", C.c_int32), ("prec", C.c_int32),
                ("fft_mx", C.c_int64), ("fft_my", C.c_int64), ("max_residual", C.c_double),
                ("device_bytes", C.c_int64), ("jacobi_sweeps", C.c_int32), ("jacobi_sweeps_fp32", C.c_int32),
                ("breakdowns", C.c_int32), ("pad_", C.c_int32)]


class ssa_tune_result(C.Structure):
    _fields_ = [("krylov_dim", C.c_int32), ("ytk", C.c_int32), ("n_tried", C.c_int32), ("pad_", C.c_int32),
                ("ms_default", C.c_double), ("ms_best", C.c_double)]


class ssa_server_config(C.Structure):
    _fields_ = [("memory_budget", C.c_int64), ("max_live", C.c_int32), ("prec", C.c_int32)]


class ssa_server_result(C.Structure):
    _fields_ = [("ticket", C.c_int64), ("status", C.c_int32), ("rank", C.c_int32), ("out_len", C.c_int64),
                ("restarts", C.c_int32), ("pad_", C.c_int32), ("max_residual", C.c_double),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double),
                ("device_bytes", C.c_int64), ("estimated_bytes", C.c_int64)]


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> C.CDLL:
    """Load libssa.so (building it first when asked); raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libssa.so not found at {path}; run __graft_entry__.build()")
    lib = C.CDLL(path)
    P = C.c_void_p
    lib.ssa_embed.argtypes = [C.POINTER(ssa_input), C.POINTER(ssa_window), P, C.POINTER(P)]
    lib.ssa_embed_batch.argtypes = [C.POINTER(ssa_input), C.POINTER(ssa_window), C.c_int32, P, C.POINTER(P),
                                    C.POINTER(C.c_int32)]
    lib.ssa_decompose.argtypes = [P, C.POINTER(ssa_params)]
    lib.ssa_continue.argtypes = [P, C.POINTER(ssa_params)]
    lib.ssa_decompose_batch.argtypes = [C.POINTER(P), C.c_int32, C.POINTER(ssa_params), C.POINTER(C.c_int32)]
    lib.ssa_get_info.argtypes = [P, C.POINTER(ssa_info)]
    lib.ssa_get_sigma.argtypes = [P, C.POINTER(C.c_double), C.c_int32]
    lib.ssa_get_vectors.argtypes = [P, P, P, C.c_int32]
    lib.ssa_reconstruct.argtypes = [P, C.POINTER(C.c_int32), C.c_int32, C.c_int32, P, C.c_int32]
    lib.ssa_wcor.argtypes = [P, C.POINTER(C.c_int32), C.c_int32, P, P]
    lib.ssa_forecast.argtypes = [P, C.POINTER(C.c_int32), C.c_int32, C.c_int32, P]
    lib.ssa_forecast_vector.argtypes = [P, C.POINTER(C.c_int32), C.c_int32, C.c_int32, P]
    lib.ssa_forecast_row.argtypes = [P, C.POINTER(C.c_int32), C.c_int32, C.c_int32, C.c_int32, P]
    lib.ssa_reconstruct_batch.argtypes = [C.POINTER(P), C.c_int32, C.POINTER(C.c_int32), C.c_int32,
                                          C.c_int32, C.POINTER(P), C.c_int32]
    lib.ssa_get_shape.argtypes = [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), P, P]
    lib.ssa_matvec.argtypes = [P, C.c_int32, C.c_int32, P, P, C.c_int32]
    lib.ssa_synchronize.argtypes = [P]
    lib.ssa_destroy.argtypes = [P]
    lib.ssa_destroy.restype = None
    lib.ssa_strerror.argtypes = [C.c_int]
    lib.ssa_strerror.restype = C.c_char_p
    lib.ssa_last_error.argtypes = []
    lib.ssa_last_error.restype = C.c_char_p
    lib.ssa_version.restype = C.c_char_p
    lib.ssa_profile_enable.argtypes = [C.c_int32]
    lib.ssa_profile_reset.argtypes = []
    lib.ssa_profile_read.argtypes = [C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    lib.ssa_kernel_launches.argtypes = []
    lib.ssa_kernel_launches.restype = C.c_int64
    lib.ssa_matvec_series_noalloc.argtypes = [P, C.c_int64, C.c_int64, C.c_int32, P, P, P]
    lib.ssa_noalloc_last_error.argtypes = []
    lib.ssa_noalloc_last_error.restype = C.c_char_p
    lib.ssa_autotune.argtypes = [P, C.POINTER(ssa_params), C.POINTER(ssa_tune_result)]
    lib.ssa_plans_export.argtypes = [C.c_char_p, C.c_int64, C.POINTER(C.c_int64)]
    lib.ssa_plans_import.argtypes = [C.c_char_p]
    lib.ssa_server_create.argtypes = [C.POINTER(ssa_server_config), P, C.POINTER(P)]
    lib.ssa_server_submit.argtypes = [P, C.POINTER(ssa_input), C.POINTER(ssa_window), C.POINTER(ssa_params),
                                      P, C.c_int32, C.c_int32, C.POINTER(C.c_int64)]
    lib.ssa_server_step.argtypes = [P, C.POINTER(C.c_int32)]
    lib.ssa_server_stats.argtypes = [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                     C.POINTER(C.c_int64)]
    lib.ssa_server_finished.argtypes = [P, C.POINTER(C.c_int64), C.c_int32, C.POINTER(C.c_int32)]
    lib.ssa_server_take.argtypes = [P, C.c_int64, C.POINTER(ssa_server_result), P, P]
    lib.ssa_server_clock.argtypes = [P]
    lib.ssa_server_clock.restype = C.c_double
    lib.ssa_server_destroy.argtypes = [P]
    lib.ssa_server_destroy.restype = None
    _lib = lib
    return lib


class SSAError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = load(False)
        msg = lib.ssa_strerror(code).decode()
        detail = lib.ssa_last_error().decode()
        super().__init__(f"{where}: {msg} ({code}): {detail}")
        self.code = code


def check(rc: int, where: str) -> int:
    if rc != SSA_OK:
        raise SSAError(rc, where)
    return rc


def profile_enable(on: bool = True) -> None:
    check(load().ssa_profile_enable(1 if on else 0), "ssa_profile_enable")


def profile_reset() -> None:
    check(load().ssa_profile_reset(), "ssa_profile_reset")


def profile_read() -> dict:
    """{phase: (device ms, kernel launches, phase instances)} since the last reset."""
    lib = load()
    out = {}
    for i, name in enumerate(PHASES):
        ms, la, ca = C.c_double(), C.c_int64(), C.c_int64()
        check(lib.ssa_profile_read(i, C.byref(ms), C.byref(la), C.byref(ca)), "ssa_profile_read")
        out[name] = (ms.value, la.value, ca.value)
    return out


def kernel_launches() -> int:
    return int(load().ssa_kernel_launches())


def matvec_series_noalloc(x, L: int, v, out, transpose: bool = False, stream=None) -> None:
    """Hankel trajectory-matrix product of one FP32 series without any device
    allocation (see ssa_matvec_series_noalloc in include/ssa.h).  x, v, out are
    CUDA float32 tensors owned by the caller."""
    lib = load()
    sp = None if stream is None else C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    rc = lib.ssa_matvec_series_noalloc(x.data_ptr(), int(x.numel()), int(L), 1 if transpose else 0,
                                       v.data_ptr(), out.data_ptr(), sp)
    if rc != SSA_OK:
        raise RuntimeError(f"ssa_matvec_series_noalloc: {lib.ssa_strerror(rc).decode()} ({rc}): "
                           f"{lib.ssa_noalloc_last_error().decode()}")


def plans_export() -> str:
    """The tuned plans (ssa_plans_export) as text."""
    lib = load()
    n = C.c_int64()
    check(lib.ssa_plans_export(None, 0, C.byref(n)), "ssa_plans_export")
    buf = C.create_string_buffer(int(n.value) + 1)
    check(lib.ssa_plans_export(buf, int(n.value) + 1, C.byref(n)), "ssa_plans_export")
    return buf.value.decode()


def plans_import(text: str) -> None:
    check(load().ssa_plans_import(text.encode()), "ssa_plans_import")
