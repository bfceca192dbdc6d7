"""ctypes binding of ``libpoisson.so`` (include/poisson.h): argument marshalling only.

Every step of the solve runs in the library's CUDA kernels; this module only converts torch
tensors to device pointers and the current torch stream to a ``cudaStream_t``.  There is no
fallback: if the library is missing the import of ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpoisson.so")

PS_OK, PS_EINVAL, PS_EUNSUPPORTED, PS_ENOMEM, PS_ECUDA, PS_ETIMEOUT, PS_ENONFINITE, PS_ENOWORKSPACE = range(8)
PP_FP64, PP_FP32, PP_FP32_REFINED = 0, 1, 2
PT_AUTO, PT_THOMAS, PT_PDD_EXACT, PT_PDD_TRUNCATED = 0, 1, 2, 3
POISSON_STATIC_WS_MAX_BYTES = 8 * 1024 * 1024
POISSON_CHECK_FINITE = 0x1
POISSON_TIMING = 0x2
POISSON_GENERIC_FFT = 0x4
POISSON_SELFTEST_WAIT = 0x8
POISSON_BATCH_PERSISTENT = 0x10

# Every symbol declared in include/poisson.h.
EXPORTS = (
    "poisson_plan_create", "poisson_workspace_size", "poisson_set_workspace", "poisson_solve",
    "poisson_solve_adjoint", "poisson_solve_static_ws", "poisson_plan_batched", "poisson_solve_batched", "poisson_autotune",
    "projection_step", "projection_step_adjoint", "projection_step_host", "momentum_predictor",
    "projection_timestep", "projection_timestep_host", "poisson_divergence", "poisson_plan_set_chain",
    "poisson_fp64_fma_rate", "poisson_device_status",
    "poisson_last_launch_count", "poisson_stage_times", "poisson_plan_destroy", "poisson_status_string",
)


class PoissonDesc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("lx", ctypes.c_double), ("lz", ctypes.c_double),
        ("y_faces", ctypes.POINTER(ctypes.c_double)),
        ("precision", ctypes.c_int), ("tridiag", ctypes.c_int), ("pdd_parts", ctypes.c_int),
        ("fp64_low_modes", ctypes.c_int), ("refine_steps", ctypes.c_int), ("flags", ctypes.c_uint),
    ]


class PoissonError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} (status {code})")


_LIB = None


def lib() -> ctypes.CDLL:
    """Load libpoisson.so (built in-tree by ``paper_2104_08863_gb300.build``); raise if absent."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    L.poisson_plan_create.argtypes = [ctypes.POINTER(PoissonDesc), ctypes.POINTER(vp)]
    L.poisson_workspace_size.argtypes = [vp, ctypes.POINTER(sz)]
    L.poisson_set_workspace.argtypes = [vp, vp, sz, vp]
    L.poisson_solve.argtypes = [vp, vp, vp, vp]
    L.poisson_solve_adjoint.argtypes = [vp, vp, vp, vp]
    L.poisson_solve_static_ws.argtypes = [vp, vp, vp, vp]
    L.poisson_plan_batched.argtypes = [ctypes.POINTER(PoissonDesc), i, ctypes.POINTER(vp)]
    L.poisson_solve_batched.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
    L.poisson_autotune.argtypes = [ctypes.POINTER(PoissonDesc), vp, ctypes.POINTER(i), ctypes.POINTER(ctypes.c_uint),
                                   ctypes.POINTER(ctypes.c_float)]
    L.projection_step.argtypes = [vp, vp, vp, vp, vp, d, vp]
    L.projection_step_adjoint.argtypes = [vp, vp, vp, vp, vp]
    L.projection_step_host.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, d, vp]
    L.momentum_predictor.argtypes = [vp, vp, vp, vp, vp, vp, vp, d, d, d, vp]
    L.projection_timestep.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, d, d, d, vp]
    L.projection_timestep_host.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, d, d, d, vp]
    L.poisson_plan_set_chain.argtypes = [vp, i, i]
    L.poisson_divergence.argtypes = [vp, vp, vp, vp, vp, d, vp]
    L.poisson_fp64_fma_rate.argtypes = [vp, sz, vp, ctypes.POINTER(d)]
    L.poisson_device_status.argtypes = [vp, vp]
    L.poisson_last_launch_count.argtypes = [vp]
    L.poisson_last_launch_count.restype = i
    L.poisson_stage_times.argtypes = [vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_char_p), i]
    L.poisson_stage_times.restype = i
    L.poisson_plan_destroy.argtypes = [vp]
    L.poisson_status_string.argtypes = [i]
    L.poisson_status_string.restype = ctypes.c_char_p
    for name in ("poisson_plan_create", "poisson_workspace_size", "poisson_set_workspace", "poisson_solve",
                 "poisson_solve_adjoint", "poisson_solve_static_ws", "poisson_plan_batched", "poisson_solve_batched", "poisson_autotune",
                 "projection_step", "projection_step_adjoint", "projection_step_host", "momentum_predictor",
                 "projection_timestep", "projection_timestep_host", "poisson_divergence", "poisson_plan_set_chain",
                 "poisson_fp64_fma_rate", "poisson_device_status",
                 "poisson_plan_destroy"):
        getattr(L, name).restype = i
    _LIB = L
    return L


def status_string(code: int) -> str:
    return lib().poisson_status_string(int(code)).decode()


def check(code: int, where: str) -> None:
    if code != PS_OK:
        raise PoissonError(code, where)
