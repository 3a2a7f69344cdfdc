"""ctypes binding of libspuma.so (the C ABI in include/spuma.h).

Argument marshalling only: every step of the solve runs in the library's CUDA
kernels.  Tensors are passed by device pointer, streams as the current torch
stream.  The library must have been built (``paper_2512_22215_gb300.build``);
loading fails loudly otherwise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libspuma.so")

SPUMA_OK = 0
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "NOT_UPPER_TRIANGULAR", 3: "CUDA", 4: "WORKSPACE_TOO_SMALL",
                5: "SINGULAR", 6: "NOT_SPD", 7: "NONFINITE", 8: "DEVICE_TIMEOUT", 9: "HOST"}
F64, MIXED, F32, MIXED_RESTART = 0, 1, 2, 3
PRECOND_NONE, PRECOND_DIAGONAL, PRECOND_DIC, PRECOND_DILU = 0, 1, 2, 3
WORKSPACE_ASYMMETRIC = 1
BATCH_AUTOTUNE, BATCH_ALLOW_DIRECT, BATCH_NO_GRAPH = 1, 2, 4
GAMG_RICHARDSON, GAMG_GAUSS_SEIDEL_2STAGE = 0, 1


class Controls(C.Structure):
    _fields_ = [("precond", C.c_int32), ("precision", C.c_int32), ("tolerance", C.c_double),
                ("rel_tol", C.c_double), ("inner_rel_tol", C.c_double), ("max_iter", C.c_int32),
                ("min_iter", C.c_int32), ("max_outer", C.c_int32), ("block_threads", C.c_int32)]


class Perf(C.Structure):
    _fields_ = [("initial_residual", C.c_double), ("final_residual", C.c_double),
                ("true_rel_residual_l2", C.c_double), ("n_iter", C.c_int32), ("n_outer", C.c_int32),
                ("converged", C.c_int32), ("singular", C.c_int32), ("status", C.c_int32), ("n_levels", C.c_int32)]


PERF_BYTES = C.sizeof(Perf)
assert PERF_BYTES == 48


class SpumaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"spuma: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None

_P = C.c_void_p
_I = C.c_int32
_H = C.c_void_p
_SIGS = {
    "spuma_workspace_bytes": (C.c_size_t, [_I, _I, _I]),
    "spuma_ldu_create": (_I, [_I, _I, _P, _P, _P, C.c_size_t, _P, C.POINTER(_H)]),
    "spuma_ldu_create_with_centres": (_I, [_I, _I, _P, _P, _P, _P, C.c_size_t, _P, C.POINTER(_H)]),
    "spuma_ldu_destroy": (_I, [_H]),
    "spuma_ldu_info": (_I, [_H, C.POINTER(_I), C.POINTER(_I), C.POINTER(_I)]),
    "spuma_ldu_device_status": (_I, [_H, _P]),
    "spuma_assemble_laplacian": (_I, [_H, _P, _P, _P, _I, _P, _P, _P, _P, _P, _P, _P, _P]),
    "spuma_assemble_laplacian_adjoint": (_I, [_H, _P, _P, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "spuma_amul": (_I, [_H, _I, _P, _P, _P, _P, _P]),
    "spuma_fv_weights": (_I, [_H, _P, _P, _P, _P, _P]),
    "spuma_fv_grad": (_I, [_H, _P, _P, _P, _I, _P, _P, _P, _P, _P, _P]),
    "spuma_pressure_rhs": (_I, [_H, _P, _P, _P, _P, _P, _P, _I, _P, _P, _P, _P, _P]),
    "spuma_pressure_flux": (_I, [_H, _P, _P, _P, _P, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "spuma_fv_div": (_I, [_H, _P, _I, _P, _P, _P, _P]),
    "spuma_matrix_prepare": (_I, [_H, _P, _P, _I, _P]),
    "spuma_read_rD": (_I, [_H, _P, _P]),
    "spuma_amul_prepared": (_I, [_H, _I, _P, _P, _P]),
    "spuma_permute": (_I, [_H, _I, _P, _P, _P]),
    "spuma_precondition": (_I, [_H, _I, _P, _P, _P]),
    "spuma_pcg_solve": (_I, [_H, _P, _P, _P, _P, C.POINTER(Controls), _P, _P]),
    "spuma_static_workspace_bytes": (C.c_size_t, []),
    "spuma_pcg_solve_static": (_I, [_I, _I, _P, _P, _P, _P, _P, _P, C.POINTER(Controls), _P, _P]),
    "spuma_gamg_create": (_I, [_H, _P, _P, C.POINTER(_H)]),
    "spuma_gamg_workspace_bytes": (C.c_size_t, [_H]),
    "spuma_gamg_bind": (_I, [_H, _P, C.c_size_t, _P]),
    "spuma_gamg_info": (_I, [_H, C.POINTER(_I), _P, _I]),
    "spuma_gamg_solve": (_I, [_H, _P, _P, _P, _P, C.POINTER(Controls), _P, _P]),
    "spuma_gamg_set_options": (_I, [_H, _I, _I]),
    "spuma_gamg_destroy": (_I, [_H]),
    "spuma_pbicg_solve": (_I, [_H, _P, _P, _P, _P, _P, C.POINTER(Controls), _P, _P]),
    "spuma_pcg_adjoint": (_I, [_H, _P, _P, _P, _P, _P, _P, _P, C.POINTER(Controls), _P, _P]),
    "spuma_batch_create": (_I, [_I, C.POINTER(_H), C.POINTER(_P), C.POINTER(_P), C.POINTER(_P), C.POINTER(_P),
                                C.POINTER(Controls), _P, _I, _P, C.POINTER(_H)]),
    "spuma_batch_run": (_I, [_H, _P]),
    "spuma_batch_info": (_I, [_H, C.POINTER(_I), C.POINTER(_I), C.POINTER(C.c_double), C.POINTER(_I)]),
    "spuma_batch_trials": (_I, [_H, _I, _P, _P, _P, _P]),
    "spuma_batch_destroy": (_I, [_H]),
    "spuma_batch_solve": (_I, [_I, C.POINTER(_H), C.POINTER(_P), C.POINTER(_P), C.POINTER(_P), C.POINTER(_P),
                               C.POINTER(Controls), _P, _P]),
    "spuma_batch_split": (_I, [_I, C.POINTER(C.c_double), _I, C.POINTER(_I)]),
    "spuma_tune_cache_lookup": (_I, [C.c_char_p, C.c_char_p, C.POINTER(_I), C.POINTER(_I), C.POINTER(_I),
                                     C.POINTER(C.c_double)]),
    "spuma_tune_cache_store": (_I, [C.c_char_p, C.c_char_p, _I, _I, _I, C.c_double]),
    "spuma_read_phase_clocks": (_I, [_H, C.POINTER(C.c_int64), _I, _P]),
    "spuma_status_string": (C.c_char_p, [_I]),
    "spuma_last_error": (C.c_char_p, []),
    "spuma_launch_count": (C.c_uint64, []),
    "spuma_set_barrier_timeout_ns": (None, [C.c_uint64]),
}


def lib():
    """Load libspuma.so; raise if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libspuma.so not built at {LIB_PATH}: run "
                               "python -c 'import __graft_entry__ as g; g.build()'")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int, what: str = ""):
    if status != SPUMA_OK:
        msg = lib().spuma_last_error().decode(errors="replace")
        raise SpumaError(status, f"{what}: {msg}")


def ptr(t) -> int | None:
    """Device pointer of a torch tensor (None for None / empty)."""
    if t is None:
        return None
    return t.data_ptr() if t.numel() > 0 else None


def stream_ptr(stream=None) -> int | None:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream or None
