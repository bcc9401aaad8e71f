"""ctypes declarations of libnefty's C ABI (include/nefty.h).

This module only marshals arguments.  The library is loaded from this package
directory; if it is missing the import of any compute entry point fails with an
error that says how to build it (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnefty.so")

NEFTY_OK, NEFTY_EINVAL, NEFTY_ENOMEM, NEFTY_ENOTCONV = 0, 1, 2, 3
NEFTY_ECUDA, NEFTY_ETIMEOUT, NEFTY_EBUSY, NEFTY_ECANCELLED, NEFTY_ENOTFOUND = 4, 5, 6, 7, 8
NEFTY_FP32, NEFTY_FP64 = 0, 1
NEFTY_BC_NEUMANN, NEFTY_BC_PERIODIC_XY = 0, 1


class nefty_problem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("dt", ctypes.c_double), ("nt", ctypes.c_int32), ("bc", ctypes.c_int32),
                ("robin_h", ctypes.c_double), ("obs_face", ctypes.c_int32), ("prec", ctypes.c_int32),
                ("rtol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("ckpt_every", ctypes.c_int32),
                ("loss_scale", ctypes.c_double), ("extrap", ctypes.c_int32),
                ("jacobi_k", ctypes.c_int32), ("residual", ctypes.c_int32)]


class nefty_field_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("n_freq", ctypes.c_int32), ("width", ctypes.c_int32), ("depth", ctypes.c_int32),
                ("freq_lo", ctypes.c_double), ("freq_hi", ctypes.c_double),
                ("alpha_min", ctypes.c_double), ("alpha_max", ctypes.c_double),
                ("skip_layer", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("keep_activations", ctypes.c_int32)]


class nefty_stats(ctypes.Structure):
    _fields_ = [("fwd_iters", ctypes.c_int64), ("recompute_iters", ctypes.c_int64),
                ("adj_iters", ctypes.c_int64), ("fwd_steps", ctypes.c_int32),
                ("recompute_steps", ctypes.c_int32), ("adj_steps", ctypes.c_int32),
                ("max_step_iters", ctypes.c_int32), ("not_converged", ctypes.c_int32),
                ("ckpt_every", ctypes.c_int32), ("n_checkpoints", ctypes.c_int32),
                ("max_rel_residual", ctypes.c_double), ("workspace_bytes", ctypes.c_uint64),
                ("grid_blocks", ctypes.c_int32), ("kernel_launches", ctypes.c_int32),
                ("fwd_ms", ctypes.c_double), ("recompute_ms", ctypes.c_double),
                ("adj_ms", ctypes.c_double), ("tma_staged", ctypes.c_int32), ("folded_last_iters", ctypes.c_int32),
                ("carried_solves", ctypes.c_int32)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


NEFTY_JOB_FORWARD, NEFTY_JOB_INVERSION = 0, 1
NEFTY_JOB_QUEUED, NEFTY_JOB_RUNNING, NEFTY_JOB_DONE, NEFTY_JOB_FAILED, NEFTY_JOB_CANCELLED = 0, 1, 2, 3, 4


class nefty_job(ctypes.Structure):
    _fields_ = [("problem", nefty_problem), ("kind", ctypes.c_int32), ("iters", ctypes.c_int32),
                ("lr", ctypes.c_double), ("alpha_floor", ctypes.c_double), ("alpha", ctypes.c_void_p),
                ("T0", ctypes.c_void_p), ("q_face", ctypes.c_void_p), ("q_steps", ctypes.c_int32),
                ("q_full", ctypes.c_void_p), ("obs", ctypes.c_void_p), ("frames_out", ctypes.c_void_p)]


class nefty_job_result(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int32), ("lane", ctypes.c_int32),
                ("iters_done", ctypes.c_int32), ("t_submit_ns", ctypes.c_uint64), ("t_admit_ns", ctypes.c_uint64),
                ("t_done_ns", ctypes.c_uint64), ("loss", ctypes.c_double), ("launches", ctypes.c_int32),
                ("shared_launches", ctypes.c_int32)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class nefty_serve_config(ctypes.Structure):
    _fields_ = [("lanes", ctypes.c_int32), ("max_queue", ctypes.c_int32), ("mem_budget_bytes", ctypes.c_uint64),
                ("batched", ctypes.c_int32), ("chunk_steps", ctypes.c_int32), ("launch_us", ctypes.c_int32)]


class NeftyError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{status_name(status)}: {message}")
        self.status = status


_lock = threading.Lock()
_lib = None

_vp = ctypes.c_void_p
_P = ctypes.POINTER(nefty_problem)
_ST = ctypes.POINTER(nefty_stats)
_SIGNATURES = {
    "nefty_create": ([ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_uint64], ctypes.c_int),
    "nefty_destroy": ([_vp], ctypes.c_int),
    "nefty_last_error": ([_vp], ctypes.c_char_p),
    "nefty_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "nefty_problem_check": ([_P], ctypes.c_int),
    "nefty_debug_barrier_fault": ([_vp, ctypes.c_uint32, ctypes.c_uint64], ctypes.c_int),
    "nefty_forward": ([_vp, _P, _vp, _vp, _vp, ctypes.c_int32, _vp, _vp, _vp, _vp,
                       ctypes.POINTER(ctypes.c_double), _ST, _vp], ctypes.c_int),
    "nefty_adjoint_grad": ([_vp, _P, _vp, _vp, _vp, ctypes.c_int32, _vp, _vp,
                            ctypes.POINTER(ctypes.c_double), _vp, _vp, _ST, _vp], ctypes.c_int),
    "nefty_field_param_count": ([ctypes.c_void_p], ctypes.c_uint64),
    "nefty_field_activation_reuses": ([_vp], ctypes.c_uint64),
    "nefty_field_eval": ([_vp, _vp, _vp, _vp, _vp, _vp], ctypes.c_int),
    "nefty_field_backward": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp], ctypes.c_int),
    "nefty_gemm_bf16": ([_vp, _vp, ctypes.c_int32, _vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                         ctypes.c_int32, _vp, _vp], ctypes.c_int),
    "nefty_tv": ([_vp, _P, _vp, ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double), _vp, _vp],
                 ctypes.c_int),
    "nefty_forward_static": ([ctypes.c_int, _P, _vp, _vp, _vp, ctypes.c_int32, _vp, _vp, _vp,
                              ctypes.POINTER(ctypes.c_double), _vp], ctypes.c_int),
    "nefty_serve_start": ([_vp, ctypes.POINTER(nefty_serve_config)], ctypes.c_int),
    "nefty_serve_submit": ([_vp, ctypes.POINTER(nefty_job), ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "nefty_serve_poll": ([_vp, ctypes.c_uint64, ctypes.POINTER(nefty_job_result)], ctypes.c_int),
    "nefty_serve_cancel": ([_vp, ctypes.c_uint64], ctypes.c_int),
    "nefty_serve_stop": ([_vp], ctypes.c_int),
}


def load():
    """Load libnefty.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(
                    f"libnefty.so not found at {LIB_PATH}; build it with "
                    "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc, sm_103a)")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in _SIGNATURES.items():
                fn = getattr(lib, name, None)
                if fn is None:
                    continue
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def status_name(status: int) -> str:
    try:
        return load().nefty_status_string(int(status)).decode()
    except ImportError:
        return f"status {status}"


def check(status: int, handle=None, allow=()):
    if status == NEFTY_OK or status in allow:
        return status
    msg = load().nefty_last_error(handle).decode(errors="replace")
    raise NeftyError(status, msg)
