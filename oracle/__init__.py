"""FP64 CPU oracle for the NeFTY hot path.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product library never
imports this package and shares no code with it.

``nefty_oracle.c`` (plain C, FP64, no fast-math) implements the paper's
definitions: CSR assembly of A(alpha) = I - dt L(alpha) with harmonic-mean face
conductances (Prop. 1, App. D.2), one CG solve per implicit-Euler step to a
1e-14 relative residual (Eq. state_eq) or, as the paper's own inner solver,
a fixed number K of Jacobi sweeps from the warm start (Eq. jacobi_iter), the reverse-time adjoint with A^T formed
by transposition (Eq. adjoint_eq), the gradient through the explicitly assembled
Jacobian d(L T)/d alpha (Eq. grad_assembly) and the discrete TV (Eq.
tv_discrete).  ``field.py`` holds the FP64 neural-field reference (Sec. 4.1,
App. D.1).  This module is the ctypes marshalling around the C code.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nefty_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_LOCK = threading.Lock()
_LIB = None

DEFAULT_TOL = 1e-14
DEFAULT_MAX_ITER = 20000


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, IEEE semantics, OpenMP loops)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Problem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("dt", ctypes.c_double), ("nt", ctypes.c_int), ("bc", ctypes.c_int),
                ("robin_h", ctypes.c_double), ("obs_face", ctypes.c_int),
                ("loss_scale", ctypes.c_double)]


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(_Problem)
            vp = ctypes.c_void_p
            lib.orc_assemble_A.argtypes = [P, vp, vp, vp, vp, vp]
            lib.orc_assemble_A.restype = ctypes.c_int
            lib.orc_apply_L.argtypes = [P, vp, vp, vp]
            lib.orc_apply_L.restype = ctypes.c_int
            lib.orc_forward.argtypes = [P, vp, vp, vp, ctypes.c_int, vp, vp, vp, vp, vp, vp,
                                        ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            lib.orc_forward.restype = ctypes.c_int
            lib.orc_adjoint_grad.argtypes = [P, vp, vp, vp, ctypes.c_int, vp, vp, vp, vp, vp,
                                             ctypes.c_double, ctypes.c_int, ctypes.c_int]
            lib.orc_adjoint_grad.restype = ctypes.c_int
            lib.orc_tv.argtypes = [P, vp, ctypes.c_double, ctypes.c_double, vp]
            lib.orc_tv.restype = ctypes.c_double
            _LIB = lib
    return _LIB


class OracleError(RuntimeError):
    pass


def problem(nx, ny, nz, dx=1.0, dy=1.0, dz=1.0, dt=0.5, nt=1, bc=0, robin_h=0.0, obs_face=0,
            loss_scale=None) -> _Problem:
    if loss_scale is None:
        loss_scale = 1.0 / (nt * nx * ny)
    return _Problem(nx, ny, nz, dx, dy, dz, dt, nt, bc, robin_h, obs_face, loss_scale)


def from_workload(w, **kw) -> _Problem:
    args = dict(nx=w.nx, ny=w.ny, nz=w.nz, dx=w.dx, dy=w.dy, dz=w.dz, dt=w.dt, nt=w.nt, bc=w.bc)
    args.update(kw)
    return problem(**args)


def _f64(a, n=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise OracleError(f"expected {n} values, got {a.size}")
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _n(p):
    return p.nx * p.ny * p.nz


def assemble_A(p: _Problem, alpha):
    """Return A(alpha) = I - dt L(alpha) as a scipy CSR matrix."""
    import scipy.sparse as sp
    lib = _lib()
    N = _n(p)
    alpha = _f64(alpha, N)
    nnz = ctypes.c_int64(0)
    rc = lib.orc_assemble_A(ctypes.byref(p), _ptr(alpha), None, None, None, ctypes.byref(nnz))
    if rc:
        raise OracleError(f"assemble rc={rc}")
    rp = np.zeros(N + 1, np.int64)
    ci = np.zeros(nnz.value, np.int32)
    v = np.zeros(nnz.value, np.float64)
    rc = lib.orc_assemble_A(ctypes.byref(p), _ptr(alpha), _ptr(rp), _ptr(ci), _ptr(v), ctypes.byref(nnz))
    if rc:
        raise OracleError(f"assemble rc={rc}")
    return sp.csr_matrix((v, ci, rp), shape=(N, N))


def apply_L(p: _Problem, alpha, T):
    N = _n(p)
    alpha, T = _f64(alpha, N), _f64(T, N)
    out = np.zeros(N)
    rc = _lib().orc_apply_L(ctypes.byref(p), _ptr(alpha), _ptr(T), _ptr(out))
    if rc:
        raise OracleError(f"apply_L rc={rc}")
    return out


def forward(p: _Problem, alpha, T0=None, q_face=None, q_steps=0, q_full=None, obs=None,
            keep_states=False, tol=DEFAULT_TOL, max_iter=DEFAULT_MAX_ITER, dense=False, jacobi_k=0):
    """Run the implicit-Euler forward sweep; returns dict(frames, loss, states, iters).
    jacobi_k > 0: each step is jacobi_k Jacobi sweeps from T^n (App. D.2) instead
    of a converged solve."""
    N, S = _n(p), p.nx * p.ny
    alpha = _f64(alpha, N)
    T0 = _f64(T0, N)
    q_face = _f64(q_face, S)
    q_full = _f64(q_full, p.nt * S)
    obs = _f64(obs, p.nt * S)
    frames = np.zeros((p.nt, p.ny, p.nx))
    states = np.zeros((p.nt + 1, p.nz, p.ny, p.nx)) if keep_states else None
    loss = ctypes.c_double(0.0)
    iters = np.zeros(p.nt, np.int32)
    rc = _lib().orc_forward(ctypes.byref(p), _ptr(alpha), _ptr(T0), _ptr(q_face), int(q_steps),
                            _ptr(q_full), _ptr(obs), _ptr(frames), _ptr(states), ctypes.byref(loss),
                            _ptr(iters), tol, max_iter, 1 if dense else 0, int(jacobi_k))
    if rc:
        raise OracleError(f"forward rc={rc}")
    return {"frames": frames, "loss": loss.value if obs is not None else None,
            "states": states, "iters": iters}


def adjoint_grad(p: _Problem, alpha, T0=None, q_face=None, q_steps=0, q_full=None, obs=None,
                 tol=DEFAULT_TOL, max_iter=DEFAULT_MAX_ITER, jacobi_k=0):
    """Loss, dJ/dalpha and dJ/dT0 by the discrete adjoint; returns a dict.
    jacobi_k > 0: every forward and adjoint solve is jacobi_k Jacobi sweeps
    from its warm start (T^n, mu^(n+1)), the paper's inner solver."""
    N, S = _n(p), p.nx * p.ny
    alpha = _f64(alpha, N)
    T0 = _f64(T0, N)
    q_face = _f64(q_face, S)
    q_full = _f64(q_full, p.nt * S)
    obs = _f64(obs, p.nt * S)
    grad = np.zeros((p.nz, p.ny, p.nx))
    gT0 = np.zeros((p.nz, p.ny, p.nx))
    loss = ctypes.c_double(0.0)
    rc = _lib().orc_adjoint_grad(ctypes.byref(p), _ptr(alpha), _ptr(T0), _ptr(q_face), int(q_steps),
                                 _ptr(q_full), _ptr(obs), ctypes.byref(loss), _ptr(grad), _ptr(gT0),
                                 tol, max_iter, int(jacobi_k))
    if rc:
        raise OracleError(f"adjoint rc={rc}")
    return {"loss": loss.value, "grad_alpha": grad, "grad_T0": gT0}


def tv(p: _Problem, alpha, lam, eps, want_grad=True):
    """lam * R(alpha) of Eq. tv_discrete and (optionally) its gradient."""
    N = _n(p)
    alpha = _f64(alpha, N)
    grad = np.zeros((p.nz, p.ny, p.nx)) if want_grad else None
    val = _lib().orc_tv(ctypes.byref(p), _ptr(alpha), float(lam), float(eps), _ptr(grad))
    return val, grad
