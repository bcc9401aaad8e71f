"""Python face of libnefty: problem description, a handle wrapper and the
autograd Function from alpha to the surface loss.

Every step of the computation runs in libnefty's CUDA kernels; this module
checks shapes and dtypes, allocates outputs with PyTorch and passes raw
pointers.  Arrays may be CUDA tensors (used in place) or CPU tensors / numpy
arrays (copied to the device inside the library call).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, fields, replace
from typing import Optional

import numpy as np
import torch

from . import _native as N

__all__ = ["Problem", "Solver", "HeatLoss", "heat_loss"]


@dataclass
class Problem:
    """Mirror of ``nefty_problem`` (include/nefty.h); zero fields take the C defaults."""
    nx: int
    ny: int
    nz: int
    dx: float = 1.0
    dy: float = 1.0
    dz: float = 1.0
    dt: float = 0.5
    nt: int = 1
    bc: int = N.NEFTY_BC_NEUMANN
    robin_h: float = 0.0
    obs_face: int = 0
    prec: str = "fp32"
    rtol: float = 0.0
    max_iter: int = 0
    ckpt_every: int = 0
    loss_scale: float = 0.0
    extrap: int = 0
    jacobi_k: int = 0
    residual: int = 0     # 0/1 carried start residual (staged FP32 path), -1 formed from the state

    @classmethod
    def from_workload(cls, w, **kw) -> "Problem":
        args = dict(nx=w.nx, ny=w.ny, nz=w.nz, dx=w.dx, dy=w.dy, dz=w.dz, dt=w.dt, nt=w.nt, bc=w.bc)
        args.update(kw)
        return cls(**args)

    def with_(self, **kw) -> "Problem":
        return replace(self, **kw)

    @property
    def n_cells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def torch_dtype(self):
        return torch.float32 if self.prec == "fp32" else torch.float64

    @property
    def np_dtype(self):
        return np.float32 if self.prec == "fp32" else np.float64

    def to_c(self) -> N.nefty_problem:
        if self.prec not in ("fp32", "fp64"):
            raise ValueError("prec must be 'fp32' or 'fp64'")
        p = N.nefty_problem()
        for f in fields(self):
            v = getattr(self, f.name)
            if f.name == "prec":
                v = N.NEFTY_FP32 if v == "fp32" else N.NEFTY_FP64
            setattr(p, f.name, v)
        return p


def _as_array(x, dtype, count, name, allow_none=True):
    """Return (keep-alive object, pointer) for a torch tensor or numpy array."""
    if x is None:
        if allow_none:
            return None, None
        raise ValueError(f"{name} is required")
    if isinstance(x, torch.Tensor):
        if x.dtype != dtype:
            raise TypeError(f"{name}: expected {dtype}, got {x.dtype}")
        if not x.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if x.numel() != count:
            raise ValueError(f"{name}: expected {count} elements, got {x.numel()}")
        return x, ctypes.c_void_p(x.data_ptr())
    a = np.asarray(x)
    want = np.float32 if dtype == torch.float32 else np.float64
    if a.dtype != want:
        raise TypeError(f"{name}: expected {np.dtype(want)}, got {a.dtype}")
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError(f"{name} must be C-contiguous")
    if a.size != count:
        raise ValueError(f"{name}: expected {count} elements, got {a.size}")
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _empty_like_home(ref, shape, dtype):
    """Output array on the same side (device / host) as the reference input."""
    if isinstance(ref, torch.Tensor):
        return torch.empty(shape, dtype=dtype, device=ref.device)
    return torch.empty(shape, dtype=dtype)


def _stream_for(ref, stream):
    if stream is not None:
        return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    if isinstance(ref, torch.Tensor) and ref.is_cuda:
        return ctypes.c_void_p(torch.cuda.current_stream(ref.device).cuda_stream)
    return None


class Solver:
    """Owns one ``nefty_handle`` (device workspace reused across calls)."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0):
        self._lib = N.load()
        h = ctypes.c_void_p()
        N.check(self._lib.nefty_create(ctypes.byref(h), int(device), int(mem_budget_bytes)))
        self._h = h
        self.device = device

    def close(self):
        if getattr(self, "_h", None):
            self._lib.nefty_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def forward(self, prob: Problem, alpha, T0=None, q_face=None, q_steps: int = 0, q_full=None,
                obs=None, frames: bool = True, T_final: bool = False, stream=None,
                allow_notconv: bool = False):
        """Implicit-Euler forward sweep.  Returns dict(frames, T_final, loss, stats)."""
        dt = prob.torch_dtype
        Nc, S = prob.n_cells, prob.nx * prob.ny
        keep = []
        a_obj, a_ptr = _as_array(alpha, dt, Nc, "alpha", allow_none=False)
        t0 = _as_array(T0, dt, Nc, "T0")
        qf = _as_array(q_face, dt, S, "q_face")
        qa = _as_array(q_full, dt, prob.nt * S, "q_full")
        ob = _as_array(obs, dt, prob.nt * S, "obs")
        keep += [a_obj, t0[0], qf[0], qa[0], ob[0]]
        fr = _empty_like_home(alpha, (prob.nt, prob.ny, prob.nx), dt) if frames else None
        tf = _empty_like_home(alpha, (prob.nz, prob.ny, prob.nx), dt) if T_final else None
        loss = ctypes.c_double(0.0)
        st = N.nefty_stats()
        cp = prob.to_c()
        status = self._lib.nefty_forward(
            self._h, ctypes.byref(cp), a_ptr, t0[1], qf[1], int(q_steps), qa[1],
            ctypes.c_void_p(fr.data_ptr()) if fr is not None else None,
            ctypes.c_void_p(tf.data_ptr()) if tf is not None else None,
            ob[1], ctypes.byref(loss) if obs is not None else None, ctypes.byref(st),
            _stream_for(alpha, stream))
        N.check(status, self._h, allow=(N.NEFTY_ENOTCONV,) if allow_notconv else ())
        return {"frames": fr, "T_final": tf, "loss": loss.value if obs is not None else None,
                "stats": st.as_dict(), "status": status}

    def adjoint_grad(self, prob: Problem, alpha, obs, T0=None, q_face=None, q_steps: int = 0,
                     q_full=None, grad_T0: bool = False, stream=None, allow_notconv: bool = False):
        """Loss, dJ/dalpha (and dJ/dT0) by the discrete adjoint."""
        dt = prob.torch_dtype
        Nc, S = prob.n_cells, prob.nx * prob.ny
        a_obj, a_ptr = _as_array(alpha, dt, Nc, "alpha", allow_none=False)
        t0 = _as_array(T0, dt, Nc, "T0")
        qf = _as_array(q_face, dt, S, "q_face")
        qa = _as_array(q_full, dt, prob.nt * S, "q_full")
        ob = _as_array(obs, dt, prob.nt * S, "obs", allow_none=False)
        keep = [a_obj, t0[0], qf[0], qa[0], ob[0]]
        ga = _empty_like_home(alpha, (prob.nz, prob.ny, prob.nx), dt)
        gt = _empty_like_home(alpha, (prob.nz, prob.ny, prob.nx), dt) if grad_T0 else None
        loss = ctypes.c_double(0.0)
        st = N.nefty_stats()
        cp = prob.to_c()
        status = self._lib.nefty_adjoint_grad(
            self._h, ctypes.byref(cp), a_ptr, t0[1], qf[1], int(q_steps), qa[1], ob[1],
            ctypes.byref(loss), ctypes.c_void_p(ga.data_ptr()),
            ctypes.c_void_p(gt.data_ptr()) if gt is not None else None, ctypes.byref(st),
            _stream_for(alpha, stream))
        N.check(status, self._h, allow=(N.NEFTY_ENOTCONV,) if allow_notconv else ())
        del keep
        return {"loss": loss.value, "grad_alpha": ga, "grad_T0": gt, "stats": st.as_dict(),
                "status": status}


    def tv(self, prob: Problem, alpha, lam: float, eps: float, grad_accum=None, stream=None):
        """lam * R(alpha) of Eq. tv_discrete; lam * dR/dalpha is added to grad_accum if given."""
        dt = prob.torch_dtype
        a_obj, a_ptr = _as_array(alpha, dt, prob.n_cells, "alpha", allow_none=False)
        g_obj, g_ptr = _as_array(grad_accum, dt, prob.n_cells, "grad_accum")
        out = ctypes.c_double(0.0)
        cp = prob.to_c()
        N.check(self._lib.nefty_tv(self._h, ctypes.byref(cp), a_ptr, float(lam), float(eps), ctypes.byref(out),
                                   g_ptr, _stream_for(alpha, stream)), self._h)
        del a_obj, g_obj
        return out.value


class HeatLoss(torch.autograd.Function):
    """J(alpha) = loss_scale * sum_n ||Pi T^n(alpha) - obs^n||^2 with the
    gradient from the discrete adjoint (Eq. adjoint_eq, Eq. grad_assembly).

    When alpha requires grad, the forward call runs libnefty's adjoint sweep
    right away (one forward + one reverse sweep in total) and keeps dJ/dalpha
    for backward."""

    @staticmethod
    def forward(ctx, alpha, solver: Solver, prob: Problem, obs, q_face, q_steps, T0):
        if ctx.needs_input_grad[0]:
            out = solver.adjoint_grad(prob, alpha.detach(), obs, T0=T0, q_face=q_face, q_steps=q_steps)
            ctx.save_for_backward(out["grad_alpha"])
        else:
            out = solver.forward(prob, alpha.detach(), T0=T0, q_face=q_face, q_steps=q_steps, obs=obs,
                                 frames=False)
        return torch.tensor(out["loss"], dtype=torch.float64, device=alpha.device)

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return grad * g.to(grad.dtype), None, None, None, None, None, None


def heat_loss(solver: Solver, prob: Problem, alpha: torch.Tensor, obs, q_face=None, q_steps=0, T0=None):
    return HeatLoss.apply(alpha, solver, prob, obs, q_face, q_steps, T0)
