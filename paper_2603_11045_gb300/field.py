"""Neural diffusivity field (Sec. 4.1, App. D.1) on the tensor cores.

``FieldSpec`` mirrors ``nefty_field_desc``; ``field_alpha`` is the autograd
Function from the packed FP32 parameter vector theta to alpha at every cell
(forward: ``nefty_field_eval``; backward: ``nefty_field_backward``);
``NeuralField`` is a module holding theta.  Defaults are the inversion-step
shape: 64 log-spaced bands per axis from pi to 128 pi (384 inputs), 4 hidden
layers of 256, alpha bracketed to [0.01, 2.0].
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

from . import _native as N
from . import synthetic

__all__ = ["FieldSpec", "FieldFn", "field_alpha", "NeuralField", "annealing_weights"]


@dataclass
class FieldSpec:
    nx: int
    ny: int
    nz: int
    n_freq: int = 64
    width: int = 256
    depth: int = 4
    freq_lo: float = math.pi
    freq_hi: float = 128 * math.pi
    alpha_min: float = 0.01
    alpha_max: float = 2.0
    skip_layer: int = 0
    precision: int = 0      # 0: BF16 operands; 1: split BF16 (hi + lo, three products each)
    keep_activations: bool = False   # the evaluation keeps what a backward at the same theta needs

    @classmethod
    def paper(cls, nx: int, ny: int, nz: int, alpha_min: float = 0.003, alpha_max: float = 0.25,
              precision: int = 0) -> "FieldSpec":
        """The paper's field (App. D.4): 12 bands 2^k pi, 10 x 512, skip at layer 4."""
        return cls(nx, ny, nz, n_freq=12, width=512, depth=10, freq_lo=math.pi, freq_hi=2.0 ** 11 * math.pi,
                   alpha_min=alpha_min, alpha_max=alpha_max, skip_layer=4, precision=precision)

    def to_c(self) -> N.nefty_field_desc:
        return N.nefty_field_desc(self.nx, self.ny, self.nz, self.n_freq, self.width, self.depth,
                                  self.freq_lo, self.freq_hi, self.alpha_min, self.alpha_max, self.skip_layer,
                                  self.precision, int(self.keep_activations))

    @property
    def n_params(self) -> int:
        d = self.to_c()
        n = int(N.load().nefty_field_param_count(ctypes.byref(d)))
        if n == 0:
            raise ValueError(f"invalid field description {self}")
        return n


def annealing_weights(n_freq: int, beta: float) -> np.ndarray:
    """Cosine frequency-annealing weights of Eq. fa_schedule (host side)."""
    k = np.arange(n_freq)
    return 0.5 * (1.0 - np.cos(math.pi * np.clip(beta - k, 0.0, 1.0)))


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class FieldFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, solver, spec: FieldSpec, band_weights):
        if theta.dtype != torch.float32 or not theta.is_contiguous():
            raise TypeError("theta must be a contiguous float32 tensor")
        out = torch.empty(spec.nz, spec.ny, spec.nx, dtype=torch.float32, device=theta.device)
        d = spec.to_c()
        bw = None if band_weights is None else band_weights.to(device=theta.device, dtype=torch.float32).contiguous()
        st = solver._lib.nefty_field_eval(solver._h, ctypes.byref(d), _ptr(theta), _ptr(bw), _ptr(out),
                                          _stream(theta))
        N.check(st, solver._h)
        ctx.solver, ctx.spec = solver, spec
        ctx.save_for_backward(theta, bw if bw is not None else torch.empty(0))
        return out

    @staticmethod
    def backward(ctx, g_alpha):
        theta, bw = ctx.saved_tensors
        bw = None if bw.numel() == 0 else bw
        g = g_alpha.to(torch.float32).contiguous()
        grad = torch.empty_like(theta)
        d = ctx.spec.to_c()
        st = ctx.solver._lib.nefty_field_backward(ctx.solver._h, ctypes.byref(d), _ptr(theta), _ptr(bw), _ptr(g),
                                                  _ptr(grad), _stream(theta))
        N.check(st, ctx.solver._h)
        return grad, None, None, None


def _stream(t):
    if t.is_cuda:
        return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)
    return None


def field_alpha(solver, spec: FieldSpec, theta: torch.Tensor, band_weights: Optional[torch.Tensor] = None):
    return FieldFn.apply(theta, solver, spec, band_weights)


class NeuralField(torch.nn.Module):
    """theta (FP32, packed as in nefty.h) with seeded Xavier-uniform init (App. D.1)."""

    def __init__(self, solver, spec: FieldSpec, seed: int = 0, device="cuda"):
        super().__init__()
        self.solver, self.spec = solver, spec
        th = synthetic.xavier_theta(spec.n_freq, spec.width, spec.depth, seed, skip=spec.skip_layer)
        assert th.size == spec.n_params
        self.theta = torch.nn.Parameter(torch.tensor(th, dtype=torch.float32, device=device))

    def forward(self, band_weights: Optional[torch.Tensor] = None) -> torch.Tensor:
        return field_alpha(self.solver, self.spec, self.theta, band_weights)
