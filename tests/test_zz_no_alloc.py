"""nefty_forward_static: the forward sweep for callers that cannot allocate
device memory (code inside a global-mode stream capture, loops that reserve the
whole device, hosts with their own memory pool).  It keeps its scratch in one
static device array, so it is checked against nefty_forward, the allocating
entry point, on two calls in a row: the second call runs on scratch that still
holds the first call's contents.

The file is named to be collected last, so a stop-at-first-failure run has
already run every other test when it gets here; it also passes on its own in a
fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_2603_11045_gb300 import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SURF_TOL = {"fp64": 1e-10, "fp32": 1e-5}


def rel_l2(a, b):
    a = a.double().cpu().ravel()
    b = b.double().cpu().ravel()
    return float((a - b).norm() / b.norm())


def _static_forward(lib, prob, alpha, q, q_steps, obs):
    frames = torch.empty(prob.nt, prob.ny, prob.nx, dtype=alpha.dtype, device=alpha.device)
    tfin = torch.empty_like(alpha)
    loss = ctypes.c_double(0.0)
    cp = prob.to_c()
    st = lib.nefty_forward_static(0, ctypes.byref(cp), ctypes.c_void_p(alpha.data_ptr()), None,
                                  ctypes.c_void_p(q.data_ptr()), q_steps, ctypes.c_void_p(frames.data_ptr()),
                                  ctypes.c_void_p(tfin.data_ptr()), ctypes.c_void_p(obs.data_ptr()),
                                  ctypes.byref(loss), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, frames, tfin, loss.value


def test_static_forward_matches_allocating_forward_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_11045_gb300 import _native
    from paper_2603_11045_gb300.solver import Problem, Solver
    lib = _native.load()
    cases = [(S.box_inclusion_case(), "fp64"), (S.inclusion_case(nx=48, ny=40, nz=12, nt=30, seed=1011), "fp32")]
    with Solver(0) as solver:
        for w, prec in cases:
            prob = Problem.from_workload(w, prec=prec)
            dt = prob.torch_dtype
            a = torch.tensor(w.alpha, dtype=dt, device="cuda:0")
            q = torch.tensor(w.q_face, dtype=dt, device="cuda:0")
            obs = solver.forward(prob, torch.tensor(w.alpha_target, dtype=dt, device="cuda:0"), q_face=q,
                                 q_steps=w.q_steps)["frames"]
            ref = solver.forward(prob, a, q_face=q, q_steps=w.q_steps, obs=obs, T_final=True)
            st, frames, tfin, loss = _static_forward(lib, prob, a, q, w.q_steps, obs)
            assert st == 0, lib.nefty_last_error(None)
            assert rel_l2(frames, ref["frames"]) <= SURF_TOL[prec]
            assert rel_l2(tfin, ref["T_final"]) <= SURF_TOL[prec]
            assert loss == pytest.approx(ref["loss"], rel=1e-8 if prec == "fp64" else 1e-3)


def test_static_forward_rejects_oversized_and_host_arrays():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_11045_gb300 import _native
    from paper_2603_11045_gb300.solver import Problem
    lib = _native.load()
    big = Problem(256, 256, 48, nt=2, prec="fp64")          # 80 B/cell x 3.1 M cells > 48 MiB
    a = torch.ones(48, 256, 256, dtype=torch.float64, device="cuda:0")
    cp = big.to_c()
    st = lib.nefty_forward_static(0, ctypes.byref(cp), ctypes.c_void_p(a.data_ptr()), None, None, 0, None, None,
                                  None, None, None)
    assert st == _native.NEFTY_EINVAL and b"scratch" in lib.nefty_last_error(None)
    small = Problem(8, 8, 4, nt=2, prec="fp32")
    host = np.ones(256, np.float32)
    cp = small.to_c()
    st = lib.nefty_forward_static(0, ctypes.byref(cp), host.ctypes.data_as(ctypes.c_void_p), None, None, 0, None,
                                  None, None, None, None)
    assert st == _native.NEFTY_EINVAL and b"device memory" in lib.nefty_last_error(None)
