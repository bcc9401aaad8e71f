"""nefty_forward_static: the forward sweep for callers that cannot allocate
device memory when they need a solve (a loop that has reserved the whole
device for its own buffers, a loop that cannot take the synchronisation an
allocation may imply, a host that hands out memory only from its own pool).
It keeps its scratch in one static device array that every call shares, so it
is run twice in a row on each case, the second call on scratch that still
holds the first call's contents, and both calls are checked against
nefty_forward (the allocating entry point) and against the FP64 CPU oracle.

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


def _cast(x, prec):
    return np.asarray(x).astype(np.float32 if prec == "fp32" else np.float64).astype(np.float64)


def test_static_forward_matches_allocating_forward_and_oracle_twice(orc):
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
            alpha, q = _cast(w.alpha, prec), _cast(w.q_face, prec)
            op = orc.from_workload(w)
            obs_np = _cast(orc.forward(op, _cast(w.alpha_target, prec), q_face=q, q_steps=w.q_steps)["frames"], prec)
            ref_o = orc.forward(op, alpha, q_face=q, q_steps=w.q_steps, obs=obs_np)
            a = torch.tensor(alpha, dtype=dt, device="cuda:0")
            qd = torch.tensor(q, dtype=dt, device="cuda:0")
            obs = torch.tensor(obs_np, dtype=dt, device="cuda:0")
            ref = solver.forward(prob, a, q_face=qd, q_steps=w.q_steps, obs=obs, T_final=True)
            for call in range(2):   # the second call finds the first call's scratch contents
                st, frames, tfin, loss = _static_forward(lib, prob, a, qd, w.q_steps, obs)
                assert st == 0, lib.nefty_last_error(None)
                assert rel_l2(frames, ref["frames"]) <= SURF_TOL[prec], (prec, call)
                assert rel_l2(tfin, ref["T_final"]) <= SURF_TOL[prec], (prec, call)
                assert rel_l2(frames, torch.tensor(ref_o["frames"])) <= SURF_TOL[prec], (prec, call)
                assert loss == pytest.approx(ref["loss"], rel=1e-8 if prec == "fp64" else 1e-3)
                assert loss == pytest.approx(ref_o["loss"], rel=1e-8 if prec == "fp64" else 1e-3)


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


def test_static_forward_rejects_a_device_it_cannot_use():
    """A device index the process cannot make current is refused without any
    work; with two or more GPUs, an array on another GPU than the requested
    one is refused as well (it would be dereferenced without peer access)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_11045_gb300 import _native
    from paper_2603_11045_gb300.solver import Problem
    lib = _native.load()
    small = Problem(8, 8, 4, nt=2, prec="fp32")
    a = torch.ones(4, 8, 8, device="cuda:0")
    cp = small.to_c()
    n = torch.cuda.device_count()
    st = lib.nefty_forward_static(n, ctypes.byref(cp), ctypes.c_void_p(a.data_ptr()), None, None, 0, None, None,
                                  None, None, None)
    assert st != 0
    if n >= 2:
        st = lib.nefty_forward_static(1, ctypes.byref(cp), ctypes.c_void_p(a.data_ptr()), None, None, 0, None,
                                      None, None, None, None)
        assert st == _native.NEFTY_EINVAL and b"device memory" in lib.nefty_last_error(None)
