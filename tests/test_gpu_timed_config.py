"""Parity on exactly what the inversion-step benchmark times.

The benchmark runs, per step, the field at all 3,145,728 cell centres of a
256 x 256 x 48 grid (64 bands per axis, 4 x 256, on the tensor cores), the FP32
forward and adjoint sweeps over 1000 steps with the extrapolated CG start on
every SM, and the field backward whose weight-gradient products reduce over
all points (split-K over K = points).  These tests hold each of those, in the
launch configuration the benchmark uses, to a reference:

  * the FP32 gradient dJ/dalpha at 256 x 256 x 48 over 200 steps (the pulse
    reaches the inclusions) against the FP64 GPU path, which the oracle holds
    on the same grid over its first steps (test_gpu_solver.py); for the
    field-produced alpha of the benchmark and for an inclusion field;
  * the field at all 3.1 M points against the FP64 reference field evaluated
    at 20,000 seeded cells;
  * the field backward at 786,432 points (the long-K schedule of the split-K
    weight gradients) against FP64 autograd of the reference field;
  * a forward job and an inversion job served from the batched queue against
    the oracle directly.

Bars: surface rel-L2 <= 1e-5, gradient rel-L2 <= 1e-3 and cosine >= 0.9999
(FP32 vs FP64); field against the BF16-emulating reference rel-L2 <= 3e-4
(values; see the test for why) and <= 2e-2, cosine >= 0.999 (parameter
gradients), against the exact FP64 model rel-L2 <= 2e-2 (values).
"""
import math

import numpy as np
import pytest

from paper_2603_11045_gb300 import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# seeded weights of the benchmark's field (bench.py FIELD_SEED)
FIELD_SEED = 2001


@pytest.fixture(scope="module")
def solver():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_11045_gb300.solver import Solver
    s = Solver(0)
    yield s
    s.close()


def rel(a, b):
    a = torch.as_tensor(a).double().cpu().ravel()
    b = torch.as_tensor(b).double().cpu().ravel()
    return float((a - b).norm() / b.norm())


def cos(a, b):
    a = torch.as_tensor(a).double().cpu().ravel()
    b = torch.as_tensor(b).double().cpu().ravel()
    return float(a @ b / (a.norm() * b.norm()))


def test_bench_field_constant_matches_bench():
    import bench
    assert bench.FIELD_SEED == FIELD_SEED


def _bench_field(solver, nx=256, ny=256, nz=48):
    from paper_2603_11045_gb300.field import FieldSpec, field_alpha
    spec = FieldSpec(nx, ny, nz)
    th = S.xavier_theta(spec.n_freq, spec.width, spec.depth, FIELD_SEED)
    theta = torch.tensor(th, dtype=torch.float32, device="cuda")
    with torch.no_grad():
        a = field_alpha(solver, spec, theta)
    return spec, th, a


@pytest.mark.parametrize("source", ["field", "inclusions"])
def test_bench_grid_fp32_gradient_against_fp64(solver, source):
    """256 x 256 x 48, 200 steps: the FP32 sweeps as the benchmark launches
    them (default extrapolated start, every state kept, one CTA per SM)
    against the FP64 path at rtol 1e-13."""
    from paper_2603_11045_gb300.solver import Problem
    if source == "field":
        w = S.neural_field_case(nt=200)
        _, _, a32 = _bench_field(solver)
        targets = w.alpha            # the ground truth with inclusions, as in the benchmark
    else:
        w = S.inclusion_case(nx=256, ny=256, nz=48, nt=200, seed=2002)
        a32 = torch.tensor(w.alpha, dtype=torch.float32, device="cuda")
        targets = w.alpha_target     # the background without inclusions
    p32 = Problem.from_workload(w, prec="fp32")
    p64 = Problem.from_workload(w, prec="fp64")
    q64 = torch.tensor(w.q_face, dtype=torch.float64, device="cuda")
    obs64 = solver.forward(p64, torch.tensor(targets, dtype=torch.float64, device="cuda"), q_face=q64,
                           q_steps=w.q_steps)["frames"]
    a64 = a32.double()
    obs32 = obs64.float()
    q32 = q64.float()
    f32 = solver.forward(p32, a32, q_face=q32, q_steps=w.q_steps, obs=obs32)
    g32 = solver.adjoint_grad(p32, a32, obs32, q_face=q32, q_steps=w.q_steps)
    # the FP64 reference sees exactly the FP32 inputs
    obs_r = obs32.double()
    f64 = solver.forward(p64, a64, q_face=q32.double(), q_steps=w.q_steps, obs=obs_r)
    g64 = solver.adjoint_grad(p64, a64, obs_r, q_face=q32.double(), q_steps=w.q_steps)
    st = g32["stats"]
    assert st["grid_blocks"] >= 128 and st["ckpt_every"] == 1 and st["not_converged"] == 0, st
    assert rel(f32["frames"], f64["frames"]) <= 1e-5
    assert f32["loss"] == pytest.approx(f64["loss"], rel=1e-4)
    assert rel(g32["grad_alpha"], g64["grad_alpha"]) <= 1e-3, rel(g32["grad_alpha"], g64["grad_alpha"])
    assert cos(g32["grad_alpha"], g64["grad_alpha"]) >= 0.9999


def test_field_eval_at_bench_size_sampled(solver):
    """All 3,145,728 cell centres on the tensor cores, checked at 20,000 seeded
    cells against the reference field evaluated at those cells."""
    import oracle.field as OF
    spec, th, a = _bench_field(solver)
    M = spec.nx * spec.ny * spec.nz
    assert a.numel() == M == 3_145_728
    cells = torch.tensor(np.sort(S.rng(2010).choice(M, 20_000, replace=False)))
    args = (spec.nx, spec.ny, spec.nz, spec.n_freq, spec.width, spec.depth, spec.freq_lo, spec.freq_hi,
            spec.alpha_min, spec.alpha_max)
    th64 = torch.tensor(th, dtype=torch.float32).double()
    got = a.reshape(-1)[cells.cuda()].double().cpu()
    emu = OF.field(th64, *args, bf16=True, cells=cells)
    exact = OF.field(th64, *args, bf16=False, cells=cells)
    # Both the kernel and the reference round every activation to BF16, but
    # from sums taken in different precision and order (FP32 tensor-core
    # accumulation and FP32 features against FP64), so a sum that falls near a
    # BF16 rounding boundary rounds to neighbouring values on the two sides.
    # At this size that alone moves alpha by 1.4e-4 rel-L2 (the same network
    # evaluated with FP32 features and sums against FP64 ones, on these
    # cells); the bar is twice that.
    assert rel(got, emu) <= 3e-4
    assert float((got - emu).abs().max()) <= 4e-3
    assert rel(got, exact) <= 2e-2


def _ref_field_grad(th, spec, g_a, bf16, chunk=65536):
    """FP64 autograd of the reference field; the gradient is a sum over points,
    taken chunk by chunk."""
    import oracle.field as OF
    args = (spec.nx, spec.ny, spec.nz, spec.n_freq, spec.width, spec.depth, spec.freq_lo, spec.freq_hi,
            spec.alpha_min, spec.alpha_max)
    th64 = torch.tensor(th, dtype=torch.float32).double()
    total = torch.zeros_like(th64)
    M = g_a.numel()
    for c0 in range(0, M, chunk):
        cells = torch.arange(c0, min(M, c0 + chunk))
        t = th64.clone().requires_grad_(True)
        (OF.field(t, *args, bf16=bf16, cells=cells) * g_a[cells]).sum().backward()
        total += t.grad
    return total


def test_field_backward_long_k(solver):
    """The field backward at 786,432 points (128 x 128 x 48 centres, the
    benchmark's network): the weight-gradient products reduce over K = 786,432
    points in split-K; against FP64 autograd of the reference field."""
    from paper_2603_11045_gb300.field import field_alpha
    spec, th, _ = _bench_field(solver, 128, 128, 48)
    M = spec.nx * spec.ny * spec.nz
    assert M == 786_432
    theta = torch.tensor(th, dtype=torch.float32, device="cuda", requires_grad=True)
    g_a = torch.tensor(S.rng(2011).standard_normal(M), dtype=torch.float32)
    (field_alpha(solver, spec, theta).reshape(-1) * g_a.cuda()).sum().backward()
    g = theta.grad.double().cpu()
    emu = _ref_field_grad(th, spec, g_a.double(), bf16=True)
    assert rel(g, emu) <= 2e-2, rel(g, emu)
    assert cos(g, emu) >= 0.999


def test_served_jobs_against_oracle(solver, orc):
    """A forward job and an inversion job submitted together to the batched
    queue (their sweeps share launches), each checked against the oracle
    directly: the forward job's frames, and the inversion's alpha after its
    projected-gradient steps and the loss of its last step, replayed on the
    oracle's FP64 gradients."""
    from paper_2603_11045_gb300.serve import Server
    from paper_2603_11045_gb300.solver import Problem
    wf = S.inclusion_case(nx=64, ny=48, nz=16, nt=40, seed=3101)
    wi = S.inclusion_case(nx=32, ny=32, nz=8, nt=30, seed=3102)
    f32 = lambda x: np.asarray(x, dtype=np.float32)
    pf, pi = Problem.from_workload(wf, prec="fp32"), Problem.from_workload(wi, prec="fp32")
    opf, opi = orc.from_workload(wf), orc.from_workload(wi)
    qf, qi = f32(wf.q_face), f32(wi.q_face)
    obs_i = f32(orc.forward(opi, f32(wi.alpha_target).astype(np.float64), q_face=qi.astype(np.float64),
                            q_steps=wi.q_steps)["frames"])
    lr, floor, iters = 2.0, 0.05, 2
    dev = lambda x: torch.tensor(x, device="cuda")
    a_f, a_i = dev(f32(wf.alpha)), dev(f32(wi.alpha))
    fr = torch.empty(pf.nt, pf.ny, pf.nx, device="cuda")
    with Server(solver, lanes=2, batched=True, chunk_steps=8) as srv:
        jf = srv.submit(pf, a_f, kind="forward", q_face=dev(qf), q_steps=wf.q_steps, frames_out=fr)
        ji = srv.submit(pi, a_i, kind="inversion", iters=iters, lr=lr, alpha_floor=floor, q_face=dev(qi),
                        q_steps=wi.q_steps, obs=dev(obs_i))
        rf, ri = srv.wait(jf), srv.wait(ji)
    assert rf["state_name"] == "done" and ri["state_name"] == "done", (rf, ri)
    assert rf["launches"] >= 1 and ri["launches"] >= 1
    ref_f = orc.forward(opf, f32(wf.alpha).astype(np.float64), q_face=qf.astype(np.float64),
                        q_steps=wf.q_steps)["frames"]
    assert rel(fr, ref_f) <= 1e-5
    a = f32(wi.alpha).astype(np.float64)
    loss = None
    for _ in range(iters):
        r = orc.adjoint_grad(opi, a, q_face=qi.astype(np.float64), q_steps=wi.q_steps,
                             obs=obs_i.astype(np.float64))
        loss = r["loss"]
        a = np.maximum(a - lr * r["grad_alpha"], floor)
    assert ri["iters_done"] == iters
    assert ri["loss"] == pytest.approx(loss, rel=1e-3)
    assert rel(a_i, a) <= 1e-5
