"""Serving queue (nefty_serve_*): continuous batching of ragged jobs.

Checks on the GPU, with batched launches (the running jobs' sweeps in one
persistent grid) and with one grid per lane, that a served job computes what
the direct call computes, that its results are the same bits alone and among
other jobs, that sweeps cut into many chunks and jobs that cannot be batched
still give the direct call's results, that cancellation and refusal work, and
that jobs really overlap on the device."""
import pytest
import torch

from paper_2603_11045_gb300 import synthetic as S
from paper_2603_11045_gb300.serve import Server
from paper_2603_11045_gb300.solver import Problem, Solver

pytestmark = pytest.mark.gpu


def _case(nx, ny, nz, nt, seed, prec="fp32"):
    w = S.inclusion_case(nx=nx, ny=ny, nz=nz, nt=nt, seed=seed)
    p = Problem.from_workload(w, prec=prec)
    dt = p.torch_dtype
    alpha = torch.tensor(w.alpha, dtype=dt, device="cuda")
    q = torch.tensor(w.q_face, dtype=dt, device="cuda")
    return w, p, alpha, q


@pytest.fixture(scope="module")
def solver():
    s = Solver(0)
    yield s
    s.close()


@pytest.mark.parametrize("batched", [True, False])
def test_forward_job_matches_direct_call(solver, batched):
    w, p, alpha, q = _case(64, 48, 16, 40, 3001)
    direct = solver.forward(p, alpha, q_face=q, q_steps=w.q_steps)["frames"]
    with Server(solver, lanes=2, batched=batched) as srv:
        fr = torch.empty_like(direct)
        jid = srv.submit(p, alpha, kind="forward", q_face=q, q_steps=w.q_steps, frames_out=fr)
        r = srv.wait(jid)
    assert r["state_name"] == "done" and r["status"] == 0, r
    assert r["t_submit_ns"] <= r["t_admit_ns"] <= r["t_done_ns"]
    assert (r["launches"] >= 1) == batched, r
    err = (fr - direct).norm() / direct.norm()
    assert err < 1e-5, float(err)


@pytest.mark.parametrize("batched", [True, False])
def test_inversion_job_matches_python_loop(solver, batched):
    w, p, alpha, q = _case(48, 48, 12, 30, 3002)
    obs = solver.forward(p, torch.tensor(w.alpha_target, dtype=torch.float32, device="cuda"), q_face=q,
                         q_steps=w.q_steps)["frames"]
    lr, floor, iters = 2.0, 0.05, 3
    ref = alpha.clone()
    losses = []
    for _ in range(iters):
        out = solver.adjoint_grad(p, ref, obs, q_face=q, q_steps=w.q_steps)
        losses.append(out["loss"])
        ref = torch.clamp(ref - lr * out["grad_alpha"], min=floor)
    a = alpha.clone()
    with Server(solver, lanes=2, batched=batched) as srv:
        jid = srv.submit(p, a, kind="inversion", iters=iters, lr=lr, alpha_floor=floor, q_face=q,
                         q_steps=w.q_steps, obs=obs)
        r = srv.wait(jid)
    assert r["state_name"] == "done" and r["iters_done"] == iters, r
    assert abs(r["loss"] - losses[-1]) <= 1e-4 * abs(losses[-1]), (r["loss"], losses)
    err = (a - ref).norm() / ref.norm()
    assert err < 1e-5, float(err)
    assert losses[-1] < losses[0]


@pytest.mark.parametrize("batched", [True, False])
def test_same_result_alone_and_in_the_mix(solver, batched):
    """A job's frames alone and among other jobs.  On lanes with their own
    grids the job runs on the same CTAs either way: the same bits.  Batched,
    the job's share of the launch's CTAs follows the mix, which changes only
    the order of its reductions: the frames agree to the FP32 surface
    tolerance (and in fact to rounding)."""
    w, p, alpha, q = _case(64, 64, 16, 60, 3003)
    others = [_case(*shape, seed) for shape, seed in (((96, 64, 24, 80), 3004), ((128, 96, 20, 50), 3005),
                                                      ((32, 32, 8, 200), 3006))]
    with Server(solver, lanes=3, batched=batched, chunk_steps=9) as srv:
        alone = torch.empty(p.nt, p.ny, p.nx, dtype=torch.float32, device="cuda")
        r = srv.wait(srv.submit(p, alpha, q_face=q, q_steps=w.q_steps, frames_out=alone))
        assert r["state_name"] == "done", r
        assert r["shared_launches"] == 0, r
        ids, mixed = [], torch.empty_like(alone)
        for k, (wo, po, ao, qo) in enumerate(others):
            ids.append(srv.submit(po, ao, q_face=qo, q_steps=wo.q_steps))
            if k == 1:
                ids.append(srv.submit(p, alpha, q_face=q, q_steps=w.q_steps, frames_out=mixed))
        res = [srv.wait(i) for i in ids]
    assert all(x["state_name"] == "done" for x in res), res
    if batched:   # 60 steps in chunks of 9: 7 launches, shared with the jobs submitted before it
        assert res[2]["launches"] == 7 and res[2]["shared_launches"] > 0, res[2]
        assert float((mixed - alone).norm() / alone.norm()) <= 1e-6
    else:
        assert torch.equal(alone, mixed)


def test_launches_by_device_time(solver):
    """A tiny device-time budget per launch (300 us) makes every batched sweep
    stop part-way by time and resume in the next launch from the step it
    reached: a forward job's frames and loss and an inversion's alpha match
    the direct calls, and each job took many launches."""
    w, p, alpha, q = _case(96, 64, 24, 80, 3201)
    obs = solver.forward(p, torch.tensor(w.alpha_target, dtype=torch.float32, device="cuda"), q_face=q,
                         q_steps=w.q_steps)["frames"]
    direct = solver.forward(p, alpha, q_face=q, q_steps=w.q_steps, obs=obs)
    wi, pi, ai, qi = _case(64, 48, 16, 40, 3202)
    obs_i = solver.forward(pi, torch.tensor(wi.alpha_target, dtype=torch.float32, device="cuda"), q_face=qi,
                           q_steps=wi.q_steps)["frames"]
    lr, floor, iters = 2.0, 0.05, 2
    ref = ai.clone()
    for _ in range(iters):
        out = solver.adjoint_grad(pi, ref, obs_i, q_face=qi, q_steps=wi.q_steps)
        ref = torch.clamp(ref - lr * out["grad_alpha"], min=floor)
    with Server(solver, lanes=2, launch_us=300) as srv:
        fr = torch.empty_like(direct["frames"])
        j1 = srv.submit(p, alpha, q_face=q, q_steps=w.q_steps, obs=obs, frames_out=fr)
        a_inv = ai.clone()
        j2 = srv.submit(pi, a_inv, kind="inversion", iters=iters, lr=lr, alpha_floor=floor, q_face=qi,
                        q_steps=wi.q_steps, obs=obs_i)
        r1, r2 = srv.wait(j1), srv.wait(j2)
    assert r1["state_name"] == "done" and r2["state_name"] == "done", (r1, r2)
    assert r1["launches"] >= 5 and r2["launches"] >= 5, (r1, r2)
    assert float((fr - direct["frames"]).norm() / direct["frames"].norm()) <= 1e-6
    assert abs(r1["loss"] - direct["loss"]) <= 1e-6 * abs(direct["loss"])
    assert float((a_inv - ref).norm() / ref.norm()) <= 1e-5


def test_batched_ragged_mix_matches_direct_calls(solver):
    """Forward jobs with a loss, an inversion and a grid the batch kernel does
    not take (nx % 4 != 0) served together, their sweeps cut into 7-step
    chunks: each result matches the direct call on the solver's own handle."""
    shapes = (((64, 48, 16, 45), 3101), ((96, 64, 24, 30), 3102), ((30, 28, 8, 40), 3103))
    cases = [_case(*shape, seed) for shape, seed in shapes]
    targets, direct = [], []
    for w, p, alpha, q in cases:
        at = torch.tensor(w.alpha_target, dtype=torch.float32, device="cuda")
        obs = solver.forward(p, at, q_face=q, q_steps=w.q_steps)["frames"]
        targets.append(obs)
        direct.append(solver.forward(p, alpha, q_face=q, q_steps=w.q_steps, obs=obs))
    wi, pi, ai, qi = _case(48, 48, 12, 30, 3104)
    obs_i = solver.forward(pi, torch.tensor(wi.alpha_target, dtype=torch.float32, device="cuda"), q_face=qi,
                           q_steps=wi.q_steps)["frames"]
    lr, floor, iters = 2.0, 0.05, 2
    ref = ai.clone()
    for _ in range(iters):
        out = solver.adjoint_grad(pi, ref, obs_i, q_face=qi, q_steps=wi.q_steps)
        ref = torch.clamp(ref - lr * out["grad_alpha"], min=floor)
    with Server(solver, lanes=4, chunk_steps=7) as srv:
        frames, ids = [], []
        a_inv = ai.clone()
        ids.append(srv.submit(pi, a_inv, kind="inversion", iters=iters, lr=lr, alpha_floor=floor, q_face=qi,
                              q_steps=wi.q_steps, obs=obs_i))
        for (w, p, alpha, q), obs in zip(cases, targets):
            fr = torch.empty(p.nt, p.ny, p.nx, dtype=torch.float32, device="cuda")
            frames.append(fr)
            ids.append(srv.submit(p, alpha, q_face=q, q_steps=w.q_steps, obs=obs, frames_out=fr))
        res = [srv.wait(i) for i in ids]
    assert all(r["state_name"] == "done" and r["status"] == 0 for r in res), res
    inv, fwd = res[0], res[1:]
    assert inv["shared_launches"] > 0, inv
    assert fwd[0]["launches"] == 7 and fwd[1]["launches"] == 5, fwd   # ceil(45 / 7), ceil(30 / 7)
    assert fwd[2]["launches"] == 0, fwd[2]                             # nx % 4 != 0: the lane's own grid
    for fr, d, r in zip(frames, direct, fwd):
        err = (fr - d["frames"]).norm() / d["frames"].norm()
        assert err < 1e-5, float(err)
        assert abs(r["loss"] - d["loss"]) <= 1e-5 * abs(d["loss"]), (r["loss"], d["loss"])
    err = (a_inv - ref).norm() / ref.norm()
    assert err < 1e-5, float(err)


def test_cancel_queued_and_refuse_oversized(solver):
    w, p, alpha, q = _case(128, 128, 32, 300, 3007)
    with Server(solver, lanes=1, mem_budget_bytes=1 << 30) as srv:
        first = srv.submit(p, alpha, q_face=q, q_steps=w.q_steps)
        second = srv.submit(p, alpha, q_face=q, q_steps=w.q_steps)
        srv.cancel(second)
        r2 = srv.poll(second)
        r1 = srv.wait(first)
        assert r1["state_name"] == "done", r1
        assert r2["state_name"] == "cancelled" and r2["t_admit_ns"] == 0, r2
        big = Problem(nx=512, ny=512, nz=96, nt=2000, dt=0.2)
        a_big = torch.ones(big.nz, big.ny, big.nx, device="cuda")
        from paper_2603_11045_gb300._native import NeftyError, NEFTY_ENOMEM
        with pytest.raises(NeftyError) as e:
            srv.submit(big, a_big, kind="forward")
        assert e.value.status == NEFTY_ENOMEM


@pytest.mark.parametrize("batched", [True, False])
def test_lanes_overlap_jobs(solver, batched):
    """Two equal jobs on two lanes: with their own grids (each job has half
    of the device) they finish in well under twice one job's time; batched,
    where one job alone has the whole device, they share every launch and
    take no longer than back to back."""
    import time
    w, p, alpha, q = _case(128, 128, 32, 150, 3008)
    with Server(solver, lanes=2, batched=batched, chunk_steps=16) as srv:
        srv.wait(srv.submit(p, alpha, q_face=q, q_steps=w.q_steps))   # warm-up (workspace)
        srv.wait(srv.submit(p, alpha, q_face=q, q_steps=w.q_steps))
        t0 = time.perf_counter()
        srv.wait(srv.submit(p, alpha, q_face=q, q_steps=w.q_steps))
        one = time.perf_counter() - t0
        t0 = time.perf_counter()
        a, b = srv.submit(p, alpha, q_face=q, q_steps=w.q_steps), srv.submit(p, alpha, q_face=q, q_steps=w.q_steps)
        ra, rb = srv.wait(a), srv.wait(b)
        two = time.perf_counter() - t0
    assert {ra["lane"], rb["lane"]} == {0, 1}
    if batched:
        assert ra["shared_launches"] > 0 and rb["shared_launches"] > 0, (ra, rb)
    assert two < (2.2 if batched else 1.6) * one, (one, two)


def test_batched_lone_job_has_the_whole_device(solver):
    """With eight job slots, a job running alone is served by a grid over the
    whole device when batched, but by an eighth of it on unbatched lanes."""
    import time
    w, p, alpha, q = _case(128, 128, 32, 150, 3009)
    t = {}
    for batched in (True, False):
        with Server(solver, lanes=8, batched=batched) as srv:
            srv.wait(srv.submit(p, alpha, q_face=q, q_steps=w.q_steps))   # warm-up (workspace)
            t0 = time.perf_counter()
            r = srv.wait(srv.submit(p, alpha, q_face=q, q_steps=w.q_steps))
            t[batched] = time.perf_counter() - t0
            assert r["state_name"] == "done" and r["shared_launches"] == 0, r
    assert t[True] < 0.6 * t[False], t


def test_periodic_job_joins_the_batched_launches(solver):
    """A job on the paper's grid (periodic lateral walls) is batched like any
    other FP32 job whose rows are 16-byte multiples, and its frames match the
    direct call."""
    w = S.paper_grid_case(nt=20)
    p = Problem.from_workload(w, prec="fp32")
    alpha = torch.tensor(w.alpha, dtype=torch.float32, device="cuda")
    T0 = torch.tensor(w.T0, dtype=torch.float32, device="cuda")
    direct = solver.forward(p, alpha, T0=T0)["frames"]
    with Server(solver, lanes=2, chunk_steps=6) as srv:
        fr = torch.empty_like(direct)
        r = srv.wait(srv.submit(p, alpha, T0=T0, frames_out=fr))
    assert r["state_name"] == "done" and r["launches"] == 4, r   # ceil(20 / 6)
    err = (fr - direct).norm() / direct.norm()
    assert err < 1e-5, float(err)
