"""Python face of libnefty's serving queue (nefty_serve_* in include/nefty.h).

``Server`` attaches a queue with ``lanes`` concurrent workers (job slots) to a
``Solver``'s handle; with ``batched`` the running jobs' FP32 sweeps share one
persistent launch.  ``submit`` copies the job description into the library and returns a
job id at once; the arrays stay referenced here until the job has finished.
Every step of a job runs in libnefty (its own threads, streams and kernels);
this module only marshals arguments.
"""
from __future__ import annotations

import ctypes
import time

import torch

from . import _native as N
from .solver import Problem, Solver, _as_array

__all__ = ["Server", "STATE_NAMES"]

STATE_NAMES = {N.NEFTY_JOB_QUEUED: "queued", N.NEFTY_JOB_RUNNING: "running", N.NEFTY_JOB_DONE: "done",
               N.NEFTY_JOB_FAILED: "failed", N.NEFTY_JOB_CANCELLED: "cancelled"}
_FINAL = (N.NEFTY_JOB_DONE, N.NEFTY_JOB_FAILED, N.NEFTY_JOB_CANCELLED)


class Server:
    def __init__(self, solver: Solver, lanes: int = 2, max_queue: int = 0, mem_budget_bytes: int = 0,
                 batched: bool = True, chunk_steps: int = 0, launch_us: int = 0):
        self.solver = solver
        self._lib = solver._lib
        cfg = N.nefty_serve_config(int(lanes), int(max_queue), int(mem_budget_bytes), 1 if batched else -1,
                                   int(chunk_steps), int(launch_us))
        N.check(self._lib.nefty_serve_start(solver._h, ctypes.byref(cfg)), solver._h)
        self._keep = {}

    def submit(self, prob: Problem, alpha, kind: str = "forward", iters: int = 0, lr: float = 0.0,
               alpha_floor: float = 1e-3, T0=None, q_face=None, q_steps: int = 0, q_full=None, obs=None,
               frames_out=None) -> int:
        """Queue a job; returns its id.  ``alpha`` is updated in place by an inversion."""
        dt = prob.torch_dtype
        Nc, S = prob.n_cells, prob.nx * prob.ny
        a = _as_array(alpha, dt, Nc, "alpha", allow_none=False)
        t0 = _as_array(T0, dt, Nc, "T0")
        qf = _as_array(q_face, dt, S, "q_face")
        qa = _as_array(q_full, dt, prob.nt * S, "q_full")
        ob = _as_array(obs, dt, prob.nt * S, "obs")
        fr = _as_array(frames_out, dt, prob.nt * S, "frames_out")
        job = N.nefty_job()
        job.problem = prob.to_c()
        job.kind = N.NEFTY_JOB_INVERSION if kind == "inversion" else N.NEFTY_JOB_FORWARD
        job.iters, job.lr, job.alpha_floor = int(iters), float(lr), float(alpha_floor)
        ptr = lambda x: None if x[1] is None else x[1].value
        job.alpha, job.T0, job.q_face = ptr(a), ptr(t0), ptr(qf)
        job.q_full, job.obs, job.frames_out = ptr(qa), ptr(ob), ptr(fr)
        job.q_steps = int(q_steps)
        jid = ctypes.c_uint64(0)
        N.check(self._lib.nefty_serve_submit(self.solver._h, ctypes.byref(job), ctypes.byref(jid)), self.solver._h)
        self._keep[jid.value] = (a[0], t0[0], qf[0], qa[0], ob[0], fr[0])
        return jid.value

    def poll(self, job_id: int) -> dict:
        r = N.nefty_job_result()
        N.check(self._lib.nefty_serve_poll(self.solver._h, int(job_id), ctypes.byref(r)), self.solver._h)
        d = r.as_dict()
        d["state_name"] = STATE_NAMES.get(d["state"], "?")
        if d["state"] in _FINAL:
            self._keep.pop(int(job_id), None)
        return d

    def cancel(self, job_id: int):
        N.check(self._lib.nefty_serve_cancel(self.solver._h, int(job_id)), self.solver._h)

    def wait(self, job_id: int, timeout: float = 600.0, interval: float = 0.002) -> dict:
        """Poll until the job is done, failed or cancelled."""
        t_end = time.monotonic() + timeout
        while True:
            d = self.poll(job_id)
            if d["state"] in _FINAL:
                return d
            if time.monotonic() > t_end:
                raise TimeoutError(f"job {job_id} still {d['state_name']} after {timeout} s")
            time.sleep(interval)

    def stop(self):
        if self.solver._h:
            N.check(self._lib.nefty_serve_stop(self.solver._h), self.solver._h)
        self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.stop()
