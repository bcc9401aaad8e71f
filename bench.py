#!/usr/bin/env python
"""Benchmark of the NeFTY hot path on GB300: one step = one inversion step on a
synthetic 256x256x48 grid over 1000 implicit-Euler steps (dt = 0.25): the
neural field theta -> alpha (Fourier features, 4 x 256 ReLU MLP on the tensor
cores), the forward sweep and the reverse adjoint sweep with dJ/dalpha (FP32
vectors and stencil, compensated reductions), the TV regulariser's gradient
(lambda 1e-4), and the field's backward pass to dJ/dtheta.

Prints one JSON line (rank 0).  Under torchrun each rank runs its own replica
of the workload (no data-path collective; weak scaling) and rank 0 reports the
aggregate over the max-over-ranks time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

``--impl reference`` times the FP64 CPU oracle on the host cores, on a bounded
sample of the same workload (the first few time steps of the same grid).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import signal
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# The oracle's OpenMP loops read this once, when the library loads.
os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))

import numpy as np  # noqa: E402

METRIC = "fwd+adjoint Gcell-steps/s"
UNIT = "Gcell-steps/s"
# Algorithmic bytes per cell.  The FP32 path reads alpha and recomputes the
# face values in every pass: one PCG iteration reads and writes x, r, p (24 B)
# and reads alpha (4 B).  The FP64 path reads three stored face values and the
# Jacobi diagonal instead, all words 8 B (48 + 32 B).  Each time step also
# reads its right-hand side and writes its solution (8 B, FP64 16 B), and each
# adjoint step's gradient assembly reads T^n and updates an FP64 accumulator
# (4 + 16 B, FP64 8 + 16 B).
ALG_BYTES_ITER = {"fp32": 28, "fp64": 80}
ALG_BYTES_STEP = {"fp32": 8, "fp64": 16}
ALG_BYTES_GRAD = {"fp32": 20, "fp64": 24}
# DRAM bytes per cell-step of the FP32 CG launches, measured by ncu on this
# workload at full size (256x256x48, 1000 steps; dram__bytes_read.sum +
# dram__bytes_write.sum, one-pass metrics, every launch of a bench run): the
# forward sweep and the reverse sweep with the gradient.  bench.py multiplies
# them by the timed step's solved steps for `traffic`, and only while the
# kernel source still hashes to the captured one: once the kernels change the
# figure is stale and `traffic` is null.
DRAM_CAPTURE = {
    "fp32": {"fwd": 112.4, "adj": 186.8, "grid": [256, 256, 48], "nt": 1000,
             "kernel_source": "paper_2603_11045_gb300/csrc/cg_tiled.cu", "kernel_sha16": "225deb44661310b3",
             "profiles": ["profiles/inversion_step_256x256x48_nt1000_launches.md"]},
    "fp64": None,
}
KERNELS = {"fp32": "tiled::forward_tiled + tiled::adjoint_tiled (persistent single-reduction Jacobi-PCG, TMA-staged)",
           "fp64": "nefty::forward_kernel + nefty::adjoint_kernel (persistent Jacobi-PCG, FP64)"}


def source_sha16(rel_path):
    import hashlib
    with open(os.path.join(ROOT, rel_path), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--nx", type=int, default=256)
    ap.add_argument("--ny", type=int, default=256)
    ap.add_argument("--nz", type=int, default=48)
    ap.add_argument("--nt", type=int, default=1000)
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--ckpt-every", type=int, default=0)
    ap.add_argument("--extrap", type=int, default=0,
                    help="FP32 CG start: increments extrapolated from (0 = the library default, -1 = none)")
    ap.add_argument("--cpu-sample-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-error", action="store_true",
                    help="skip the FP32-vs-FP64 error of the timed configuration (run after timing)")
    ap.add_argument("--paper-iters", type=int, default=300, help="paper-inversion: Adam iterations")
    ap.add_argument("--paper-jacobi-k", type=int, default=50,
                    help="paper-inversion: Jacobi sweeps per solve (the paper's 50; 0 = converged Jacobi-PCG)")
    ap.add_argument("--workload", default="inversion",
                    choices=["inversion", "serving", "stress", "jacobi", "paper-inversion"],
                    help="inversion: the timed inversion step (default); serving: latency of a job stream; "
                         "stress: one forward + adjoint at 512x512x96, 2000 steps, sqrt-checkpointing")
    ap.add_argument("--stress-fp64", action="store_true", help="stress: also run the FP64 path and compare")
    ap.add_argument("--serve-scale", default="small", choices=["small", "full"],
                    help="serving stream: small (24 jobs, <= 192x160x40, 50-200 steps, 3-step inversions) "
                         "or full (64 jobs at 4/s, grids up to 256x256x64, 200-1000 steps, 10-step inversions)")
    ap.add_argument("--serve-lanes", type=int, default=8, help="job slots of the batched server")
    ap.add_argument("--serve-unbatched-lanes", type=int, default=2,
                    help="lanes of the comparison replay in which each lane runs its own grid")
    ap.add_argument("--serve-no-fp64", action="store_true", help="skip the one-at-a-time FP64 replay")
    return ap.parse_args()


TV_LAMBDA, TV_EPS = 1e-4, 1e-6
FIELD_SEED = 2001


def workload(args):
    from paper_2603_11045_gb300 import synthetic as S
    w = S.neural_field_case(nx=args.nx, ny=args.ny, nz=args.nz, nt=args.nt, dt=0.25)
    # candidate alpha for the CPU baseline (the GPU step takes alpha from the
    # neural field): the smooth background without the inclusions
    g = S.rng(w.extra["seed"])
    cand = g.uniform(0.8, 1.2, size=(w.nz, w.ny, w.nx))
    return w, cand


def field_spec(w):
    from paper_2603_11045_gb300.field import FieldSpec
    # 64 bands pi..128 pi, 4 x 256, alpha in [0.01, 2]; the backward at the
    # evaluated theta takes the evaluation's activations
    return FieldSpec(w.nx, w.ny, w.nz, keep_activations=True)


def mlp_flops(spec):
    """Multiply-adds x 2 of the dense layers: forward, and backward (input
    gradients of layers 1..depth-1 plus weight gradients of all layers)."""
    D, W, L, M = 6 * spec.n_freq, spec.width, spec.depth, spec.nx * spec.ny * spec.nz
    fwd = 2.0 * M * (D * W + (L - 1) * W * W)
    bwd = 2.0 * M * ((L - 1) * W * W) + fwd
    return fwd, bwd


def config_dict(args, w):
    return {"workload": f"inversion step, {w.nx}x{w.ny}x{w.nz} cells, {w.nt} implicit-Euler steps, dt={w.dt}",
            "grid": [w.nx, w.ny, w.nz], "nt": w.nt, "dt": w.dt, "prec": args.prec,
            "field": "64 log-spaced bands (pi..128 pi) per axis -> 4 x 256 ReLU (BF16 tensor cores) -> [0.01, 2]",
            "tv": {"lambda": TV_LAMBDA, "eps": TV_EPS},
            "solver": "Jacobi-PCG, rtol 5e-10 (FP32) / 1e-13 (FP64), CG start quadratically extrapolated from the last three increments (FP32)",
            "bc": "zero-flux walls", "forcing": "Gaussian surface pulse, sigma 20 cells, 3 steps",
            "l2": "flushed between timed steps (256 MiB write)"}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the raw samples (summarised in the JSON line's "clocks")
        self.path = os.path.join(os.environ.get("NEFTY_BENCH_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"nefty_clocks_rank{index}_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.send_signal(signal.SIGTERM)
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# -------------------------------------------------------------- CPU oracle
def oracle_sample(args, w, cand, steps):
    """The FP64 oracle (as it stands) on the first `steps` time steps of the
    same grid: forward + adjoint gradient.  Returns (Gcell-steps/s, seconds)."""
    import oracle
    p = oracle.from_workload(w, nt=steps, loss_scale=1.0 / (w.nt * w.nx * w.ny))
    obs = oracle.forward(p, w.alpha, q_face=w.q_face, q_steps=w.q_steps)["frames"]
    t = time.perf_counter()
    oracle.adjoint_grad(p, cand, q_face=w.q_face, q_steps=w.q_steps, obs=obs)
    dt = time.perf_counter() - t
    return w.n_cells * steps / dt / 1e9, dt


def cpu_cores():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def oracle_single_thread(args):
    """The same oracle sample (one time step) on one host thread, in a fresh
    process with OMP_NUM_THREADS=1; None if that process fails."""
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "0",
           "--cpu-sample-steps", "1", "--nx", str(args.nx), "--ny", str(args.ny), "--nz", str(args.nz),
           "--nt", str(args.nt)]
    env = dict(os.environ, OMP_NUM_THREADS="1", RANK="0")
    try:
        res = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=300)
        line = json.loads(res.stdout.strip().splitlines()[-1])
        return {"value": line["value"], "unit": line["unit"], "cores": 1,
                "sample": f"first 1 of {args.nt} steps of the same grid, forward + adjoint, FP64, "
                          f"{line['ms_per_step'] / 1000:.1f} s"}
    except Exception:
        return None


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w, cand = workload(args)
    steps = max(1, args.cpu_sample_steps)
    for _ in range(args.warmup):
        oracle_sample(args, w, cand, steps)
    vals, secs = [], []
    for _ in range(args.steps):
        v, s = oracle_sample(args, w, cand, steps)
        vals.append(v)
        secs.append(s)
    value = w.n_cells * steps * len(secs) / sum(secs) / 1e9
    sample = f"first {steps} of {w.nt} steps of the same {w.nx}x{w.ny}x{w.nz} grid, forward + adjoint, per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * sum(secs) / len(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(args, w),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ native
def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def field_launches(spec, reuse):
    """Kernels of one nefty_field_eval + nefty_field_backward + nefty_tv call
    (no band weights).  reuse: the backward took the evaluation's kept
    activations (one parameter comparison instead of the forward layers)."""
    L, ns = spec.depth, 3 if spec.precision == 1 else 1
    # axis tables, features (+ the skip layer's feature copies), BF16 weights, layer GEMMs
    fwd = 3 + 1 + (ns if spec.skip_layer else 0) + L + L
    ev = fwd + 1                    # + head
    # backward: the forward layers again (or the comparison); the head pass
    # (fused: g_f, top delta and its transpose, three partial sums, then their
    # three final sums; with a head too wide for its shared-memory tile, head
    # backward, 2 x 2 output-layer sums and the top delta's transpose in ns
    # blocks); L weight transposes, h_0^T; per layer 2 bias sums (the top
    # layer's in the fused pass), weight-gradient GEMM, split-K reduce; and
    # L - 1 input-gradient GEMMs
    W = spec.width
    fused = max((2 if ns == 3 else 1) * W * 32, 8 * (2 * W + 1)) * 4 <= 200 * 1024 and (W // 8 + 31) // 32 in ((1, 2, 4) if ns == 1 else (1, 2))
    head = 1 + 3 if fused else 1 + 4 + ns
    bias = 2 * (L - 1) if fused else 2 * L
    bw = (1 if reuse else fwd) + head + L + 1 + bias + 2 * L + (L - 1)
    return ev + bw + 1              # + TV


def aggregate(total_ms, units_per_rank, world, device):
    """Whole-job figures of a replica run: the slowest rank's time (all-reduce
    MAX over the process group when world > 1) and the units all ranks
    processed per second, in billions.  Returns (max_ms, value)."""
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    max_ms = float(t.item())
    return max_ms, units_per_rank * world / (max_ms / 1000.0) / 1e9


def run_native(args):
    import torch
    import torch.distributed as dist
    from paper_2603_11045_gb300.solver import Problem, Solver

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    import ctypes
    from paper_2603_11045_gb300 import synthetic as S
    from paper_2603_11045_gb300 import _native as NV
    w, cand = workload(args)
    prob = Problem.from_workload(w, prec=args.prec, ckpt_every=args.ckpt_every, extrap=args.extrap)
    dt = prob.torch_dtype
    solver = Solver(local)
    spec = field_spec(w)
    q = torch.tensor(w.q_face, dtype=dt, device=dev)
    # target frames from the ground-truth field with inclusions (setup, not timed)
    obs = solver.forward(prob, torch.tensor(w.alpha, dtype=dt, device=dev), q_face=q, q_steps=w.q_steps)["frames"]
    theta = torch.tensor(S.xavier_theta(spec.n_freq, spec.width, spec.depth, FIELD_SEED), dtype=torch.float32,
                         device=dev)
    alpha = torch.empty(w.nz, w.ny, w.nx, dtype=torch.float32, device=dev)
    g_theta = torch.empty_like(theta)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    desc = spec.to_c()
    sp = ctypes.c_void_p(stream.cuda_stream)
    field_ms = []

    def run_step(th, obs_, q_, g_out, timed=False):
        """theta -> alpha -> J, dJ/dalpha (+ TV) -> dJ/dtheta, all through the C ABI."""
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)] if timed else None
        if timed: e[0].record(stream)
        NV.check(solver._lib.nefty_field_eval(solver._h, ctypes.byref(desc), ctypes.c_void_p(th.data_ptr()),
                                              None, ctypes.c_void_p(alpha.data_ptr()), sp), solver._h)
        if timed: e[1].record(stream)
        a = alpha if dt == torch.float32 else alpha.double()
        out = solver.adjoint_grad(prob, a, obs_, q_face=q_, q_steps=w.q_steps)
        g = out["grad_alpha"]
        solver.tv(prob, a, TV_LAMBDA, TV_EPS, grad_accum=g)
        g32 = g if g.dtype == torch.float32 else g.float()
        if timed: e[2].record(stream)
        NV.check(solver._lib.nefty_field_backward(solver._h, ctypes.byref(desc), ctypes.c_void_p(th.data_ptr()), None,
                                                  ctypes.c_void_p(g32.data_ptr()), ctypes.c_void_p(g_out.data_ptr()),
                                                  sp), solver._h)
        if timed:
            e[3].record(stream)
            field_ms.append((e, out["stats"]))
        return out

    def step():
        return run_step(theta, obs, q, g_theta, timed=True)

    for _ in range(max(3, args.warmup)):
        step()
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    reuses0 = int(solver._lib.nefty_field_activation_reuses(solver._h))
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        out = step()
        ev[k][1].record(stream)
        stats.append(out["stats"])
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    # every timed backward took the evaluation's kept activations
    reused = int(solver._lib.nefty_field_activation_reuses(solver._h)) - reuses0 == args.steps
    step_ms = [a.elapsed_time(b) for a, b in ev]
    f_fwd = [e[0].elapsed_time(e[1]) for e, _ in field_ms[-args.steps:]]
    f_bwd = [e[2].elapsed_time(e[3]) for e, _ in field_ms[-args.steps:]]
    total_ms = sum(step_ms)
    max_ms, value = aggregate(total_ms, w.n_cells * w.nt * args.steps, world, dev)

    # roofline of the fused CG kernel (forward + adjoint + recompute launches)
    R = args.prec
    cg_ms = sum(s["fwd_ms"] + s["adj_ms"] + s["recompute_ms"] for s in stats) / len(stats)
    launches = stats[0]["kernel_launches"]
    iters = sum(s["fwd_iters"] + s["adj_iters"] + s["recompute_iters"] for s in stats) / len(stats)
    st0 = stats[0]
    steps_solved = st0["fwd_steps"] + st0["adj_steps"] + st0["recompute_steps"]
    alg_bytes = w.n_cells * (iters * ALG_BYTES_ITER[R] + steps_solved * ALG_BYTES_STEP[R]
                             + st0["adj_steps"] * ALG_BYTES_GRAD[R])
    pk = peaks()
    peak = pk["hbm_gbs"] if pk else 6800.0
    achieved = alg_bytes / (cg_ms / 1000.0) / 1e9
    cap = DRAM_CAPTURE[R]
    traffic, traffic_note = None, "no ncu capture of these kernels"
    if cap is not None:
        if source_sha16(cap["kernel_source"]) != cap["kernel_sha16"]:
            traffic_note = "stale: the kernel source changed since the ncu capture"
        else:
            traffic = w.n_cells * (cap["fwd"] * (st0["fwd_steps"] + st0["recompute_steps"])
                                   + cap["adj"] * st0["adj_steps"])
            same = [w.nx, w.ny, w.nz] == cap["grid"] and w.nt == cap["nt"]
            traffic_note = ("DRAM bytes per cell-step of the forward and reverse launches measured by ncu on "
                            + ("this workload" if same else "the 256x256x48x1000 workload (scaled here)")
                            + " (" + ", ".join(cap["profiles"]) + ")")
    dram_gbs = None if traffic is None else traffic / (cg_ms / 1000.0) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "traffic_note": traffic_note,
                "dram_gbs": dram_gbs, "dram_frac": None if dram_gbs is None else dram_gbs / peak,
                "kernel": KERNELS[R],
                "peak_source": ("of measured: MEASURED_PEAKS.json hbm_gbs (burst copy)" if pk
                                else "of fallback: 6.8 TB/s"),
                "alg_bytes_note": (f"{ALG_BYTES_ITER[R]} B per cell per CG iteration, {ALG_BYTES_STEP[R]} B per "
                                   f"cell per solved step, {ALG_BYTES_GRAD[R]} B per cell per adjoint step "
                                   "(gradient assembly)"),
                "cg_ms_per_step": cg_ms, "alg_bytes_per_step": alg_bytes,
                "mean_cg_iters_per_solve": iters / max(1, steps_solved)}

    fwd_fl, bwd_fl = mlp_flops(spec)
    pk_tf = (pk["bf16_tflops_sustained"] if pk and "bf16_tflops_sustained" in pk else 1700.0)
    f_fwd_ms, f_bwd_ms = float(np.mean(f_fwd)), float(np.mean(f_bwd))
    mlp_tf = (fwd_fl + bwd_fl) / ((f_fwd_ms + f_bwd_ms) / 1000.0) / 1e12
    roofline_mlp = {"bound": "tensor", "achieved": mlp_tf, "peak": pk_tf, "unit": "TFLOP/s", "frac": mlp_tf / pk_tf,
                    "traffic": None, "kernel": "tcgen05 BF16 GEMMs of the field (eval + backward calls)",
                    "peak_source": "measured sustained bf16 (MEASURED_PEAKS.json)" if pk else "fallback",
                    "field_eval_ms": f_fwd_ms, "field_backward_ms": f_bwd_ms,
                    "backward_reused_activations": reused,
                    "flops_per_step": fwd_fl + bwd_fl}

    # error of the timed configuration against the FP64 GPU path, outside the
    # timed region: the same alpha (the field's output of theta), targets and
    # flux through the FP32 path as timed and through the FP64 path (rtol
    # 1e-13); surface frames, loss and dJ/dalpha (before the TV term)
    error = None
    if R == "fp32" and not args.no_error:
        a32 = alpha.clone()
        p64 = prob.with_(prec="fp64", rtol=0.0, extrap=0)
        f32 = solver.forward(prob, a32, q_face=q, q_steps=w.q_steps, obs=obs)
        g32 = solver.adjoint_grad(prob, a32, obs, q_face=q, q_steps=w.q_steps)
        a64, q64, o64 = a32.double(), q.double(), obs.double()
        f64 = solver.forward(p64, a64, q_face=q64, q_steps=w.q_steps, obs=o64)
        g64 = solver.adjoint_grad(p64, a64, o64, q_face=q64, q_steps=w.q_steps)

        def rel(x, y):
            return float((x.double() - y).norm() / y.norm())

        gx, gy = g32["grad_alpha"].double().flatten(), g64["grad_alpha"].flatten()
        error = {"against": "FP64 GPU path (rtol 1e-13) on the same alpha, targets and flux",
                 "surface_rel_l2": rel(f32["frames"], f64["frames"]),
                 "loss_rel": abs(f32["loss"] - f64["loss"]) / abs(f64["loss"]),
                 "grad_alpha_rel_l2": rel(gx, gy),
                 "grad_alpha_cosine": float(gx @ gy / (gx.norm() * gy.norm())),
                 "bars": {"surface_rel_l2": 1e-5, "grad_alpha_rel_l2": 1e-3, "grad_alpha_cosine": 0.9999}}
        del f32, g32, f64, g64, a64, q64, o64, gx, gy, a32
        torch.cuda.empty_cache()

    # end to end through the C ABI with host buffers (pinned): theta, targets
    # and flux go in, dJ/dtheta and the loss come back, copies inside
    e2e = None
    if rank == 0 or world > 1:
        th_h = theta.cpu().pin_memory()
        o_h = obs.cpu().pin_memory()
        q_h = q.cpu().pin_memory()
        g_h = torch.empty(theta.shape, dtype=torch.float32).pin_memory()
        run_step(th_h, o_h, q_h, g_h)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            run_step(th_h, o_h, q_h, g_h)
        torch.cuda.synchronize(dev)
        e2e_s = (time.perf_counter() - t0) / args.steps
        h2d = th_h.numel() * 4 + o_h.numel() * o_h.element_size() + q_h.numel() * q_h.element_size()
        d2h = g_h.numel() * 4 + 8
        e2e = {"value": w.n_cells * w.nt * world / e2e_s / 1e9, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        steps = max(1, args.cpu_sample_steps)
        v, s = oracle_sample(args, w, cand, steps)
        cpu = {"value": v, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
               "sample": f"first {steps} of {w.nt} steps of the same grid, forward + adjoint, FP64, {s:.1f} s"}
        if cpu_cores() > 1:
            cpu["single_thread"] = oracle_single_thread(args)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": max_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if R == "fp32" else "f64",
                "data": "synthetic", "config": config_dict(args, w), "parallelism": f"replicas x{world}",
                "gpu_launches": launches * args.steps + field_launches(spec, reused) * args.steps, "e2e": e2e,
                "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                               "max": float(max(step_ms)), "per": "inversion step (device time, CUDA events)"},
                "error": error,
                "roofline": roofline, "roofline_field": roofline_mlp,
                "cpu_baseline": cpu, "clocks": clk,
                "solver_stats": {k: stats[-1][k] for k in ("fwd_iters", "adj_iters", "recompute_iters",
                                                           "max_step_iters", "max_rel_residual",
                                                           "ckpt_every", "grid_blocks", "workspace_bytes",
                                                           "folded_last_iters", "carried_solves")}}
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


# ----------------------------------------------------------------- serving
def run_serving(args):
    """Replay a Poisson stream of ragged forward / inversion jobs through the
    serving queue (arrival times honoured on the host clock) and report the
    submit-to-done latency percentiles from the library's timestamps: served
    with batched launches (the running jobs' sweeps in one persistent grid),
    served on lanes that each run their own grid, and one job at a time in
    FP32 and in FP64.  The forward jobs' surface frames of the batched FP32
    replay are compared with those of the FP64 one (surface-temperature
    error at which the latencies are compared)."""
    import torch
    from paper_2603_11045_gb300 import synthetic as S
    from paper_2603_11045_gb300.serve import Server
    from paper_2603_11045_gb300.solver import Problem, Solver
    if args.serve_scale == "full":
        jobs = S.serving_jobs(n_jobs=64, rate=4.0, seed=3000)
        inv_iters = 10
    else:
        jobs = S.serving_jobs(n_jobs=24, rate=8.0, seed=3000, steps=(50, 200), sizes=S.GRID_SIZES[:3])
        inv_iters = 3
    solver = Solver(0)
    inputs = []
    for j in jobs:   # device inputs, prepared before any timing
        w = S.inclusion_case(nx=j["nx"], ny=j["ny"], nz=j["nz"], nt=j["nt"], seed=j["seed"])
        p = Problem.from_workload(w, prec="fp32")
        a = torch.tensor(w.alpha, dtype=torch.float32, device="cuda")
        q = torch.tensor(w.q_face, dtype=torch.float32, device="cuda")
        obs = None
        if j["kind"] == "inversion":
            obs = solver.forward(p, torch.tensor(w.alpha_target, dtype=torch.float32, device="cuda"), q_face=q,
                                 q_steps=w.q_steps)["frames"]
        inputs.append((j, w, p, a, q, obs))
    torch.cuda.synchronize()

    def replay(lanes, prec, batched, keep_frames=False):
        dt = torch.float32 if prec == "fp32" else torch.float64
        srv = Server(solver, lanes=lanes, batched=batched)
        jobs_in = [(j, w, p.with_(prec=prec), a.to(dt), q.to(dt), None if o is None else o.to(dt))
                   for (j, w, p, a, q, o) in inputs]
        # warm-up: one short job per lane (workspace, kernel modules)
        warm = [srv.submit(jobs_in[0][2].with_(nt=5), jobs_in[0][3].clone(), q_face=jobs_in[0][4], q_steps=3)
                for _ in range(lanes)]
        for i in warm:
            srv.wait(i)
        frames = {}
        if keep_frames:
            for k, (j, w, p, a, q, o) in enumerate(jobs_in):
                if j["kind"] == "forward":
                    frames[k] = torch.empty(p.nt, p.ny, p.nx, dtype=dt, device="cuda")
        torch.cuda.synchronize()
        t0 = time.monotonic()
        ids = []
        for k, (j, w, p, a, q, o) in enumerate(jobs_in):
            delay = t0 + j["arrival_s"] - time.monotonic()
            if delay > 0:
                time.sleep(delay)
            if j["kind"] == "inversion":
                ids.append(srv.submit(p, a.clone(), kind="inversion", iters=inv_iters, lr=1.0, alpha_floor=0.01,
                                      q_face=q, q_steps=w.q_steps, obs=o))
            else:
                ids.append(srv.submit(p, a, q_face=q, q_steps=w.q_steps, frames_out=frames.get(k)))
        res = [srv.wait(i, timeout=3600) for i in ids]
        srv.stop()
        bad = [r for r in res if r["state_name"] != "done"]
        lat = np.array([(r["t_done_ns"] - r["t_submit_ns"]) / 1e9 for r in res])
        wait = np.array([(r["t_admit_ns"] - r["t_submit_ns"]) / 1e9 for r in res])
        span = (max(r["t_done_ns"] for r in res) - min(r["t_submit_ns"] for r in res)) / 1e9
        cell_steps = sum(j["nx"] * j["ny"] * j["nz"] * j["nt"] * (1 if j["kind"] == "forward" else 2 * inv_iters)
                         for j in jobs)
        out = {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
               "mean_s": float(lat.mean()), "max_queue_wait_s": float(wait.max()), "makespan_s": span,
               "gcell_steps_per_s": cell_steps / span / 1e9, "lanes": lanes, "prec": prec, "batched": batched,
               "failed": len(bad)}
        if batched:
            out["launches_per_job_mean"] = float(np.mean([r["launches"] for r in res]))
            out["jobs_sharing_launches"] = int(sum(r["shared_launches"] > 0 for r in res))
        return out, frames

    served, fr32 = replay(args.serve_lanes, "fp32", True, keep_frames=not args.serve_no_fp64)
    lanes_only, _ = replay(args.serve_unbatched_lanes, "fp32", False)
    single, _ = replay(1, "fp32", False)
    fp64, surf = None, None
    if not args.serve_no_fp64:
        fp64, fr64 = replay(1, "fp64", False, keep_frames=True)
        errs = [float((fr32[k].double() - fr64[k]).norm() / fr64[k].norm()) for k in fr32]
        surf = {"forward_jobs": len(errs), "max_rel_l2": max(errs), "median_rel_l2": float(np.median(errs))}
        del fr64
    del fr32
    solver.close()
    n_fwd = sum(j["kind"] == "forward" for j in jobs)
    line = {"metric": "serving p99 latency", "value": served["p99_s"], "unit": "s", "n_gpus": 1,
            "higher_is_better": False, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"serving stream ({args.serve_scale}): {len(jobs)} jobs, Poisson arrivals, "
                                   f"{n_fwd} forward + {len(jobs) - n_fwd} {inv_iters}-step inversions, "
                                   f"grids {sorted({(j['nx'], j['ny'], j['nz']) for j in jobs})}, "
                                   f"{min(j['nt'] for j in jobs)}-{max(j['nt'] for j in jobs)} steps",
                       "lanes": args.serve_lanes},
            "served": served, "served_unbatched_lanes": lanes_only, "one_at_a_time_fp32": single,
            "one_at_a_time_fp64": fp64, "surface_fp32_batched_vs_fp64": surf}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ jacobi
def run_jacobi(args):
    """The paper's inner solver against the converged one (App. D.2: K = 50
    unrolled Jacobi sweeps per solve, whose result the paper takes as the
    exact state).  For K Jacobi sweeps per forward and adjoint solve (FP32):
    the surface frames' and the gradient's distance from the converged FP64
    solve (rtol 1e-13), and the device time per forward + adjoint step, beside
    the FP32 Jacobi-PCG path, on the paper's grid and on the bench grid."""
    import torch
    from paper_2603_11045_gb300 import synthetic as S
    from paper_2603_11045_gb300.solver import Problem, Solver

    def rel(a, b):
        return float((a.double() - b.double()).norm() / b.double().norm())

    def cos(a, b):
        a, b = a.double().flatten(), b.double().flatten()
        return float(a @ b / (a.norm() * b.norm()))

    import dataclasses
    w2 = S.inclusion_case(nx=256, ny=256, nz=48, nt=200, seed=2001)
    # candidate alpha = 1 against targets from the inclusion field: a misfit
    # far above FP32 rounding, so the gradients can be compared
    w2 = dataclasses.replace(w2, alpha=np.ones_like(w2.alpha), alpha_target=w2.alpha)
    cases = [("paper grid 64x64x16, dx 0.156, dz 0.0625, dt 0.05, 100 frames, periodic lateral, post-flash T0",
              S.paper_grid_case()),
             ("inclusion field 256x256x48, dt 0.25, 200 steps, surface pulse, candidate alpha = 1", w2)]
    solver = Solver(0)
    out = []
    for name, w in cases:
        def arr(x, dt):
            return None if x is None else torch.tensor(x, dtype=dt, device="cuda")
        p64 = Problem.from_workload(w, prec="fp64", rtol=1e-13)
        q64, T064 = arr(w.q_face, torch.float64), arr(w.T0, torch.float64)
        obs = solver.forward(p64, arr(w.alpha_target, torch.float64), T0=T064, q_face=q64,
                             q_steps=w.q_steps)["frames"]
        a64 = arr(w.alpha, torch.float64)
        ref_f = solver.forward(p64, a64, T0=T064, q_face=q64, q_steps=w.q_steps)["frames"]
        ref_g = solver.adjoint_grad(p64, a64, obs, T0=T064, q_face=q64, q_steps=w.q_steps)["grad_alpha"]
        q32, T032, a32, obs32 = (arr(w.q_face, torch.float32), arr(w.T0, torch.float32),
                                 arr(w.alpha, torch.float32), obs.float())
        rows = []
        for K in [0, 10, 25, 50, 100, 200]:
            p = Problem.from_workload(w, prec="fp32", jacobi_k=K)
            f = solver.forward(p, a32, T0=T032, q_face=q32, q_steps=w.q_steps)["frames"]
            solver.adjoint_grad(p, a32, obs32, T0=T032, q_face=q32, q_steps=w.q_steps)   # warm-up
            g = solver.adjoint_grad(p, a32, obs32, T0=T032, q_face=q32, q_steps=w.q_steps)
            st = g["stats"]
            rows.append({"solver": "Jacobi-PCG (converged)" if K == 0 else f"Jacobi K={K}",
                         "surface_rel_l2": rel(f, ref_f), "grad_rel_l2": rel(g["grad_alpha"], ref_g),
                         "grad_cosine": cos(g["grad_alpha"], ref_g),
                         "ms_per_step": (st["fwd_ms"] + st["adj_ms"] + st["recompute_ms"]) / w.nt,
                         "iters_per_solve": (st["fwd_iters"] + st["adj_iters"]) / (2 * w.nt)})
        out.append({"case": name, "cells": w.nx * w.ny * w.nz, "steps": w.nt, "rows": rows})
        torch.cuda.empty_cache()
    solver.close()
    print(json.dumps({"metric": "Jacobi-K vs converged solve", "unit": "rel-L2 / ms", "n_gpus": 1,
                      "dtype": "f32", "data": "synthetic", "reference": "FP64 Jacobi-PCG, rtol 1e-13",
                      "cases": out}), flush=True)
    return 0


# --------------------------------------------------------- paper inversion
def run_paper_inversion(args):
    """The paper's inversion loop (App. D.4 hyperparameters) on its synthetic
    grid: the 10 x 512 field with the layer-4 skip and 12 bands 2^k pi, cosine
    frequency annealing over T_FA = 2500 steps (Eq. fa_schedule, beta rising
    linearly from 0 to N), Adam at 5e-5 with a 0.1 step decay per 1000
    iterations, surface MSE + 1e-3 TV (eps 1e-6), and K = 50 Jacobi sweeps per
    solve (the paper's inner solver).  Runs --paper-iters iterations (the paper
    runs 10,000) and reports the loss and the reconstruction against the
    synthetic ground truth (MSE, PSNR, IoU of the defect mask), with the time per
    iteration.  Every step of an iteration runs in libnefty except Adam's
    parameter update (torch.optim on the FP32 parameter vector)."""
    import ctypes
    import torch
    from paper_2603_11045_gb300 import synthetic as S
    from paper_2603_11045_gb300 import _native as NV
    from paper_2603_11045_gb300.field import FieldSpec, annealing_weights
    from paper_2603_11045_gb300.solver import Problem, Solver
    w = S.paper_grid_case(seed=5000, nt=100)
    spec = FieldSpec.paper(w.nx, w.ny, w.nz)
    spec.keep_activations = True   # each backward runs at the evaluated theta
    prob = Problem.from_workload(w, prec="fp32", jacobi_k=args.paper_jacobi_k)
    solver = Solver(0)
    dev = torch.device("cuda", 0)
    gt = torch.tensor(w.alpha, dtype=torch.float32, device=dev)
    T0 = torch.tensor(w.T0, dtype=torch.float32, device=dev)
    obs = solver.forward(prob, gt, T0=T0)["frames"]
    theta = torch.nn.Parameter(torch.tensor(S.xavier_theta(spec.n_freq, spec.width, spec.depth, 7,
                                                            skip=spec.skip_layer), dtype=torch.float32, device=dev))
    opt = torch.optim.Adam([theta], lr=5e-5)
    sched = torch.optim.lr_scheduler.StepLR(opt, step_size=1000, gamma=0.1)
    T_FA, lam, eps = 2500, 1e-3, 1e-6
    alpha = torch.empty(w.nz, w.ny, w.nx, dtype=torch.float32, device=dev)
    desc = spec.to_c()
    stream = torch.cuda.current_stream(dev)
    sp = ctypes.c_void_p(stream.cuda_stream)
    lib, h = solver._lib, solver._h
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    defect = gt < 0.05          # defects 0.005-0.015 against a background of 0.1-0.2
    curve = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for it in range(args.paper_iters):
        beta = spec.n_freq * min(1.0, it / T_FA)
        bw = torch.tensor(annealing_weights(spec.n_freq, beta), dtype=torch.float32, device=dev)
        NV.check(lib.nefty_field_eval(h, ctypes.byref(desc), ptr(theta), ptr(bw), ptr(alpha), sp), h)
        out = solver.adjoint_grad(prob, alpha, obs, T0=T0)
        g = out["grad_alpha"]
        tv = solver.tv(prob, alpha, lam, eps, grad_accum=g)
        grad = torch.empty_like(theta)
        NV.check(lib.nefty_field_backward(h, ctypes.byref(desc), ptr(theta), ptr(bw), ptr(g.contiguous()),
                                          ptr(grad), sp), h)
        theta.grad = grad
        opt.step()
        sched.step()
        if it % max(1, args.paper_iters // 10) == 0 or it == args.paper_iters - 1:
            mse = float(((alpha - gt) ** 2).mean())
            curve.append({"iter": it, "loss": out["loss"], "tv": tv, "alpha_mse": mse})
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    NV.check(lib.nefty_field_eval(h, ctypes.byref(desc), ptr(theta), None, ptr(alpha), sp), h)
    torch.cuda.synchronize()
    mse = float(((alpha - gt) ** 2).mean())
    rng_gt = float(gt.max() - gt.min())
    pred = alpha < 0.05
    inter, union = int((pred & defect).sum()), int((pred | defect).sum())
    solver.close()
    print(json.dumps({"metric": "paper inversion", "unit": "s/iteration", "value": wall / args.paper_iters,
                      "n_gpus": 1, "dtype": "f32 solver, bf16 field", "data": "synthetic",
                      "config": {"workload": "paper grid 64x64x16, 100 frames, dt 0.05, periodic lateral, "
                                             "post-flash T0, 1-4 defects; field 12 bands 2^k pi, 10 x 512, "
                                             "skip at layer 4; Adam 5e-5, decay 0.1/1000, T_FA 2500, TV 1e-3",
                                 "inner_solver": (f"{args.paper_jacobi_k} Jacobi sweeps" if args.paper_jacobi_k
                                                  else "Jacobi-PCG"),
                                 "iterations": args.paper_iters, "params": spec.n_params},
                      "curve": curve,
                      "final": {"alpha_mse": mse, "psnr_db": 10 * math.log10(rng_gt ** 2 / max(mse, 1e-30)),
                                "defect_iou": inter / union if union else 1.0, "defect_cells": int(defect.sum())},
                      "wall_s": wall}), flush=True)
    return 0


# ------------------------------------------------------------------ stress
def run_stress(args):
    """The largest configuration: 512x512x96 cells, 2000 steps of dt = 0.2,
    8 layers with 20 one-cell delaminations, checkpoint stride chosen by the
    memory budget (every state kept does not fit, so about sqrt(nt)).  One
    forward + adjoint gradient, timed with the library's CUDA events; device
    memory the call holds; recompute overhead; with --stress-fp64 the FP64 path
    on the same inputs and the agreement of the two gradients."""
    import torch
    from paper_2603_11045_gb300 import synthetic as S
    from paper_2603_11045_gb300.solver import Problem, Solver
    w = S.layered_delamination_case()
    solver = Solver(0)
    res = {}
    for prec in (["fp32", "fp64"] if args.stress_fp64 else ["fp32"]):
        dt = torch.float32 if prec == "fp32" else torch.float64
        p = Problem.from_workload(w, prec=prec, rtol=1e-13 if prec == "fp64" else 0.0)
        q = torch.tensor(w.q_face, dtype=dt, device="cuda")
        obs = solver.forward(p, torch.tensor(w.alpha_target, dtype=dt, device="cuda"), q_face=q,
                             q_steps=w.q_steps)["frames"]
        a = torch.tensor(w.alpha, dtype=dt, device="cuda")
        free0 = torch.cuda.mem_get_info()[0]
        t0 = time.perf_counter()
        out = solver.adjoint_grad(p, a, obs, q_face=q, q_steps=w.q_steps)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        st = out["stats"]
        dev_ms = st["fwd_ms"] + st["adj_ms"] + st["recompute_ms"]
        res[prec] = (out, {"prec": prec, "wall_s": wall, "device_ms": dev_ms,
                           "gcell_steps_per_s": w.n_cells * w.nt / (dev_ms / 1e3) / 1e9,
                           "ckpt_every": st["ckpt_every"], "states_held": st["n_checkpoints"],
                           "workspace_gb": st["workspace_bytes"] / 1e9,
                           "device_free_gb_before": free0 / 1e9,
                           "recompute_overhead": st["recompute_ms"] / max(1e-9, st["fwd_ms"] + st["adj_ms"]),
                           "iters": {"fwd": st["fwd_iters"], "recompute": st["recompute_iters"],
                                     "adj": st["adj_iters"]},
                           "fwd_ms": st["fwd_ms"], "recompute_ms": st["recompute_ms"], "adj_ms": st["adj_ms"],
                           "loss": out["loss"]})
        del obs, a, q
        torch.cuda.empty_cache()
    line = {"metric": "stress fwd+adjoint Gcell-steps/s", "value": res["fp32"][1]["gcell_steps_per_s"],
            "unit": "Gcell-steps/s", "n_gpus": 1, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"stress: {w.nx}x{w.ny}x{w.nz} cells, {w.nt} steps dt={w.dt}, 8 layers + 20 "
                                   "delaminations, Gaussian pulse 3 steps, checkpoint stride by memory budget"},
            "fp32": res["fp32"][1]}
    if "fp64" in res:
        g32, g64 = res["fp32"][0]["grad_alpha"].double(), res["fp64"][0]["grad_alpha"]
        line["fp64"] = res["fp64"][1]
        line["fp32_vs_fp64"] = {"grad_rel_l2": float((g32 - g64).norm() / g64.norm()),
                                "grad_cosine": float((g32 * g64).sum() / (g32.norm() * g64.norm())),
                                "loss_rel": abs(res["fp32"][1]["loss"] - res["fp64"][1]["loss"]) / abs(res["fp64"][1]["loss"])}
    solver.close()
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "stress":
        return run_stress(args)
    if args.workload == "jacobi":
        return run_jacobi(args)
    if args.workload == "paper-inversion":
        return run_paper_inversion(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
