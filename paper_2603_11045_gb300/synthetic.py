"""Seeded synthetic workloads shaped like the paper's thermography benchmark.

This module only draws inputs: diffusivity fields, surface flux maps, initial
temperatures and job streams.  It holds none of the solver's arithmetic, so both
the CUDA path and the CPU oracle can consume the same arrays.

The paper's own dataset (Sec. 5.1 "Datasets"; App. F.1: 64x64x16 grid, 1-4
defects with alpha_defect/alpha_base about 1:20, homogeneous or 3-4 layers) is
not available; every generator below draws fields with that structure from a
seeded ``numpy.random.Generator(PCG64(seed))``.

All arrays are float64 in ``[z][y][x]`` order (x fastest).  Callers cast to the
precision of the path they run.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

__all__ = [
    "Workload", "box_inclusion_case", "random_inclusions", "gaussian_pulse",
    "inclusion_case", "neural_field_case", "layered_delamination_case",
    "paper_grid_case", "serving_jobs", "rng", "xavier_theta",
]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class Workload:
    """One synthetic problem: grid, spacing, time step and forcing."""
    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    dt: float
    nt: int
    alpha: np.ndarray                      # [nz, ny, nx] cell diffusivity
    q_face: Optional[np.ndarray] = None    # [ny, nx] surface flux on the z=0 face
    q_steps: int = 0                       # flux applied for steps n < q_steps
    T0: Optional[np.ndarray] = None        # [nz, ny, nx] initial temperature (None = 0)
    bc: int = 0                            # 0 = zero-flux walls, 1 = periodic in x and y
    alpha_target: Optional[np.ndarray] = None  # field whose surface frames are the targets
    extra: dict = field(default_factory=dict)

    @property
    def n_cells(self) -> int:
        return self.nx * self.ny * self.nz


def box_inclusion_case(nx=32, ny=32, nz=8, nt=100, dt=0.5) -> Workload:
    """32x32x8 box-inclusion case: background alpha 1.0, one box of alpha 0.1 over
    x 12-19, y 12-19, z 3-4; unit surface flux on z=0 for the first 2 steps; the
    target frames come from the same run at uniform alpha 1.0."""
    alpha = np.ones((nz, ny, nx))
    alpha[3:5, 12:20, 12:20] = 0.1
    return Workload("box_inclusion_32x32x8", nx, ny, nz, 1.0, 1.0, 1.0, dt, nt,
                    alpha=alpha, q_face=np.ones((ny, nx)), q_steps=2,
                    alpha_target=np.ones((nz, ny, nx)))


def random_inclusions(shape, g: np.random.Generator, n_range, extent_range,
                      depth_range, ratio_range, base: np.ndarray) -> np.ndarray:
    """Multiply ``base`` inside 'n' random boxes or ellipsoids by a random ratio.

    n ~ U{n_range}, per-axis extents ~ U{extent_range} cells (z extent capped at
    the slab), top depth ~ U{depth_range}, ratio ~ U(ratio_range)."""
    nz, ny, nx = shape
    a = base.copy()
    n = int(g.integers(n_range[0], n_range[1] + 1))
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for _ in range(n):
        ex = int(g.integers(extent_range[0], extent_range[1] + 1))
        ey = int(g.integers(extent_range[0], extent_range[1] + 1))
        ez = int(g.integers(max(1, extent_range[0] // 4), max(2, extent_range[1] // 4) + 1))
        top = int(g.integers(depth_range[0], depth_range[1] + 1))
        top = min(top, nz - 1)
        ez = max(1, min(ez, nz - top))
        cx = int(g.integers(0, max(1, nx - ex) + 1))
        cy = int(g.integers(0, max(1, ny - ey) + 1))
        ratio = float(g.uniform(ratio_range[0], ratio_range[1]))
        kind = int(g.integers(0, 2))
        if kind == 0:   # box
            m = ((xx >= cx) & (xx < cx + ex) & (yy >= cy) & (yy < cy + ey)
                 & (zz >= top) & (zz < top + ez))
        else:           # ellipsoid inscribed in the same box
            rx, ry, rz = ex / 2.0, ey / 2.0, ez / 2.0
            m = (((xx + 0.5 - cx - rx) / rx) ** 2 + ((yy + 0.5 - cy - ry) / ry) ** 2
                 + ((zz + 0.5 - top - rz) / rz) ** 2) <= 1.0
        a[m] *= ratio
    return a


def gaussian_pulse(nx: int, ny: int, sigma: float = 20.0) -> np.ndarray:
    """Peak-1 Gaussian surface flux map centred on the face, width sigma cells."""
    x = np.arange(nx) + 0.5 - nx / 2.0
    y = np.arange(ny) + 0.5 - ny / 2.0
    return np.exp(-(y[:, None] ** 2 + x[None, :] ** 2) / (2.0 * sigma ** 2))


def inclusion_case(nx=128, ny=128, nz=32, nt=500, dt=0.25, seed=1000,
                   n_range=(3, 8), name=None) -> Workload:
    """Background alpha ~ U(0.8,1.2) per cell plus 3-8 box/ellipsoid inclusions,
    extents 4-24 cells, depth 1-20, ratio ~ U(0.02,0.3); Gaussian surface pulse
    (sigma 20 cells) on z=0 for 3 steps.  Targets: the same run at the
    background field without inclusions."""
    g = rng(seed)
    base = g.uniform(0.8, 1.2, size=(nz, ny, nx))
    alpha = random_inclusions((nz, ny, nx), g, n_range, (4, 24), (1, 20), (0.02, 0.3), base)
    return Workload(name or f"inclusions_{nx}x{ny}x{nz}", nx, ny, nz, 1.0, 1.0, 1.0, dt, nt,
                    alpha=alpha, q_face=gaussian_pulse(nx, ny, 20.0), q_steps=3,
                    alpha_target=base, extra={"seed": seed})


def neural_field_case(nx=256, ny=256, nz=48, nt=1000, dt=0.25, seed=2000) -> Workload:
    """Inversion-step case: ground-truth alpha ~ U(0.8,1.2) background with 5-12
    inclusions; the solver's alpha comes from the neural field, so ``alpha``
    here is the ground truth that produces the target frames."""
    g = rng(seed)
    base = g.uniform(0.8, 1.2, size=(nz, ny, nx))
    truth = random_inclusions((nz, ny, nx), g, (5, 12), (4, 24), (1, 20), (0.02, 0.3), base)
    return Workload(f"neural_field_{nx}x{ny}x{nz}", nx, ny, nz, 1.0, 1.0, 1.0, dt, nt,
                    alpha=truth, q_face=gaussian_pulse(nx, ny, 20.0), q_steps=3,
                    alpha_target=truth, extra={"seed": seed})


def layered_delamination_case(nx=512, ny=512, nz=96, nt=2000, dt=0.2, seed=4000,
                              n_layers=8, n_delam=20) -> Workload:
    """Layered background (8 z-layers, alpha ~ U(0.5,1.5)) with 20 one-cell-thick
    delaminations, 10-60 cells wide, alpha 0.01 (overwrite)."""
    g = rng(seed)
    alpha = np.empty((nz, ny, nx))
    edges = np.linspace(0, nz, n_layers + 1).round().astype(int)
    for l in range(n_layers):
        alpha[edges[l]:edges[l + 1]] = g.uniform(0.5, 1.5)
    target = alpha.copy()
    for _ in range(n_delam):
        wx = int(g.integers(10, 61)); wy = int(g.integers(10, 61))
        x0 = int(g.integers(0, max(1, nx - wx) + 1)); y0 = int(g.integers(0, max(1, ny - wy) + 1))
        k = int(g.integers(1, nz - 1))
        alpha[k, y0:y0 + wy, x0:x0 + wx] = 0.01
    return Workload(f"layered_{nx}x{ny}x{nz}", nx, ny, nz, 1.0, 1.0, 1.0, dt, nt,
                    alpha=alpha, q_face=gaussian_pulse(nx, ny, 20.0), q_steps=3,
                    alpha_target=target, extra={"seed": seed})


def paper_grid_case(seed=5000, nt=100, layered=False) -> Workload:
    """The paper's synthetic grid (App. D.4 table of hyperparameters): 64x64x16,
    dx=dy=0.156, dz=0.0625, dt=0.05, lateral periodic, z adiabatic; alpha_base ~
    U(0.1,0.2), 1-4 defects with alpha ~ U(0.005,0.015); Gaussian post-flash
    initial temperature near the front face (App. A.5)."""
    g = rng(seed)
    nx, ny, nz = 64, 64, 16
    dx = dy = 10.0 / nx
    dz = 1.0 / nz
    if layered:
        alpha = np.empty((nz, ny, nx))
        nl = int(g.integers(3, 5))
        edges = np.linspace(0, nz, nl + 1).round().astype(int)
        for l in range(nl):
            alpha[edges[l]:edges[l + 1]] = g.uniform(0.1, 0.2)
    else:
        alpha = np.full((nz, ny, nx), g.uniform(0.1, 0.2))
    target = alpha.copy()
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for _ in range(int(g.integers(1, 5))):
        val = g.uniform(0.005, 0.015)
        cx, cy = g.uniform(12, 52, size=2)
        r = g.uniform(3, 8)
        top = int(g.integers(2, 10)); th = int(g.integers(1, 4))
        m = (((xx + 0.5 - cx) ** 2 + (yy + 0.5 - cy) ** 2) <= r * r) & (zz >= top) & (zz < top + th)
        alpha[m] = val
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dy
    z = (np.arange(nz) + 0.5) * dz
    w_xy, w_z = 1.5, 0.1
    T0 = (np.exp(-((x[None, None, :] - 5.0) ** 2 + (y[None, :, None] - 5.0) ** 2) / (2 * w_xy ** 2))
          * np.exp(-(z[:, None, None] ** 2) / (2 * w_z ** 2)))
    return Workload("paper_grid_64x64x16", nx, ny, nz, dx, dy, 1.0 / nz, 0.05, nt,
                    alpha=alpha, T0=T0, bc=1, alpha_target=target, extra={"seed": seed})


GRID_SIZES = [(64, 64, 16), (128, 128, 32), (192, 160, 40), (256, 256, 64)]


def serving_jobs(n_jobs=64, rate=4.0, seed=3000, steps=(200, 1000), sizes=GRID_SIZES):
    """Poisson arrivals (rate per second) of forward or 10-iteration inversion jobs
    on ragged grids; alpha fields as in ``inclusion_case``."""
    g = rng(seed)
    t = 0.0
    jobs = []
    for j in range(n_jobs):
        t += float(g.exponential(1.0 / rate))
        nx, ny, nz = sizes[int(g.integers(0, len(sizes)))]
        nt = int(g.integers(steps[0], steps[1] + 1))
        kind = "forward" if g.uniform() < 0.5 else "inversion"
        jobs.append({"id": j, "arrival_s": t, "nx": nx, "ny": ny, "nz": nz, "nt": nt,
                     "kind": kind, "iters": 10 if kind == "inversion" else 0,
                     "seed": int(seed * 100 + j)})
    return jobs


def xavier_theta(F, W, depth, seed, skip=0):
    """Seeded Xavier-uniform weights and zero biases for the neural field
    (App. D.1), packed as W_0 [W x 6F], b_0, W_l [W x in_l], b_l (l = 1..depth-1;
    in_l = W + 6F at the skip layer, else W), w_out [W], b_out [1]; weights
    row-major [out][in]."""
    import math
    g = rng(seed)
    D = 6 * F
    parts = []
    for l in range(depth):
        n_in = D if l == 0 else (W + D if l == skip else W)
        lim = math.sqrt(6.0 / (n_in + W))
        parts += [g.uniform(-lim, lim, size=W * n_in), np.zeros(W)]
    lim = math.sqrt(6.0 / (W + 1))
    parts += [g.uniform(-lim, lim, size=W), np.zeros(1)]
    return np.concatenate(parts)
