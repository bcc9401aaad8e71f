"""The seeded input generators draw what the input recipe states: grid,
spacing, time step, forcing, and the value ranges and structure of the
diffusivity fields and the serving stream.  Host only."""
import math

import numpy as np
import pytest

from paper_2603_11045_gb300 import synthetic as S


def test_box_case():
    w = S.box_inclusion_case()
    assert (w.nx, w.ny, w.nz, w.dt, w.nt, w.q_steps) == (32, 32, 8, 0.5, 100, 2)
    assert (w.dx, w.dy, w.dz) == (1.0, 1.0, 1.0)
    box = np.zeros((8, 32, 32), bool)
    box[3:5, 12:20, 12:20] = True
    assert np.all(w.alpha[box] == 0.1) and np.all(w.alpha[~box] == 1.0)
    assert np.all(w.alpha_target == 1.0) and np.all(w.q_face == 1.0) and w.bc == 0


def test_gaussian_pulse():
    q = S.gaussian_pulse(64, 48, 20.0)
    assert q.shape == (48, 64)
    assert np.allclose(q, q[::-1, ::-1])                      # centred on the face
    assert q.max() == pytest.approx(math.exp(-0.25 / 400.0))  # cell centres 0.5 off the middle
    # one sigma along x from the middle row pair
    assert q[24, 32 + 20] / q[24, 32] == pytest.approx(math.exp(-(20.5 ** 2 - 0.5 ** 2) / 800.0))


def test_inclusion_case():
    w = S.inclusion_case(nx=48, ny=40, nz=12, nt=30, seed=1007)
    base = w.alpha_target
    assert (w.nx, w.ny, w.nz, w.dt, w.q_steps) == (48, 40, 12, 0.25, 3)
    assert base.min() >= 0.8 and base.max() <= 1.2
    r = w.alpha / base
    inside = r != 1.0
    assert inside.any()
    assert r[inside].max() <= 0.3 + 1e-12 and r[inside].min() > 0.0   # products of U(0.02, 0.3) ratios
    assert not inside[0].any()                                        # inclusions start at depth >= 1
    assert np.allclose(w.q_face, S.gaussian_pulse(48, 40, 20.0))


def test_neural_field_case():
    w = S.neural_field_case(nx=40, ny=36, nz=10, nt=8, seed=2001)
    assert np.array_equal(w.alpha, w.alpha_target)     # the ground truth; the candidate comes from the field
    assert w.alpha.min() > 0.0 and w.alpha.max() <= 1.2 and w.q_steps == 3 and w.dt == 0.25


def test_layered_delamination_case():
    w = S.layered_delamination_case(nx=80, ny=72, nz=96, nt=10, seed=4001)
    t = w.alpha_target
    for l in range(8):
        layer = t[12 * l:12 * (l + 1)]
        assert np.all(layer == layer.flat[0]) and 0.5 <= layer.flat[0] <= 1.5
    d = w.alpha != t
    assert d.any() and np.all(w.alpha[d] == 0.01)
    planes = np.nonzero(d.any(axis=(1, 2)))[0]
    assert planes.min() >= 1 and planes.max() <= 94    # one cell thick, inside the slab


@pytest.mark.parametrize("layered", [False, True])
def test_paper_grid_case(layered):
    w = S.paper_grid_case(seed=5003, nt=20, layered=layered)
    assert (w.nx, w.ny, w.nz, w.dt, w.bc) == (64, 64, 16, 0.05, 1)
    assert w.dx == pytest.approx(0.156, abs=1e-3) and w.dz == 0.0625
    assert w.alpha_target.min() >= 0.1 and w.alpha_target.max() <= 0.2
    d = w.alpha != w.alpha_target
    assert d.any() and w.alpha[d].min() >= 0.005 and w.alpha[d].max() <= 0.015
    assert 1 <= len(np.unique(w.alpha[d])) <= 4        # 1-4 defects, one value each
    k, y, x = np.unravel_index(np.argmax(w.T0), w.T0.shape)
    assert k == 0 and abs(x - 31.5) <= 1 and abs(y - 31.5) <= 1 and w.T0.max() <= 1.0


def test_serving_stream():
    jobs = S.serving_jobs(n_jobs=64, rate=4.0, seed=3000)
    t = np.array([j["arrival_s"] for j in jobs])
    assert len(jobs) == 64 and np.all(np.diff(t) > 0)
    assert 0.6 / 4.0 <= np.mean(np.diff(np.r_[0.0, t])) <= 1.4 / 4.0
    for j in jobs:
        assert (j["nx"], j["ny"], j["nz"]) in S.GRID_SIZES and 200 <= j["nt"] <= 1000
        assert j["iters"] == (10 if j["kind"] == "inversion" else 0)
    kinds = {j["kind"] for j in jobs}
    assert kinds == {"forward", "inversion"}
    assert jobs == S.serving_jobs(n_jobs=64, rate=4.0, seed=3000)


def test_xavier_theta_layout():
    F, W, depth, skip = 5, 16, 4, 2
    th = S.xavier_theta(F, W, depth, 9, skip=skip)
    D = 6 * F
    ins = [D] + [W + D if l == skip else W for l in range(1, depth)]
    assert th.size == sum(W * n + W for n in ins) + W + 1
    o = 0
    for n in ins:
        lim = math.sqrt(6.0 / (n + W))
        assert np.abs(th[o:o + W * n]).max() <= lim and np.all(th[o + W * n:o + W * n + W] == 0)
        o += W * n + W
    assert np.abs(th[o:o + W]).max() <= math.sqrt(6.0 / (W + 1)) and th[-1] == 0


def test_seeded_and_reproducible():
    a = S.inclusion_case(nx=24, ny=20, nz=6, nt=4, seed=11)
    b = S.inclusion_case(nx=24, ny=20, nz=6, nt=4, seed=11)
    c = S.inclusion_case(nx=24, ny=20, nz=6, nt=4, seed=12)
    assert np.array_equal(a.alpha, b.alpha) and not np.array_equal(a.alpha, c.alpha)
