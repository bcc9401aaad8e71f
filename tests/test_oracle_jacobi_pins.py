"""Pins for the oracle's Jacobi-K mode (App. D.2, Eq. jacobi_iter: K sweeps of
x <- D^{-1}(b - R x) from the warm start, no stopping test).

Each check is a fact the mathematics fixes, not a re-typed formula: the exact
per-step amplification of a lateral Fourier mode under K sweeps (and the
matching adjoint recurrence), the textbook max-norm contraction bound of the
Jacobi error, and the limit K -> infinity, where the sweeps converge to the
exact solve that the CG mode computes.
"""
import math

import numpy as np
import pytest

from paper_2603_11045_gb300 import synthetic as S


def _mode_case(orc, K, nt=5):
    """A 2D periodic grid (nz = 1, so no z faces and every cell has the same
    diagonal), uniform alpha, T0 a lateral Fourier mode, no forcing."""
    nx, ny, alpha, dt, h = 16, 12, 0.7, 0.5, 1.0
    mx, my = 2, 1
    p = orc.problem(nx, ny, 1, dx=h, dy=h, dz=1.0, dt=dt, nt=nt, bc=1)
    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    v = np.cos(2 * math.pi * (mx * i / nx + my * j / ny))[None]
    lam = alpha / h**2 * (2 - 2 * math.cos(2 * math.pi * mx / nx)) + alpha / h**2 * (2 - 2 * math.cos(2 * math.pi * my / ny))
    d = 1 + dt * 4 * alpha / h**2          # diagonal of A: four lateral faces of alpha / h^2
    rho = (d - 1 - dt * lam) / d           # the Jacobi factor on this mode
    return p, np.full((1, ny, nx), alpha), v, lam, dt, rho


@pytest.mark.parametrize("K", [1, 3, 12])
def test_jacobi_mode_amplification(orc, K):
    """The mode is an eigenvector of D and R alike, so K sweeps from T^n map
    c v to c g_K v with g_K = 1/(1 + dt lam) + rho^K dt lam/(1 + dt lam): the
    converged factor plus the Jacobi error left after K sweeps."""
    p, a, v, lam, dt, rho = _mode_case(orc, K)
    out = orc.forward(p, a, T0=v, jacobi_k=K)
    g = 1 / (1 + dt * lam) + rho**K * dt * lam / (1 + dt * lam)
    for n in range(p.nt):
        np.testing.assert_allclose(out["frames"][n], g ** (n + 1) * v[0], rtol=0, atol=1e-13)
    # K sweeps are not the converged solve: the frames differ from it
    exact = orc.forward(p, a, T0=v)["frames"]
    if K < 12:
        assert np.abs(out["frames"] - exact).max() > 1e-6


@pytest.mark.parametrize("K", [2, 5])
def test_jacobi_mode_adjoint(orc, K):
    """With the whole grid observed and zero targets, the adjoint source is
    2 s T^n = 2 s g^n v, a mode again; K sweeps from mu^(n+1) = m v give
    m_n = a* + rho^K (m_{n+1} - a*), a* = (m_{n+1} + 2 s g^n)/(1 + dt lam).
    Checks the loss and dJ/dT0 = mu^1."""
    p, a, v, lam, dt, rho = _mode_case(orc, K, nt=4)
    obs = np.zeros((p.nt, p.ny, p.nx))
    out = orc.adjoint_grad(p, a, T0=v, obs=obs, jacobi_k=K)
    g = 1 / (1 + dt * lam) + rho**K * dt * lam / (1 + dt * lam)
    s = p.loss_scale
    vv = float((v * v).sum())
    assert out["loss"] == pytest.approx(s * vv * sum(g ** (2 * n) for n in range(1, p.nt + 1)), rel=1e-13)
    m = 0.0
    for n in range(p.nt, 0, -1):
        astar = (m + 2 * s * g**n) / (1 + dt * lam)
        m = astar + rho**K * (m - astar)
    np.testing.assert_allclose(out["grad_T0"], m * v, rtol=0, atol=1e-14 * max(1.0, abs(m)))


def test_jacobi_error_contraction(orc):
    """One step on a heterogeneous grid: the error after K sweeps is at most
    rho_inf^K times the error of the warm start in the max norm, rho_inf the
    largest row sum of |D^{-1} R| (< 1 by strict diagonal dominance)."""
    nx, ny, nz = 6, 5, 4
    w = S.inclusion_case(nx=nx, ny=ny, nz=nz, nt=1, seed=77)
    p = orc.from_workload(w)
    A = orc.assemble_A(p, w.alpha).toarray()
    D = np.diag(A)
    rho_inf = ((np.abs(A).sum(axis=1) - np.abs(D)) / D).max()
    assert rho_inf < 1
    T0 = S.rng(5).uniform(0, 1, size=(nz, ny, nx))
    Tstar = orc.forward(p, w.alpha, T0=T0, q_face=w.q_face, q_steps=1, keep_states=True, dense=True)["states"][1]
    e0 = np.abs(T0 - Tstar).max()
    prev = None
    for K in (1, 2, 4, 8, 16):
        TK = orc.forward(p, w.alpha, T0=T0, q_face=w.q_face, q_steps=1, keep_states=True, jacobi_k=K)["states"][1]
        eK = np.abs(TK - Tstar).max()
        assert eK <= rho_inf**K * e0 * (1 + 1e-12) + 1e-15
        if prev is not None:
            assert eK < prev
        prev = eK


def test_jacobi_large_k_is_the_exact_solve(orc):
    """K -> infinity: the sweeps converge to the unique solution (strict
    diagonal dominance, App. D.2), so frames, loss and gradient equal those of
    the converged (CG) mode."""
    w = S.inclusion_case(nx=8, ny=6, nz=4, nt=6, seed=78)
    p = orc.from_workload(w)
    tgt = orc.forward(p, w.alpha_target, q_face=w.q_face, q_steps=w.q_steps)["frames"]
    cg = orc.adjoint_grad(p, w.alpha, q_face=w.q_face, q_steps=w.q_steps, obs=tgt)
    jk = orc.adjoint_grad(p, w.alpha, q_face=w.q_face, q_steps=w.q_steps, obs=tgt, jacobi_k=3000)
    assert jk["loss"] == pytest.approx(cg["loss"], rel=1e-11)
    g, gj = cg["grad_alpha"], jk["grad_alpha"]
    assert np.linalg.norm(gj - g) <= 1e-10 * np.linalg.norm(g)
    f_cg = orc.forward(p, w.alpha, q_face=w.q_face, q_steps=w.q_steps)["frames"]
    f_jk = orc.forward(p, w.alpha, q_face=w.q_face, q_steps=w.q_steps, jacobi_k=3000)["frames"]
    assert np.abs(f_jk - f_cg).max() <= 1e-13 * np.abs(f_cg).max()
