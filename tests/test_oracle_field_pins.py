"""Pins for the FP64 neural-field reference (oracle/field.py)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2603_11045_gb300 import synthetic as S


@pytest.fixture(scope="module")
def F():
    import oracle.field as f
    return f


def test_paper_frequencies_are_powers_of_two(F):
    """Eq. posenc: 2^k pi, k < N, is the log-spaced ladder with ratio 2^(N-1)."""
    N = 12
    w = F.band_frequencies(N, math.pi, math.pi * 2 ** (N - 1))
    assert torch.allclose(w, math.pi * 2.0 ** torch.arange(N, dtype=torch.float64), rtol=1e-15, atol=0)


def test_annealing_weights_closed_form(F):
    """Eq. fa_schedule: 0 before band k starts, 1/2 half-way, 1 after."""
    w = F.annealing_weights(6, 2.5)
    assert torch.allclose(w, torch.tensor([1, 1, 0.5, 0, 0, 0], dtype=torch.float64), atol=1e-15)
    assert torch.all(F.annealing_weights(6, 0.0) == 0) and torch.all(F.annealing_weights(6, 6.0) == 1)


def test_encoding_identities(F):
    """sin^2 + cos^2 = wt^2 per band and axis; the centre cell of an odd axis
    sits at x = 0 (sin 0, cos 1); x is antisymmetric about the centre."""
    X = F.cell_centres(5, 3, 7)
    assert torch.allclose(X[:, 0].reshape(7, 3, 5)[0, 0], -X[:, 0].reshape(7, 3, 5)[0, 0].flip(0), atol=1e-15)
    wt = torch.linspace(0.2, 1.0, 4, dtype=torch.float64)
    E = F.encode(X, 4, 1.0, 9.0, wt).reshape(-1, 3, 4, 2)
    assert torch.allclose((E ** 2).sum(-1), (wt ** 2).expand(E.shape[0], 3, 4), atol=1e-14)
    centre = (3 * 3 + 1) * 5 + 2          # (k=3, j=1, i=2): the centre of every axis
    assert torch.allclose(E[centre, :, :, 0], torch.zeros(3, 4, dtype=torch.float64), atol=1e-15)
    assert torch.allclose(E[centre, :, :, 1], wt.expand(3, 4), atol=1e-15)


def test_constant_output_without_weights(F):
    """All weights zero: alpha = alpha_min + (alpha_max - alpha_min) sigmoid(b_out)."""
    Fq, W, depth = 4, 8, 3
    th = torch.zeros(F.param_count(Fq, W, depth), dtype=torch.float64)
    th[-1] = 0.7
    a = F.field(th, 3, 4, 2, Fq, W, depth, 1.0, 8.0, 0.01, 2.0)
    assert torch.allclose(a, torch.full_like(a, 0.01 + 1.99 / (1 + math.exp(-0.7))), atol=1e-15)


def test_single_unit_network_closed_form(F):
    """One hidden unit reading the cos feature of the first y band pins the
    feature order and the packing: alpha = lo + (hi-lo) sigmoid(relu(cos(w0 y)) + b)."""
    Fq, W, depth = 4, 8, 2
    th = torch.zeros(F.param_count(Fq, W, depth), dtype=torch.float64)
    D = 6 * Fq
    th[0 * D + (1 * 2 * Fq + 0 * 2 + 1)] = 1.0      # W_0[0, axis y, band 0, cos]
    p1 = W * D + W                                  # start of W_1
    th[p1 + 0 * W + 0] = 1.0                        # W_1[0, 0] passes unit 0 through
    p_out = p1 + W * W + W
    th[p_out + 0] = 1.0                             # w_out[0]
    th[-1] = -0.3
    nx, ny, nz = 2, 5, 3
    a = F.field(th, nx, ny, nz, Fq, W, depth, 2.0, 16.0, 0.05, 1.5)
    y = 2.0 * (np.arange(ny) + 0.5) / ny - 1.0
    expect = 0.05 + 1.45 / (1 + np.exp(-(np.maximum(np.cos(2.0 * y), 0.0) - 0.3)))
    assert np.allclose(a.numpy(), np.broadcast_to(expect[None, :, None], (nz, ny, nx)), atol=1e-14)


def test_field_gradient_finite_differences(F):
    """Autograd of the FP64 field vs central differences on random parameters."""
    Fq, W, depth = 4, 8, 3
    th0 = torch.tensor(S.xavier_theta(Fq, W, depth, 5), dtype=torch.float64)
    g_a = torch.tensor(S.rng(6).standard_normal((2, 3, 4)))
    th = th0.clone().requires_grad_(True)
    J = (F.field(th, 4, 3, 2, Fq, W, depth, 1.0, 8.0, 0.01, 2.0) * g_a).sum()
    J.backward()
    idx = S.rng(7).integers(0, th0.numel(), 12)
    for i in idx:
        e = 1e-6
        tp = th0.clone(); tp[i] += e
        tm = th0.clone(); tm[i] -= e
        fd = ((F.field(tp, 4, 3, 2, Fq, W, depth, 1.0, 8.0, 0.01, 2.0) * g_a).sum()
              - (F.field(tm, 4, 3, 2, Fq, W, depth, 1.0, 8.0, 0.01, 2.0) * g_a).sum()) / (2 * e)
        assert float(th.grad[i]) == pytest.approx(float(fd), rel=1e-6, abs=1e-9)
