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


def test_skip_with_zero_encoding_columns_is_the_plain_network(F):
    """App. D.1 skip connection: with the encoding columns of the skip layer's
    weights zero, the network is exactly the one without the skip on the same
    hidden weights."""
    Fq, W, depth, s = 4, 8, 4, 2
    D = 6 * Fq
    th = torch.tensor(S.xavier_theta(Fq, W, depth, 11, skip=s), dtype=torch.float64)
    assert th.numel() == F.param_count(Fq, W, depth, s)
    layers, w_out, b_out = F.unpack(th, Fq, W, depth, s)
    Ws, bs = layers[s]
    Ws = Ws.clone(); Ws[:, W:] = 0.0
    plain = []
    for l, (Wl, bl) in enumerate(layers):
        Wl = Ws[:, :W] if l == s else Wl
        plain += [Wl.reshape(-1), bl + 0.1 * l]
    plain += [w_out, b_out]
    packed = []
    for l, (Wl, bl) in enumerate(layers):
        packed += [(Ws if l == s else Wl).reshape(-1), bl + 0.1 * l]
    packed += [w_out, b_out]
    a_skip = F.field(torch.cat(packed), 3, 4, 2, Fq, W, depth, 1.0, 8.0, 0.01, 2.0, skip=s)
    a_plain = F.field(torch.cat(plain), 3, 4, 2, Fq, W, depth, 1.0, 8.0, 0.01, 2.0)
    assert torch.allclose(a_skip, a_plain, rtol=0, atol=1e-15)


def test_skip_reinjects_the_encoding_closed_form(F):
    """All layers before the skip layer zero (so h_s = 0): one unit of the skip
    layer reading the sin feature of x band 1 in the re-injected block gives
    alpha = lo + (hi-lo) sigmoid(relu(sin(w1 x)) - 0.2), which pins where the
    encoding sits in the skip layer's input."""
    Fq, W, depth, s = 4, 8, 3, 2
    D = 6 * Fq
    th = torch.zeros(F.param_count(Fq, W, depth, s), dtype=torch.float64)
    p_s = (W * D + W) + (W * W + W)                 # start of W_2 (after layers 0 and 1)
    th[p_s + 0 * (W + D) + W + (0 * 2 * Fq + 1 * 2 + 0)] = 1.0   # W_2[0, W + (axis x, band 1, sin)]
    p_out = p_s + W * (W + D) + W
    th[p_out + 0] = 1.0
    th[-1] = -0.2
    nx, ny, nz = 6, 2, 3
    a = F.field(th, nx, ny, nz, Fq, W, depth, 1.0, 27.0, 0.02, 1.0, skip=s)
    x = 2.0 * (np.arange(nx) + 0.5) / nx - 1.0
    w1 = 1.0 * 27.0 ** (1 / 3)
    expect = 0.02 + 0.98 / (1 + np.exp(-(np.maximum(np.sin(w1 * x), 0.0) - 0.2)))
    assert np.allclose(a.numpy(), np.broadcast_to(expect[None, None, :], (nz, ny, nx)), atol=1e-14)


def test_skip_field_gradient_finite_differences(F):
    """Autograd through the concatenation vs central differences."""
    Fq, W, depth, s = 3, 8, 4, 2
    th0 = torch.tensor(S.xavier_theta(Fq, W, depth, 12, skip=s), dtype=torch.float64)
    g_a = torch.tensor(S.rng(13).standard_normal((2, 3, 4)))
    th = th0.clone().requires_grad_(True)
    J = (F.field(th, 4, 3, 2, Fq, W, depth, 1.0, 8.0, 0.01, 2.0, skip=s) * g_a).sum()
    J.backward()
    p_s = (W * 6 * Fq + W) + (W * W + W)
    idx = list(S.rng(14).integers(0, th0.numel(), 8)) + [p_s + W + 5, p_s + 3 * (W + 6 * Fq) + W + 1]
    for i in idx:
        e = 1e-6
        tp = th0.clone(); tp[i] += e
        tm = th0.clone(); tm[i] -= e
        fd = ((F.field(tp, 4, 3, 2, Fq, W, depth, 1.0, 8.0, 0.01, 2.0, skip=s) * g_a).sum()
              - (F.field(tm, 4, 3, 2, Fq, W, depth, 1.0, 8.0, 0.01, 2.0, skip=s) * g_a).sum()) / (2 * e)
        assert float(th.grad[i]) == pytest.approx(float(fd), rel=1e-6, abs=1e-9)


def test_field_at_chosen_cells_is_the_full_field_there(F):
    """Evaluating at a list of flat cell indices c = (k ny + j) nx + i gives the
    centre 2 (i + 1/2) / n - 1 per axis (checked by hand on three cells) and
    the full field's values at those cells, bit for bit."""
    nx, ny, nz = 7, 5, 3
    cells = torch.tensor([0, nx * ny * nz - 1, (2 * ny + 3) * nx + 4])
    OF = F
    X = OF.cell_centres(nx, ny, nz, cells)
    want = torch.tensor([[1 / 7 - 1, 1 / 5 - 1, 1 / 3 - 1], [13 / 7 - 1, 9 / 5 - 1, 5 / 3 - 1],
                         [9 / 7 - 1, 7 / 5 - 1, 5 / 3 - 1]], dtype=torch.float64)
    assert torch.allclose(X, want, rtol=0, atol=1e-15)
    nf, W, depth = 3, 8, 2
    th = torch.tensor(S.rng(31).standard_normal(OF.param_count(nf, W, depth)) * 0.5)
    args = (nx, ny, nz, nf, W, depth, math.pi, 4 * math.pi, 0.01, 2.0)
    full = OF.field(th, *args).reshape(-1)
    some = torch.tensor(S.rng(32).choice(nx * ny * nz, 20, replace=False))
    for bf16 in (False, True):
        full = OF.field(th, *args, bf16=bf16).reshape(-1)
        assert torch.equal(OF.field(th, *args, bf16=bf16, cells=some), full[some])
