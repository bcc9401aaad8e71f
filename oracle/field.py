"""FP64 CPU reference of the neural diffusivity field (Sec. 4.1; App. D.1).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain PyTorch CPU ops in
float64, written from the paper's definitions:

  * cell centres normalised to [-1, 1]: x_d = 2 (i + 1/2) / N_d - 1;
  * Fourier encoding (Eq. posenc): sin/cos of each coordinate at each band
    frequency; bands log-spaced between freq_lo and freq_hi (the paper's
    2^k pi is the special case freq_hi / freq_lo = 2^(F-1));
  * cosine frequency-annealing weights w_k(beta) (Eq. fa_schedule);
  * ReLU MLP; bounded output alpha = alpha_min + (alpha_max - alpha_min) sigmoid(f)
    (Eq. bracket).

``bf16=True`` evaluates the same network the way the tensor-core path does
(weights and hidden activations rounded to bfloat16, sums in float64), to
check that path's arithmetic tightly; ``bf16=False`` is the exact FP64 model.
Parameter packing: W_0 [W x 6F], b_0 [W], W_l [W x W], b_l [W] for
l = 1..depth-1, w_out [W], b_out [1]; weights row-major [out][in].
"""
from __future__ import annotations

import math

import torch


def band_frequencies(F, freq_lo, freq_hi):
    if F == 1:
        return torch.tensor([freq_lo], dtype=torch.float64)
    b = torch.arange(F, dtype=torch.float64)
    return freq_lo * (freq_hi / freq_lo) ** (b / (F - 1))


def annealing_weights(F, beta):
    """Eq. fa_schedule: w_k = (1 - cos(pi clamp(beta - k, 0, 1))) / 2."""
    k = torch.arange(F, dtype=torch.float64)
    return 0.5 * (1.0 - torch.cos(math.pi * torch.clamp(beta - k, 0.0, 1.0)))


def cell_centres(nx, ny, nz, cells=None):
    """[N, 3] normalised centres in the cell order c = (k ny + j) nx + i, or,
    with ``cells`` (flat cell indices c), the centres of those cells only."""
    if cells is not None:
        c = torch.as_tensor(cells, dtype=torch.int64)
        i, j, k = c % nx, (c // nx) % ny, c // (nx * ny)
        return torch.stack([2.0 * (t.to(torch.float64) + 0.5) / n - 1.0 for t, n in ((i, nx), (j, ny), (k, nz))],
                           dim=1)
    axes = [2.0 * (torch.arange(n, dtype=torch.float64) + 0.5) / n - 1.0 for n in (nx, ny, nz)]
    z, y, x = torch.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    return torch.stack([x.reshape(-1), y.reshape(-1), z.reshape(-1)], dim=1)


def encode(X, F, freq_lo, freq_hi, band_weights=None):
    """[N, 6F]: for axis d, band b -> columns d*2F + 2b (sin), d*2F + 2b + 1 (cos)."""
    w = band_frequencies(F, freq_lo, freq_hi)
    wt = torch.ones(F, dtype=torch.float64) if band_weights is None else torch.as_tensor(band_weights, dtype=torch.float64)
    cols = []
    for d in range(3):
        arg = X[:, d:d + 1] * w[None, :]
        pair = torch.stack([wt * torch.sin(arg), wt * torch.cos(arg)], dim=2)   # [N, F, 2]
        cols.append(pair.reshape(X.shape[0], 2 * F))
    return torch.cat(cols, dim=1)


def unpack(theta, F, W, depth, skip=0):
    """Split the packed parameters; layer `skip` (> 0) takes [h, gamma(x)] as input."""
    theta = torch.as_tensor(theta, dtype=torch.float64)
    D = 6 * F
    out, p = [], 0
    for l in range(depth):
        n_in = D if l == 0 else (W + D if l == skip else W)
        Wl = theta[p:p + W * n_in].reshape(W, n_in); p += W * n_in
        bl = theta[p:p + W]; p += W
        out.append((Wl, bl))
    w_out = theta[p:p + W]; p += W
    b_out = theta[p:p + 1]; p += 1
    assert p == theta.numel(), (p, theta.numel())
    return out, w_out, b_out


def param_count(F, W, depth, skip=0):
    return W * 6 * F + W + (depth - 1) * (W * W + W) + (W * 6 * F if skip else 0) + W + 1


def _bf16(t):
    return t.to(torch.bfloat16).to(torch.float64)


def field(theta, nx, ny, nz, F, W, depth, freq_lo, freq_hi, alpha_min, alpha_max, band_weights=None, bf16=False,
          skip=0, cells=None):
    """alpha at every cell centre, [nz, ny, nx] (differentiable in theta), or
    at the given flat cell indices only ([len(cells)]).
    skip > 0: the encoding is concatenated to the input of hidden layer `skip`
    (App. D.1, the re-injection at the middle layer)."""
    layers, w_out, b_out = unpack(theta, F, W, depth, skip)
    gamma = encode(cell_centres(nx, ny, nz, cells), F, freq_lo, freq_hi, band_weights)
    if bf16:
        gamma = _bf16(gamma)
    h = gamma
    for l, (Wl, bl) in enumerate(layers):
        Wl = _bf16(Wl) if bf16 else Wl
        x = torch.cat([h, gamma], dim=1) if (skip and l == skip) else h
        h = torch.relu(x @ Wl.T + bl)
        if bf16:
            h = _bf16(h)
    f = h @ w_out + b_out
    alpha = alpha_min + (alpha_max - alpha_min) * torch.sigmoid(f)
    return alpha if cells is not None else alpha.reshape(nz, ny, nx)
