"""Shared helpers for the GPU parity tests (oracle on the CPU, library on the GPU)."""
import numpy as np

import oracle as O
from paper_1511_03703_gb300 import inputs


def gpu():
    import torch
    return torch.device("cuda:0")


def to_dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(gpu())


def to_np(t):
    return t.detach().cpu().numpy()


def oracle_members(N, M, xi_samples, sigma=0.1, kappa0=1.0, L=1.0):
    """Per-sample oracle assembly: lists of values[nnz], b[n] (one per sample)."""
    row_map, col = O.graph(N)
    vals, bs = [], []
    for xi in xi_samples:
        v, b = O.assemble(N, M, xi, row_map, col, L=L, sigma=sigma, kappa0=kappa0)
        vals.append(v)
        bs.append(b)
    return row_map, col, vals, bs


def spmv_bound(row_map, col, vals, x, rel=1e-12):
    """rel * (|A| |x|)_i, the componentwise SpMV tolerance."""
    return rel * O.spmv(row_map, col, np.abs(vals), np.abs(x))


def samples(seed, first, s, M):
    return inputs.kl_samples(seed, first, s, M)


def leading_mode_threshold(N, L=1.0, kappa0=1.0):
    """sigma* at which a(x) = kappa0 - sigma kappa_1(x) (M = 1, xi_1 = -1)
    first reaches 0 at a Gauss point of the N^3 mesh, from the closed form
    of the leading KL mode: kappa_1 = sqrt(lambda) phi(x) phi(y) phi(z) with
    phi(t) = cos(w (t - 1/2)) / sqrt(1/2 + sin(w) / (2 w)), w the root of
    c - w tan(w/2) = 0 in (0, pi), c = 1/L, lambda = (2c / (w^2 + c^2))^3.
    phi > 0 on [0, 1], so the minimum of a sits where phi^3 is largest."""
    from scipy.optimize import brentq
    c = 1.0 / L
    w = brentq(lambda t: c - t * np.tan(t / 2), 1e-12, np.pi - 1e-12)
    lam1 = 2 * c / (w * w + c * c)
    d = 0.5 / np.sqrt(3.0)
    g = np.concatenate([(np.arange(N) + 0.5 - d) / N, (np.arange(N) + 0.5 + d) / N])
    phi = np.cos(w * (g - 0.5)) / np.sqrt(0.5 + np.sin(w) / (2 * w))
    return kappa0 / (lam1 ** 1.5 * phi.max() ** 3)
