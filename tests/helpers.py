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
