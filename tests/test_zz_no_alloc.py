"""ens_dot_static: the dot entry point for callers that cannot allocate.

Callers that cannot call cudaMalloc when they need a dot product (an
allocator that is locked or owned by another runtime, for instance) use
ens_dot_static, which takes its scratch from a static device array inside the
library.  These tests call it through the C ABI and check it against ens_dot,
the entry point with a caller workspace, on two calls in a row with different
sizes, so that contents left in the shared array by one call cannot leak into
the next.  The file is collected last so that a stop at the first failure has
already run every other test; it passes alone in a fresh process as well.
"""
import ctypes
import math

import numpy as np
import pytest

import oracle as O
import paper_1511_03703_gb300 as E
from paper_1511_03703_gb300 import inputs

pytestmark = pytest.mark.gpu


def run_both(torch, n, s, seed):
    dev = torch.device("cuda:0")
    U = [inputs.random_vector(seed + e, n) for e in range(s)]
    V = [inputs.random_vector(seed + 100 + e, n, -2.0, 3.0) for e in range(s)]
    u = torch.from_numpy(O.to_ensemble(U)).to(dev)
    v = torch.from_numpy(O.to_ensemble(V)).to(dev)
    ref = torch.empty(s, dtype=torch.float64, device=dev)
    work = torch.empty(E.dot_workspace_size(n, s), dtype=torch.uint8, device=dev)
    E.dot(n, s, u, v, ref, work)
    out = torch.full((s,), float("nan"), dtype=torch.float64, device=dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = E.lib().ens_dot_static(n, s, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                                ctypes.c_void_p(out.data_ptr()), stream)
    assert rc == 0, E.lib().ens_last_error()
    got, want = out.cpu().numpy(), ref.cpu().numpy()
    for e in range(s):
        prod = U[e] * V[e]
        scale = np.sum(np.abs(prod))
        assert abs(got[e] - want[e]) <= 1e-13 * scale, e
        assert abs(got[e] - math.fsum(prod.tolist())) <= 1e-13 * scale, e
    return got


def test_static_dot_matches_workspace_dot_twice():
    import torch
    assert torch.cuda.is_available()
    run_both(torch, 40000, 8, 11)          # first call: larger tree, leaves partials behind
    run_both(torch, 1025, 32, 23)          # second call: different size and width


def test_static_dot_rejects_sizes_beyond_its_array():
    import torch
    dev = torch.device("cuda:0")
    n, s = 2146689, 32
    assert E.dot_workspace_size(n, s) > 4 * 1024 * 1024
    out = torch.empty(s, dtype=torch.float64, device=dev)
    u = torch.zeros(16, dtype=torch.float64, device=dev)   # never read: the size check comes first
    with pytest.raises(E.EnsError) as ei:
        E.dot_static(n, s, u, u, out)
    assert ei.value.code == 2 and "static" in str(ei.value)
