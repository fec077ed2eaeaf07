"""Mixed precision (FP32 / BF16 values, FP64 iterative refinement) against the
FP64 oracle.

Bars: the low-precision copy is exactly the round-to-nearest of the FP64
values (BF16 through FP32); with the compensated diagonal every low-precision
row sums to fl32 of the FP64 row sum; refined solutions reach the FP64
residual tolerance and agree with an oracle solve at 1e-12 to 1e-8 relative.
"""
import numpy as np
import pytest

import oracle as O
import paper_1511_03703_gb300 as E
from paper_1511_03703_gb300 import inputs
from helpers import gpu, oracle_members, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as T
    assert T.cuda.is_available()
    E.lib()
    return T


def setup(torch, N, s, seed, M=10):
    mesh = E.Mesh(N, M)
    xs = inputs.kl_samples(seed, 0, s, M)
    vals, b = mesh.assemble(s, to_dev(inputs.ensemble_layout(xs)))
    return mesh, xs, vals, b


@pytest.mark.parametrize("s", [1, 4, 32])
def test_convert_values_rounding_and_compensated_diagonal(torch, s):
    mesh, xs, vals, b = setup(torch, 6, s, 71)
    v64 = to_np(vals).reshape(-1, s)
    v32 = torch.empty_like(vals, dtype=torch.float32)
    E.convert_values(mesh.graph, s, vals, v32)
    assert np.array_equal(to_np(v32).reshape(-1, s), v64.astype(np.float32))
    vb = torch.empty_like(vals, dtype=torch.bfloat16)
    diag = torch.empty(mesh.n * s, dtype=torch.float32, device=gpu())
    E.convert_values(mesh.graph, s, vals, vb, diag)
    ref_b = torch.from_numpy(v64.astype(np.float32)).bfloat16()
    rm, col = to_np(mesh.row_map), to_np(mesh.col_entry)
    rows = np.repeat(np.arange(mesh.n), np.diff(rm))
    isdiag = col == rows
    got_b = vb.reshape(-1, s).float().cpu().numpy()
    exp_b = ref_b.float().numpy()
    exp_b[isdiag, :] = 0.0
    assert np.array_equal(got_b, exp_b)
    D = to_np(diag).reshape(-1, s)
    for e in range(s):
        rowsum = np.bincount(rows, weights=v64[:, e], minlength=mesh.n)
        offsum = np.bincount(rows, weights=exp_b[:, e].astype(np.float64), minlength=mesh.n)
        assert np.array_equal(D[:, e], (rowsum - offsum).astype(np.float32))


def mixed_solve(torch, mesh, vals, b, s, dtype, comp, tol, **kw):
    lo = torch.empty_like(vals, dtype=dtype)
    diag = torch.empty(mesh.n * s, dtype=torch.float32, device=gpu()) if comp else None
    E.convert_values(mesh.graph, s, vals, lo, diag)
    x = torch.zeros(mesh.n * s, dtype=torch.float64, device=gpu())
    work = torch.empty(E.cg_mixed_workspace_size(mesh.n, s), dtype=torch.uint8, device=gpu())
    oi, ii, rr, st, stats = E.cg_mixed(mesh.graph, s, vals, lo, b, x, tol, work, diag_lo=diag, **kw)
    return to_np(x).reshape(-1, s), oi, ii, rr, st


@pytest.mark.parametrize("dtype,comp", [("float32", False), ("float32", True), ("bfloat16", True)])
@pytest.mark.parametrize("N,s", [(8, 4), (13, 8), (16, 32)])
def test_mixed_refinement_matches_fp64_oracle(torch, dtype, comp, N, s):
    mesh, xs, vals, b = setup(torch, N, s, 300 + N)
    inner = 1e-2 if dtype == "bfloat16" else 1e-4
    X, oi, ii, rr, st = mixed_solve(torch, mesh, vals, b, s, getattr(torch, dtype), comp, 1e-10,
                                    inner_tol=inner)
    assert st == [0] * s and max(rr) <= 1e-10
    assert max(oi) <= (12 if dtype == "bfloat16" else 6)
    rm, col, ov, ob = oracle_members(N, 10, xs)
    for e in range(s):
        xo, _, _, sto = O.cg(rm, col, ov[e], ob[e], tol=1e-12)
        assert sto == 0
        assert np.linalg.norm(X[:, e] - xo) <= 1e-8 * np.linalg.norm(xo), e


def test_mixed_edge_cases_and_s_invariance(torch):
    mesh, xs, vals, b = setup(torch, 7, 4, 91)
    b.view(-1, 4)[:, 2] = 0.0
    X, oi, ii, rr, st = mixed_solve(torch, mesh, vals, b, 4, torch.float32, False, 1e-10)
    assert st == [0, 0, 0, 0] and np.all(X[:, 2] == 0.0) and oi[2] == 0
    # refinement cap: one step cannot reach 1e-14
    X, oi, ii, rr, st = mixed_solve(torch, mesh, vals, b, 4, torch.float32, False, 1e-14, max_outer=1)
    assert st[0] == 5 and oi[0] == 1
    # member result independent of the ensemble size (bitwise)
    xs32 = inputs.kl_samples(92, 0, 32, 10)
    ref = None
    for s in (1, 4, 32):
        vals_s, b_s = mesh.assemble(s, to_dev(inputs.ensemble_layout(xs32[:s])))
        X, oi, ii, rr, st = mixed_solve(torch, mesh, vals_s, b_s, s, torch.bfloat16, True, 1e-9,
                                        inner_tol=1e-2)
        cur = (X[:, 0].copy(), oi[0], ii[0])
        ref = cur if ref is None else ref
        assert np.array_equal(cur[0], ref[0]) and cur[1:] == ref[1:], s
