"""GPU parity at the benchmark's full size (64^3 cells, M = 10, s = 32) on the
exact path bench.py times, and the double-float assembly where its grid-stride
loop wraps.

The paper's commuted ensemble system is member-equivalent (Sect. 3: the s
samples of an ensemble are s independent systems that share a graph), so every
member of the ensemble solve must match its own per-sample oracle solve.

Bars (the same as the small-mesh tests):
  assembled values: |d| <= 1e-13 * A_II;  right-hand side: 1e-13 * max |b|
  SpMV, every arithmetic form: |d y_i| <= 1e-12 * (|A| |x|)_i componentwise
  CG: iteration counts within one; ||x - x_oracle|| / ||x_oracle|| <= 1e-8 at
      equal counts, else both sides re-run for max(counts) iterations and
      compared at 1e-10 (rounding decided the last stopping test).
Oracle inputs and expected values come from the oracle alone; the GPU's
values are never fed to it.
"""
import numpy as np
import pytest

import oracle as O
import paper_1511_03703_gb300 as E
from paper_1511_03703_gb300 import inputs
from helpers import gpu, oracle_members, spmv_bound, to_dev, to_np

pytestmark = pytest.mark.gpu

N64, M_KL, S32 = 64, 10, 32
PICKS = [0, 1, 17, 31]   # first and last member and two inside


@pytest.fixture(scope="module")
def torch():
    import torch as T
    assert T.cuda.is_available(), "GPU tests need a CUDA device"
    E.lib()
    return T


@pytest.fixture(scope="module")
def full(torch):
    """The benchmark's first ensemble: mesh set-up, the KL variables of samples
    0..31 of the 64^3 workload, the oracle's assembly of the picked members."""
    mesh = E.Mesh(N64, M_KL)
    xs = inputs.kl_samples(inputs.SEED_SCALE, 0, S32, M_KL)
    rm, col, ov, ob = oracle_members(N64, M_KL, xs[PICKS])
    return mesh, xs, rm, col, ov, ob


def diag_of(row_map, col, vals):
    n = len(row_map) - 1
    rows = np.repeat(np.arange(n), np.diff(row_map))
    d = np.zeros(n)
    sel = col == rows
    d[rows[sel]] = vals[sel]
    return d[rows]


def bench_solve(torch, mesh, s, vals, vdf, b, tol, max_iter):
    """The benchmark's solve call: ens_cg_df on the pre-split copy, x0 = 0
    stated, CUDA-graph replay of 8 iterations between host checks."""
    x = torch.zeros(mesh.n * s, dtype=torch.float64, device=gpu())
    work = torch.empty(E.cg_workspace_size(mesh.n, s), dtype=torch.uint8, device=gpu())
    it, rr, st, _ = E.cg(mesh.graph, s, vals, b, x, tol, max_iter, work,
                         flags=E.CG_X0_ZERO | E.CG_GRAPH, check_every=8, values_df=vdf)
    return to_np(x).reshape(-1, s), it, rr, st


def test_bench_path_64cubed_s32(torch, full):
    """ens_assemble_df with its pre-split copy, then ens_cg_df with
    ENS_CG_X0_ZERO | ENS_CG_GRAPH and check_every = 8 to 1e-8: values, right-
    hand sides and solutions of members 0, 1, 17 and 31 against per-sample
    oracle assemblies and CG solves."""
    mesh, xs, rm, col, ov, ob = full
    s = S32
    xi = to_dev(inputs.ensemble_layout(xs))
    vdf = torch.empty(2 * mesh.nnz * s, dtype=torch.float32, device=gpu())
    vals, b = mesh.assemble(s, xi, values_df=vdf)
    # the split copy is exactly what converting these values writes
    chk = torch.empty_like(vdf)
    E.convert_values(mesh.graph, s, vals, chk, dtype=E.F64_DF)
    assert torch.equal(chk, vdf)
    del chk
    V, B = to_np(vals).reshape(-1, s), to_np(b).reshape(-1, s)
    for i, e in enumerate(PICKS):
        assert np.all(np.abs(V[:, e] - ov[i]) <= 1e-13 * np.abs(diag_of(rm, col, ov[i]))), e
        assert np.max(np.abs(B[:, e] - ob[i])) <= 1e-13 * np.max(np.abs(ob[i])), e
    X, it, rr, st = bench_solve(torch, mesh, s, vals, vdf, b, 1e-8, 10000)
    assert st == [0] * s and max(rr) <= 1.01e-8
    rerun = {}
    for i, e in enumerate(PICKS):
        xo, ito, rro, sto = O.cg(rm, col, ov[i], ob[i], tol=1e-8)
        assert sto == 0 and abs(it[e] - ito) <= 1, (e, it[e], ito)
        if it[e] == ito:
            err = np.linalg.norm(X[:, e] - xo) / np.linalg.norm(xo)
            assert err <= 1e-8, (e, err)
        else:
            rerun[i] = max(it[e], ito)
    # members whose stopping test rounding decided: both sides for the same count
    for i, k in rerun.items():
        e = PICKS[i]
        X2, it2, _, _ = bench_solve(torch, mesh, s, vals, vdf, b, 0.0, k)
        xo2, _, _, _ = O.cg(rm, col, ov[i], ob[i], tol=0.0, max_iter=k)
        assert it2[e] == k
        assert np.linalg.norm(X2[:, e] - xo2) <= 1e-10 * np.linalg.norm(xo2), e


@pytest.mark.parametrize("form", ["f64", "df", "split", "dfv"])
def test_spmv_every_form_64cubed_s32(torch, full, form):
    """Every SpMV arithmetic form at 64^3, s = 32, all 32 members element by
    element: the oracle's values of the four picked samples tiled over the
    members, one random vector per member."""
    mesh, xs, rm, col, ov, ob = full
    s, n = S32, mesh.n
    vt = to_dev(O.to_ensemble([ov[e % len(ov)] for e in range(s)]))
    xm = [inputs.random_vector(1600 + e, n) for e in range(s)]
    x = to_dev(O.to_ensemble(xm))
    y = torch.empty(n * s, dtype=torch.float64, device=gpu())
    if form == "dfv":
        vdf = torch.empty(2 * vt.numel(), dtype=torch.float32, device=gpu())
        E.convert_values(mesh.graph, s, vt, vdf, dtype=E.F64_DF)
        E.spmv(mesh.graph, s, vt, x, y, values_df=vdf)
    else:
        E.spmv(mesh.graph, s, vt, x, y, df=form == "df", split=form == "split")
    Y = to_np(y).reshape(-1, s)
    for e in range(s):
        v = ov[e % len(ov)]
        ref = O.spmv(rm, col, v, xm[e])
        assert np.all(np.abs(Y[:, e] - ref) <= spmv_bound(rm, col, v, xm[e])), e


@pytest.mark.parametrize("s", [1, 4, 8, 16, 32])
def test_assemble_df_grid_stride_wraps(torch, s):
    """32^3 cells (912,673 entries): the double-float assembly runs one wave
    of resident CTAs (about 150 K threads), so each thread takes its
    grid-stride loop several times (about 6 at s = 1, 24 at s = 32).  Every
    member against the oracle; the split copy is the conversion of the
    values."""
    N = 32
    mesh = E.Mesh(N, M_KL)
    xs = inputs.kl_samples(1700 + s, 0, s, M_KL)
    vdf = torch.empty(2 * mesh.nnz * s, dtype=torch.float32, device=gpu())
    vals, b = mesh.assemble(s, to_dev(inputs.ensemble_layout(xs)), values_df=vdf)
    chk = torch.empty_like(vdf)
    E.convert_values(mesh.graph, s, vals, chk, dtype=E.F64_DF)
    assert torch.equal(chk, vdf)
    V, B = to_np(vals).reshape(-1, s), to_np(b).reshape(-1, s)
    rm, col, ov, ob = oracle_members(N, M_KL, xs)
    for e in range(s):
        assert np.all(np.abs(V[:, e] - ov[e]) <= 1e-13 * np.abs(diag_of(rm, col, ov[e]))), e
        assert np.max(np.abs(B[:, e] - ob[e])) <= 1e-13 * np.max(np.abs(ob[e])), e
