"""Pre-split double-float values (ens_convert_values ENS_F64_DF + ens_cg_df).

Bars: the split pairs are exactly the truncation of each value to 47
significant bits (hi + lo), with out-of-range and non-finite values marked
(NaN, 0); ens_cg_df reproduces ens_cg with ENS_CG_DF64 bitwise (solution,
iteration counts, residuals), also when some values take the FP64 path.
"""
import numpy as np
import pytest

import paper_1511_03703_gb300 as E
from paper_1511_03703_gb300 import inputs
from helpers import gpu, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as T
    assert T.cuda.is_available()
    E.lib()
    return T


def split_pairs(torch, graph, s, vals):
    out = torch.empty(vals.numel() * 2, dtype=torch.float32, device=gpu())
    E.convert_values(graph, s, vals, out, dtype=E.F64_DF)
    return out


@pytest.mark.parametrize("s", [1, 4, 32])
def test_split_pairs_are_the_47_bit_truncation(torch, s):
    mesh = E.Mesh(5, 10)
    v = inputs.random_vector(71, mesh.nnz * s, -1.0, 1.0) * 10.0 ** inputs.random_vector(72, mesh.nnz * s, -30, 30)
    v[::97] = 0.0
    v[1::101] = 1e-120           # below 2^-103
    v[2::103] = -3e200           # above 2^128
    v[3::107] = np.nan
    v[4::109] = 2.0 ** -103      # smallest in range
    v[5::113] = -(2.0 ** 128) * (1 - 2.0 ** -52)  # largest in range
    hl = to_np(split_pairs(torch, mesh.graph, s, to_dev(v))).reshape(-1, 2).astype(np.float64)
    a = np.abs(v)
    ok = (v == 0) | ((a >= 2.0 ** -103) & (a < 2.0 ** 128))
    trunc = (v.view(np.uint64) & ~np.uint64(0x3F)).view(np.float64)
    assert np.array_equal(hl[ok, 0] + hl[ok, 1], trunc[ok])
    hi_exp = (v.view(np.uint64) & ~np.uint64((1 << 29) - 1)).view(np.float64)
    assert np.array_equal(hl[ok, 0], hi_exp[ok])
    assert np.all(np.isnan(hl[~ok, 0])) and np.all(hl[~ok, 1] == 0.0)


def ensemble(torch, N, s, seed, M=10):
    mesh = E.Mesh(N, M)
    xs = inputs.kl_samples(seed, 0, s, M)
    vals, b = mesh.assemble(s, to_dev(inputs.ensemble_layout(xs)))
    return mesh, vals, b


def run(torch, mesh, s, vals, b, flags, values_df=None, tol=1e-10, max_iter=5000, x0=None):
    x = torch.zeros(mesh.n * s, dtype=torch.float64, device=gpu()) if x0 is None else x0.clone()
    work = torch.empty(E.cg_workspace_size(mesh.n, s), dtype=torch.uint8, device=gpu())
    it, rr, st, stats = E.cg(mesh.graph, s, vals, b, x, tol, max_iter, work, flags=flags, check_every=4,
                             values_df=values_df)
    return to_np(x), it, rr, st, stats


@pytest.mark.parametrize("s", [1, 4, 8, 16, 32])
@pytest.mark.parametrize("flags", [0, E.CG_GRAPH, E.CG_COUPLED])
def test_cg_df_bitwise_equals_df64(torch, s, flags):
    mesh, vals, b = ensemble(torch, 13, s, 800 + s)
    vdf = split_pairs(torch, mesh.graph, s, vals)
    x1, it1, rr1, st1, _ = run(torch, mesh, s, vals, b, flags | E.CG_DF64)
    x2, it2, rr2, st2, _ = run(torch, mesh, s, vals, b, flags, values_df=vdf)
    assert st1 == st2 == [0] * s
    assert it1 == it2 and rr1 == rr2 and np.array_equal(x1, x2)


@pytest.mark.parametrize("s", [1, 8, 32])
def test_cg_df_marked_values_take_the_fp64_path(torch, s):
    """Values below the split range (marked (NaN, 0) in the pre-split copy)
    make their rows recompute from the FP64 values: still bitwise ens_cg
    with ENS_CG_DF64, here over a fixed number of iterations."""
    mesh, vals, b = ensemble(torch, 7, s, 820 + s)
    v = to_np(vals).copy()
    v.reshape(-1, s)[5::37, :] *= 1e-110
    vals2 = to_dev(v)
    vdf = split_pairs(torch, mesh.graph, s, vals2)
    marked = v.reshape(-1, s)[5::37, :] != 0.0   # stored zeros stay (0, 0)
    assert marked.any() and np.isnan(to_np(vdf).reshape(-1, s, 2)[5::37, :, 0][marked]).all()
    x1, it1, rr1, st1, _ = run(torch, mesh, s, vals2, b, E.CG_DF64, tol=0.0, max_iter=12)
    x2, it2, rr2, st2, _ = run(torch, mesh, s, vals2, b, 0, values_df=vdf, tol=0.0, max_iter=12)
    assert it1 == it2 and st1 == st2 and rr1 == rr2 and np.array_equal(x1, x2)


def test_cg_df_with_guess_fallback(torch):
    s = 8
    mesh, vals, b = ensemble(torch, 9, s, 840)
    vdf = split_pairs(torch, mesh.graph, s, vals)
    x0 = to_dev(1e3 * inputs.random_vector(841, mesh.n * s))
    x1, it1, rr1, st1, s1 = run(torch, mesh, s, vals, b, E.CG_DF64)
    x2, it2, rr2, st2, s2 = run(torch, mesh, s, vals, b, E.CG_GUESS_FALLBACK, values_df=vdf, x0=x0)
    assert s2.guess_fallbacks == s and it1 == it2 and np.array_equal(x1, x2)


def test_cg_df_argument_errors(torch):
    mesh, vals, b = ensemble(torch, 4, 4, 850)
    work = torch.empty(E.cg_workspace_size(mesh.n, 4), dtype=torch.uint8, device=gpu())
    x = torch.zeros(mesh.n * 4, dtype=torch.float64, device=gpu())
    vdf = split_pairs(torch, mesh.graph, 4, vals)
    with pytest.raises(E.EnsError) as ei:
        E.cg(mesh.graph, 4, vals, b, x, 1e-8, 100, work, values_df=vdf[1:])  # misaligned
    assert ei.value.code == 3
    with pytest.raises(E.EnsError) as ei:
        E.convert_values(mesh.graph, 4, vals, vdf, diag_lo=x.float(), dtype=E.F64_DF)
    assert ei.value.code == 1


# ------------------------------------------------- double-float assembly
def diag_of(row_map, col, vals):
    n = len(row_map) - 1
    rows = np.repeat(np.arange(n), np.diff(row_map))
    d = np.zeros(n)
    sel = col == rows
    d[rows[sel]] = vals[sel]
    return d[rows]


@pytest.mark.parametrize("N,s", [(5, 1), (5, 4), (8, 8), (5, 32), (13, 16)])
def test_assemble_df_matches_oracle_and_writes_the_split(torch, N, s):
    import oracle as O
    from helpers import oracle_members
    M = 10
    mesh = E.Mesh(N, M)
    xs = inputs.kl_samples(900 + N, 0, s, M)
    xi = to_dev(inputs.ensemble_layout(xs))
    vdf = torch.empty(2 * mesh.nnz * s, dtype=torch.float32, device=gpu())
    vals, b = mesh.assemble(s, xi, values_df=vdf)
    V = to_np(vals).reshape(-1, s)
    rm, col, ov, ob = oracle_members(N, M, xs)
    for e in range(s):
        assert np.all(np.abs(V[:, e] - ov[e]) <= 1e-13 * np.abs(diag_of(rm, col, ov[e]))), e
    # the split is exactly what the conversion of these values writes
    assert torch.equal(vdf, split_pairs(torch, mesh.graph, s, vals))
    # FP64 assembly: the two agree to the double-float error of the KL terms
    # (mode values truncated to 47 bits, the terms summed as float pairs; the
    # kappa0 term is an FP64 FMA)
    v64, b64 = mesh.assemble(s, xi)
    assert torch.equal(b64, b)
    d = np.abs(to_np(v64).reshape(-1, s) - V)
    worst = max(float(np.max(d[:, e] / np.abs(diag_of(rm, col, ov[e])))) for e in range(s))
    print(f"df assembly vs FP64: max |dA| / A_II = {worst:.2e}")
    assert worst <= 1e-14


def test_assemble_df_s_invariant_and_fp64_fallback(torch):
    N, M = 6, 10
    mesh = E.Mesh(N, M)
    xs = inputs.kl_samples(950, 0, 32, M)
    ref = None
    for s in (1, 4, 8, 16, 32):
        vals, _ = mesh.assemble(s, to_dev(inputs.ensemble_layout(xs[:s])), df=True)
        v0 = to_np(vals).reshape(-1, s)[:, 0].copy()
        ref = v0 if ref is None else ref
        assert np.array_equal(v0, ref), s
    # coefficients outside the split range: the FP64 combination, bitwise
    xi = to_dev(inputs.ensemble_layout(xs[:4]))
    vd, _ = mesh.assemble(4, xi, sigma=1e200, df=True, check=False)
    v64, _ = mesh.assemble(4, xi, sigma=1e200, check=False)
    assert torch.equal(vd, v64)


def test_cg_df_on_df_assembly_matches_oracle(torch):
    import oracle as O
    from helpers import oracle_members
    N, M, s = 10, 10, 8
    mesh = E.Mesh(N, M)
    xs = inputs.kl_samples(960, 0, s, M)
    vdf = torch.empty(2 * mesh.nnz * s, dtype=torch.float32, device=gpu())
    vals, b = mesh.assemble(s, to_dev(inputs.ensemble_layout(xs)), values_df=vdf)
    x, it, rr, st, _ = run(torch, mesh, s, vals, b, E.CG_GRAPH, values_df=vdf, tol=1e-10)
    assert st == [0] * s and max(rr) <= 1.01e-10
    X = x.reshape(-1, s)
    rm, col, ov, ob = oracle_members(N, M, xs)
    for e in range(s):
        xo = O.cg(rm, col, ov[e], ob[e], tol=1e-13)[0]
        assert np.linalg.norm(X[:, e] - xo) <= 1e-8 * np.linalg.norm(xo), e


@pytest.mark.parametrize("presplit", [False, True])
def test_x0_zero_flag_is_bitwise_the_plain_start(torch, presplit):
    s = 8
    mesh, vals, b = ensemble(torch, 9, s, 970)
    vdf = split_pairs(torch, mesh.graph, s, vals) if presplit else None
    fl = 0 if presplit else E.CG_SPLIT64
    x1, it1, rr1, st1, s1 = run(torch, mesh, s, vals, b, fl, values_df=vdf)
    x2, it2, rr2, st2, s2 = run(torch, mesh, s, vals, b, fl | E.CG_X0_ZERO, values_df=vdf)
    assert it1 == it2 and rr1 == rr2 and np.array_equal(x1, x2)
