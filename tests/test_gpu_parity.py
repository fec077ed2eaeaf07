"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

Tolerances (north star, and the arithmetic they follow from):
  graph, ElemGraph, boundary mask, iteration counts on small meshes: exact
  KL eigenvalues: 1e-14 relative; coefficient at Gauss points: 1e-14
  assembled values: |d| <= 1e-13 * A_II (row diagonal; off-diagonal entries
      of a constant-coefficient row cancel to ~0 so a relative test is void)
  SpMV: |d y_i| <= 1e-12 * (|A| |x|)_i componentwise
  dot: |d| <= 1e-13 * sum |u v| against exactly rounded summation (fsum)
  CG: ||x - x_oracle|| / ||x_oracle|| <= 1e-8; if the iteration counts differ
      by one (stopping test decided by rounding), both are re-run for the same
      fixed number of iterations and must agree to 1e-10.
"""
import math

import numpy as np
import pytest

import oracle as O
import paper_1511_03703_gb300 as E
from paper_1511_03703_gb300 import inputs
from helpers import gpu, leading_mode_threshold, oracle_members, spmv_bound, to_dev, to_np

pytestmark = pytest.mark.gpu
S_ALL = [1, 4, 8, 16, 32]


@pytest.fixture(scope="module")
def torch():
    import torch as T
    assert T.cuda.is_available(), "GPU tests need a CUDA device"
    E.lib()
    return T


def ens_cols(flat, s):
    return np.asarray(flat).reshape(-1, s)


# ---------------------------------------------------------------- A1 graph
@pytest.mark.parametrize("N", [1, 2, 3, 8, 13, 16])
def test_graph_bit_exact(torch, N):
    n, nnz, nc = E.mesh_sizes(N)
    rm = torch.empty(n + 1, dtype=torch.int32, device=gpu())
    col = torch.empty(nnz, dtype=torch.int32, device=gpu())
    eg = torch.empty(nc * 64, dtype=torch.int32, device=gpu())
    bm = torch.empty(n, dtype=torch.uint8, device=gpu())
    E.graph_build(N, rm, col, eg, bm)
    orm, ocol = O.graph(N)
    assert np.array_equal(to_np(rm), orm)
    assert np.array_equal(to_np(col), ocol)
    assert np.array_equal(to_np(eg), O.elem_graph(N, orm, ocol))
    assert np.array_equal(to_np(bm), O.bmask(N))


# ------------------------------------------------------------------- A2 KL
@pytest.mark.parametrize("N,M", [(8, 3), (8, 10), (5, 17), (64, 10)])
def test_kl_setup_matches_oracle(torch, N, M):
    tab = torch.empty(E.kl_table_size(N, M), dtype=torch.float64, device=gpu())
    lam, pqr = E.kl_setup(N, M, 1.0, tab)
    opqr, olam = O.kl_modes(M)
    assert pqr == opqr.tolist()
    assert np.max(np.abs(np.array(lam) - olam) / olam) < 1e-14
    T = to_np(tab)[: 3 * M * 2 * N].reshape(3, M, 2 * N)
    xi = inputs.kl_samples(5, 0, 1, M)[0]
    a_or = O.kl_coeff_qp(N, M, xi)
    t = np.arange(N)
    for q in range(8):
        tx, ty, tz = 2 * t + (q & 1), 2 * t + ((q >> 1) & 1), 2 * t + ((q >> 2) & 1)
        kap = (T[0][:, tx][:, None, None, :] * T[1][:, ty][:, None, :, None] *
               T[2][:, tz][:, :, None, None])          # [k, ck, cj, ci]
        a = 1.0 + 0.1 * np.tensordot(xi, kap, axes=(0, 0)).reshape(-1)
        assert np.max(np.abs(a - a_or[:, q])) < 1e-14


# ------------------------------------------------------------- A3 assembly
def diag_of(row_map, col, vals):
    n = len(row_map) - 1
    rows = np.repeat(np.arange(n), np.diff(row_map))
    d = np.zeros(n)
    sel = col == rows
    d[rows[sel]] = vals[sel]
    return d[rows]


@pytest.mark.parametrize("N,M,s", [(8, 3, 4), (5, 10, 1), (5, 10, 4), (5, 10, 8), (5, 10, 16),
                                   (5, 10, 32), (13, 10, 8)])
def test_assembly_matches_oracle(torch, N, M, s):
    mesh = E.Mesh(N, M)
    xs = inputs.kl_samples(100 + N, 0, s, M)
    values, b = mesh.assemble(s, to_dev(inputs.ensemble_layout(xs)))
    V, B = ens_cols(to_np(values), s), ens_cols(to_np(b), s)
    rm, col, ov, ob = oracle_members(N, M, xs)
    for e in range(s):
        tol = 1e-13 * np.abs(diag_of(rm, col, ov[e]))
        assert np.all(np.abs(V[:, e] - ov[e]) <= tol), e
        assert np.max(np.abs(B[:, e] - ob[e])) <= 1e-13 * np.max(np.abs(ob[e]))


# --------------------------------------- A3 coefficient positivity (status 7)
@pytest.mark.parametrize("df", [False, True])
def test_assemble_nonpositive_coefficient_status(torch, df):
    """Member 2's KL variables scaled by 40 (|xi| >> 1) make its coefficient
    negative somewhere: ens_assemble(_df) returns ENS_ERR_NONPOS_COEFF naming
    that member, as the oracle's assembly reports, and still writes every
    member's values (the good members against the oracle)."""
    N, M, s = 6, 10, 4
    mesh = E.Mesh(N, M)
    xs = inputs.kl_samples(1800, 0, s, M)
    xs[2] *= 40.0
    assert [O.coeff_min(N, M, x) <= 0 for x in xs] == [False, False, True, False]
    vals = torch.empty(mesh.nnz * s, dtype=torch.float64, device=gpu())
    b = torch.empty(mesh.n * s, dtype=torch.float64, device=gpu())
    vdf = torch.empty(2 * mesh.nnz * s, dtype=torch.float32, device=gpu()) if df else None
    with pytest.raises(E.EnsError) as ei:
        mesh.assemble(s, to_dev(inputs.ensemble_layout(xs)), values=vals, b=b, df=df, values_df=vdf)
    assert ei.value.code == 7 and "member 2" in str(ei.value)
    rm, col = O.graph(N)
    V = ens_cols(to_np(vals), s)
    for e in (0, 1, 3):
        ov, ob = O.assemble(N, M, xs[e], rm, col)
        assert np.all(np.abs(V[:, e] - ov) <= 1e-13 * np.abs(diag_of(rm, col, ov))), e
    with pytest.raises(O.NonPositiveCoefficient):
        O.assemble(N, M, xs[2], rm, col)
    # the unscaled draws pass the check (the bound alone clears them)
    mesh.assemble(s, to_dev(inputs.ensemble_layout(inputs.kl_samples(1800, 0, s, M))), df=df)


@pytest.mark.parametrize("s", [1, 8])
def test_assemble_coefficient_check_exact_minimum(torch, s):
    """M = 1: with xi_1 = +1 a large sigma defeats the bound but the exact
    minimum over the Gauss points stays positive (no error); with xi_1 = -1
    the status flips exactly at the closed-form threshold sigma*, on the
    same side as the oracle."""
    N = 7
    mesh = E.Mesh(N, 1)
    sstar = leading_mode_threshold(N)
    ones = np.ones((s, 1))
    mesh.assemble(s, to_dev(inputs.ensemble_layout(ones)), sigma=50 * sstar)      # exact path, positive
    neg = to_dev(inputs.ensemble_layout(-ones))
    mesh.assemble(s, neg, sigma=sstar * (1 - 1e-7))
    with pytest.raises(E.EnsError) as ei:
        mesh.assemble(s, neg, sigma=sstar * (1 + 1e-7), df=True)
    assert ei.value.code == 7
    assert O.coeff_min(N, 1, [-1.0], sigma=sstar * (1 - 1e-7)) > 0 > O.coeff_min(N, 1, [-1.0],
                                                                                sigma=sstar * (1 + 1e-7))
    with pytest.raises(E.EnsError) as ei:
        mesh.assemble(s, neg, sigma=float("nan"))
    assert ei.value.code == 7


def test_assemble_coefficient_check_concurrent_threads(torch):
    """Eight host threads check coefficients at once, each on its own stream
    (the bounds come back through pinned slots shared per device), while a
    large device-to-host copy is in flight on another stream: every thread gets
    its own members' verdict, and the good ensembles' values equal a serial
    assembly bitwise."""
    import threading
    N, M, s = 8, 10, 8
    mesh = E.Mesh(N, M)
    cases = []
    for t in range(8):
        xs = inputs.kl_samples(2400 + t, 0, s, M)
        if t % 3 == 1:
            xs[t % s] *= 40.0   # member t % s has a negative coefficient
        cases.append(xs)
    ref = []
    for xs in cases:
        bad = [O.coeff_min(N, M, x) <= 0 for x in xs]
        v = torch.empty(mesh.nnz * s, dtype=torch.float64, device=gpu())
        b = torch.empty(mesh.n * s, dtype=torch.float64, device=gpu())
        mesh.assemble(s, to_dev(inputs.ensemble_layout(xs)), values=v, b=b, check=False)
        ref.append((bad.index(True) if any(bad) else -1, to_np(v)))
    big = torch.ones(64 << 20, dtype=torch.float64, device=gpu())
    host = torch.empty(big.shape, dtype=torch.float64).pin_memory()
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        host.copy_(big, non_blocking=True)   # 512 MB in flight while the checks run
    out = [None] * len(cases)

    def work(t):
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            v = torch.empty(mesh.nnz * s, dtype=torch.float64, device=gpu())
            b = torch.empty(mesh.n * s, dtype=torch.float64, device=gpu())
            xi = to_dev(inputs.ensemble_layout(cases[t]))
            st.synchronize()
            try:
                mesh.assemble(s, xi, values=v, b=b, stream=st)
                out[t] = (-1, to_np(v))
            except E.EnsError as err:
                out[t] = (int(str(err).split("member ")[1].split(":")[0]) if err.code == 7 else -99, None)

    threads = [threading.Thread(target=work, args=(t,)) for t in range(len(cases))]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    side.synchronize()
    for t, (got, want) in enumerate(zip(out, ref)):
        assert got is not None and got[0] == want[0], t
        if want[0] < 0:
            assert np.array_equal(got[1], want[1]), t


# ------------------------------------------------------------------ A4 SpMV
@pytest.mark.parametrize("N", [3, 8, 13])
@pytest.mark.parametrize("s", S_ALL)
@pytest.mark.parametrize("dtype", ["float64", "float64_df", "float64_split", "float64_dfv", "float32",
                                   "bfloat16"])
def test_spmv_matches_oracle(torch, N, s, dtype):
    M = 10
    xs = inputs.kl_samples(200 + N, 0, min(s, 4), M)
    rm, col, ov, _ = oracle_members(N, M, xs)
    ov = [ov[e % len(ov)] for e in range(s)]
    n = len(rm) - 1
    xm = [inputs.random_vector(300 + e, n) for e in range(s)]
    df, split, dfv = dtype == "float64_df", dtype == "float64_split", dtype == "float64_dfv"
    vt = torch.from_numpy(O.to_ensemble(ov)).to(getattr(torch, "float64" if df or split or dfv else dtype))
    vq = [vt.reshape(-1, s)[:, e].double().numpy() for e in range(s)]   # values as stored
    y = torch.empty(n * s, dtype=torch.float64, device=gpu())
    graph = E.Graph(to_dev(rm), to_dev(col))
    vdf = None
    if dfv:
        vdf = torch.empty(2 * vt.numel(), dtype=torch.float32, device=gpu())
        E.convert_values(graph, s, vt.to(gpu()), vdf, dtype=E.F64_DF)
    E.spmv(graph, s, vt.to(gpu()), to_dev(O.to_ensemble(xm)), y, df=df, split=split, values_df=vdf)
    Y = ens_cols(to_np(y), s)
    for e in range(s):
        ref = O.spmv(rm, col, vq[e], xm[e])
        assert np.all(np.abs(Y[:, e] - ref) <= spmv_bound(rm, col, vq[e], xm[e])), e


@pytest.mark.parametrize("s", [1, 8, 32])
@pytest.mark.parametrize("form", ["df", "split", "dfv"])
def test_spmv_df_extreme_values_take_exact_path(torch, s, form):
    """Values outside the double-float split range ([2^-103, 2^128)), exact
    zeros and mixed magnitudes within a row stay inside the 1e-12 bound."""
    N, M = 5, 10
    xs = inputs.kl_samples(250, 0, 1, M)
    rm, col, ov, _ = oracle_members(N, M, xs)
    n = len(rm) - 1
    scale = np.ones(len(col))
    scale[::7] = 1e-120      # below the split range: FP64 fallback
    scale[3::11] = 1e60      # above it
    scale[5::13] = 0.0       # exact zeros
    vals = [ov[0] * scale * (1.0 + 0.01 * e) for e in range(s)]
    xm = [inputs.random_vector(330 + e, n, -1e3, 1e3) for e in range(s)]
    y = torch.empty(n * s, dtype=torch.float64, device=gpu())
    graph = E.Graph(to_dev(rm), to_dev(col))
    spmv_form(torch, graph, s, to_dev(O.to_ensemble(vals)), to_dev(O.to_ensemble(xm)), y, form)
    Y = ens_cols(to_np(y), s)
    for e in range(s):
        ref = O.spmv(rm, col, vals[e], xm[e])
        assert np.all(np.abs(Y[:, e] - ref) <= spmv_bound(rm, col, vals[e], xm[e])), e


def spmv_form(torch, graph, s, vals, x, y, form):
    """ens_spmv in the double-float form `form` (df, split) or ens_spmv_df
    on the ENS_F64_DF copy of vals (dfv)."""
    vdf = None
    if form == "dfv":
        vdf = torch.empty(2 * vals.numel(), dtype=torch.float32, device=gpu())
        E.convert_values(graph, s, vals, vdf, dtype=E.F64_DF)
    E.spmv(graph, s, vals, x, y, df=form == "df", split=form == "split", values_df=vdf)


def test_spmv_s_invariant_bitwise(torch):
    N, M = 9, 10
    mesh = E.Mesh(N, M)
    xs = inputs.kl_samples(41, 0, 32, M)
    xm = [inputs.random_vector(500 + e, mesh.n) for e in range(32)]
    ref = None
    for s in S_ALL:
        vals, _ = mesh.assemble(s, to_dev(inputs.ensemble_layout(xs[:s])))
        y = torch.empty(mesh.n * s, dtype=torch.float64, device=gpu())
        E.spmv(mesh.graph, s, vals, to_dev(O.to_ensemble(xm[:s])), y)
        Y = ens_cols(to_np(y), s)
        E.spmv(mesh.graph, s, vals, to_dev(O.to_ensemble(xm[:s])), y, df=True)
        Ydf = ens_cols(to_np(y), s)
        E.spmv(mesh.graph, s, vals, to_dev(O.to_ensemble(xm[:s])), y, split=True)
        Ysp = ens_cols(to_np(y), s)
        if ref is None:
            ref = (Y[:, 0].copy(), Ydf[:, 0].copy(), Ysp[:, 0].copy())
        assert np.array_equal(Y[:, 0], ref[0]) and np.array_equal(Ydf[:, 0], ref[1]), s
        assert np.array_equal(Ysp[:, 0], ref[2]), s


# ------------------------------------------------------------------- A5 dot
@pytest.mark.parametrize("n", [1, 31, 32, 33, 1025, 40000])
@pytest.mark.parametrize("s", S_ALL)
def test_dot_matches_exact_sum(torch, n, s):
    U = [inputs.random_vector(600 + e, n) for e in range(s)]
    V = [inputs.random_vector(700 + e, n, -2.0, 3.0) for e in range(s)]
    out = torch.empty(s, dtype=torch.float64, device=gpu())
    work = torch.empty(E.dot_workspace_size(n, s), dtype=torch.uint8, device=gpu())
    E.dot(n, s, to_dev(O.to_ensemble(U)), to_dev(O.to_ensemble(V)), out, work)
    got = to_np(out)
    for e in range(s):
        prod = U[e] * V[e]
        assert abs(got[e] - math.fsum(prod.tolist())) <= 1e-13 * np.sum(np.abs(prod)), e
    # repeated call reuses the self-resetting counters
    E.dot(n, s, to_dev(O.to_ensemble(U)), to_dev(O.to_ensemble(V)), out, work)
    assert np.array_equal(to_np(out), got)


def test_dot_s_invariant_bitwise(torch):
    n = 10007
    U = [inputs.random_vector(800 + e, n) for e in range(32)]
    ref = None
    for s in S_ALL:
        out = torch.empty(s, dtype=torch.float64, device=gpu())
        work = torch.empty(E.dot_workspace_size(n, s), dtype=torch.uint8, device=gpu())
        u = to_dev(O.to_ensemble(U[:s]))
        E.dot(n, s, u, u, out, work)
        v = to_np(out)[0]
        ref = v if ref is None else ref
        assert v == ref, s


# -------------------------------------------------------------------- A6 CG
def gpu_solve(mesh, xs, tol, max_iter=10000, flags=0, x0=None, check_every=8, presplit=False):
    """presplit: ens_cg_df on the ENS_F64_DF copy of the values."""
    import torch
    s = xs.shape[0]
    vals, b = mesh.assemble(s, to_dev(inputs.ensemble_layout(xs)))
    vdf = None
    if presplit:
        vdf = torch.empty(2 * vals.numel(), dtype=torch.float32, device=gpu())
        E.convert_values(mesh.graph, s, vals, vdf, dtype=E.F64_DF)
    x = torch.zeros(mesh.n * s, dtype=torch.float64, device=gpu()) if x0 is None else x0.clone()
    work = torch.empty(E.cg_workspace_size(mesh.n, s), dtype=torch.uint8, device=gpu())
    it, rr, st, stats = E.cg(mesh.graph, s, vals, b, x, tol, max_iter, work, flags=flags,
                             check_every=check_every, values_df=vdf)
    return ens_cols(to_np(x), s), it, rr, st, stats


def compare_cg(mesh, xs, tol, xg, itg, flags=0):
    rm, col, ov, ob = oracle_members(mesh.N, mesh.M, xs)
    for e in range(xs.shape[0]):
        xo, ito, rro, sto = O.cg(rm, col, ov[e], ob[e], tol=tol)
        assert sto == 0
        assert abs(itg[e] - ito) <= 1, (e, itg[e], ito)
        err = np.linalg.norm(xg[:, e] - xo) / np.linalg.norm(xo)
        if itg[e] == ito:
            assert err <= 1e-8, (e, err)
        else:  # stopping decided by rounding: compare at a fixed iteration count
            k = max(itg[e], ito)
            xo2, _, _, _ = O.cg(rm, col, ov[e], ob[e], tol=0.0, max_iter=k)
            xg2, it2, _, _, _ = gpu_solve(mesh, xs, 0.0, max_iter=k, flags=flags)
            assert it2[e] == k
            assert np.linalg.norm(xg2[:, e] - xo2) / np.linalg.norm(xo2) <= 1e-10


def test_cg_small_workload_exact_iterations(torch):
    # 8^3 cells, M = 3, s = 4, 4 samples, relative residual 1e-10
    mesh = E.Mesh(8, 3)
    xs = inputs.kl_samples(inputs.SEED_SMALL, 0, 4, 3)
    xg, it, rr, st, _ = gpu_solve(mesh, xs, 1e-10)
    assert st == [0, 0, 0, 0]
    rm, col, ov, ob = oracle_members(8, 3, xs)
    for e in range(4):
        xo, ito, rro, sto = O.cg(rm, col, ov[e], ob[e], tol=1e-10)
        assert it[e] == ito
        assert np.linalg.norm(xg[:, e] - xo) / np.linalg.norm(xo) <= 1e-8
        assert rr[e] <= 2e-10 and abs(rr[e] - rro) <= 1e-12
        assert np.all(xg[to_np(mesh.bmask) == 1, e] == 0.0)


@pytest.mark.parametrize("s", S_ALL)
@pytest.mark.parametrize("flags", [0, E.CG_DF64, E.CG_SPLIT64])
def test_cg_matches_oracle_ragged_mesh(torch, s, flags):
    mesh = E.Mesh(13, 10)   # 2744 rows: 85 full 32-row chunks and a ragged one
    xs = inputs.kl_samples(900, 0, s, 10)
    xg, it, rr, st, _ = gpu_solve(mesh, xs, 1e-8, flags=flags)
    assert all(v == 0 for v in st)
    compare_cg(mesh, xs, 1e-8, xg, it, flags)


@pytest.mark.parametrize("s", S_ALL)
@pytest.mark.parametrize("form", ["f64", "df", "split", "dfv"])
def test_cg_spmv_mapping_knob_is_bitwise_neutral(torch, s, form):
    """Every mapping of the CG's SpMV (ENS_CG_K1_CHUNKS, ENS_CG_K1_DEFER) gives
    bitwise the default's solution, iteration counts and residuals: all sums
    are ordered by row index.  13^3 cells: 86 chunks, so the wider mappings
    end with a partly filled CTA and the deferred tree has three level-1
    groups; a 2^3-cell mesh is one chunk; a mapping beyond 1024 threads is
    refused."""
    from paper_1511_03703_gb300 import autotune
    mesh = E.Mesh(13, 10)
    xs = inputs.kl_samples(910, 0, s, 10)
    flags = {"f64": 0, "df": E.CG_DF64, "split": E.CG_SPLIT64, "dfv": 0}[form]
    ref = gpu_solve(mesh, xs, 1e-9, flags=flags | E.CG_GRAPH, presplit=form == "dfv")
    for c in autotune.k1_mapping_choices(s):
        got = gpu_solve(mesh, xs, 1e-9, flags=flags | E.CG_GRAPH | E.cg_k1_chunks(c), presplit=form == "dfv")
        assert got[1] == ref[1] and got[2] == ref[2] and np.array_equal(got[0], ref[0]), c
    # the deferred tree on a mesh of one chunk (the top is the chunk's partials)
    small = E.Mesh(2, 10)
    a = gpu_solve(small, xs, 1e-9, flags=flags, presplit=form == "dfv")
    d = gpu_solve(small, xs, 1e-9, flags=flags | E.CG_K1_DEFER, presplit=form == "dfv")
    assert a[1] == d[1] and a[2] == d[2] and np.array_equal(a[0], d[0])
    too_wide = 2 * max(autotune.k1_chunk_choices(s))
    if too_wide <= 8:
        with pytest.raises(E.EnsError) as ei:
            gpu_solve(mesh, xs, 1e-9, flags=flags | E.cg_k1_chunks(too_wide))
        assert ei.value.code == 1


def test_cg_identical_members_bitwise(torch):
    mesh = E.Mesh(7, 10)
    xs = np.repeat(inputs.kl_samples(77, 3, 1, 10), 8, axis=0)
    vals, b = mesh.assemble(8, to_dev(inputs.ensemble_layout(xs)))
    V = ens_cols(to_np(vals), 8)
    assert all(np.array_equal(V[:, 0], V[:, e]) for e in range(8))
    xg, it, rr, st, _ = gpu_solve(mesh, xs, 1e-10)
    assert len(set(it)) == 1 and all(np.array_equal(xg[:, 0], xg[:, e]) for e in range(8))


@pytest.mark.parametrize("flags", [0, E.CG_DF64, E.CG_SPLIT64])
def test_cg_sample_result_independent_of_s_bitwise(torch, flags):
    mesh = E.Mesh(9, 10)
    xs = inputs.kl_samples(4242, 0, 32, 10)
    ref = None
    for s in S_ALL:
        xg, it, rr, st, _ = gpu_solve(mesh, xs[:s], 1e-9, flags=flags)
        cur = (xg[:, 0].copy(), it[0], rr[0])
        if ref is None:
            ref = cur
        assert np.array_equal(cur[0], ref[0]) and cur[1] == ref[1] and cur[2] == ref[2], s


def test_cg_graph_replay_matches_direct_launches(torch):
    mesh = E.Mesh(8, 3)
    xs = inputs.kl_samples(inputs.SEED_SMALL, 0, 4, 3)
    a = gpu_solve(mesh, xs, 1e-10)
    b = gpu_solve(mesh, xs, 1e-10, flags=E.CG_GRAPH, check_every=5)
    assert np.array_equal(a[0], b[0]) and a[1] == b[1]
    # SpMV timing inside the graph: event-record nodes, same results
    for presplit in (False, True):
        c = gpu_solve(mesh, xs, 1e-10, flags=E.CG_GRAPH | E.CG_TIME_SPMV, check_every=5, presplit=presplit)
        d = gpu_solve(mesh, xs, 1e-10, flags=E.CG_TIME_SPMV, check_every=5, presplit=presplit)
        assert np.array_equal(c[0], d[0]) and c[1] == d[1]
        assert c[4].spmv_launches == max(c[1]) and c[4].spmv_ms > 0.0
        assert d[4].spmv_launches == max(d[1])


@pytest.mark.parametrize("s,flags,presplit", [(4, 0, False), (32, E.CG_DF64, False), (32, 0, True),
                                              (8, E.CG_COUPLED, False), (16, E.cg_k1_chunks("defer"), True)])
def test_cg_device_loop_matches_host_polled_loop(torch, s, flags, presplit):
    """ENS_CG_GRAPH without timing runs the convergence test between blocks on
    the device (a graph while node); with ENS_CG_TIME_SPMV the host polls after
    every replay.  Both run the same number of blocks: identical bits,
    iterations and statuses, and the device loop polls nothing."""
    mesh = E.Mesh(10, 10)
    xs = inputs.kl_samples(97, 0, s, 10)
    for ce in (1, 5, 8):
        a = gpu_solve(mesh, xs, 1e-10, flags=flags | E.CG_GRAPH, check_every=ce, presplit=presplit)
        b = gpu_solve(mesh, xs, 1e-10, flags=flags | E.CG_GRAPH | E.CG_TIME_SPMV, check_every=ce,
                      presplit=presplit)
        assert np.array_equal(a[0], b[0]) and a[1] == b[1] and a[2] == b[2] and a[3] == b[3], ce
        assert a[4].host_checks == 0 and b[4].host_checks >= 1
        blocks = b[4].host_checks
        assert a[4].kernel_launches == b[4].kernel_launches + blocks  # one control kernel per block
    # max_iter reached inside the device loop: the same bounded result as the host loop
    a = gpu_solve(mesh, xs, 0.0, max_iter=13, flags=flags | E.CG_GRAPH, check_every=4, presplit=presplit)
    b = gpu_solve(mesh, xs, 0.0, max_iter=13, flags=flags | E.CG_GRAPH | E.CG_TIME_SPMV, check_every=4,
                  presplit=presplit)
    assert np.array_equal(a[0], b[0]) and a[1] == b[1] and max(a[1]) == 13
    assert all(v == 5 for v in a[3])   # ENS_ERR_NOT_CONVERGED for every member


def test_cg_member_edge_cases(torch):
    mesh = E.Mesh(6, 10)
    s = 4
    xs = inputs.kl_samples(31, 0, s, 10)
    vals, b = mesh.assemble(s, to_dev(inputs.ensemble_layout(xs)))
    ref = gpu_solve(mesh, xs, 1e-10)
    # member 1: zero right-hand side -> x = 0 in 0 iterations; member 2: -A is
    # negative definite -> breakdown at the first p'Ap; members 0 and 3 unaffected
    b.view(-1, s)[:, 1] = 0.0
    vals.view(-1, s)[:, 2] *= -1.0
    x = torch.full((mesh.n * s,), 0.0, dtype=torch.float64, device=gpu())
    x.view(-1, s)[:, 1] = 1.0
    work = torch.empty(E.cg_workspace_size(mesh.n, s), dtype=torch.uint8, device=gpu())
    it, rr, st, _ = E.cg(mesh.graph, s, vals, b, x, 1e-10, 1000, work)
    X = ens_cols(to_np(x), s)
    assert st == [0, 0, 6, 0] and it[1] == 0 and np.all(X[:, 1] == 0.0)
    for e in (0, 3):
        assert it[e] == ref[1][e] and np.array_equal(X[:, e], ref[0][:, e])
    # iteration cap -> not converged, exactly max_iter iterations
    xg, it, rr, st, _ = gpu_solve(mesh, xs, 1e-12, max_iter=3)
    assert st == [5] * s and it == [3] * s
    # resume from the capped iterate converges to the same solution
    x0 = to_dev(np.ascontiguousarray(xg).reshape(-1))
    xr, itr, rrr, str_, _ = gpu_solve(mesh, xs, 1e-10, x0=x0)
    assert str_ == [0] * s
    assert np.linalg.norm(xr - ref[0]) <= 1e-8 * np.linalg.norm(ref[0])


def test_cg_coupled_ensemble(torch):
    mesh = E.Mesh(8, 10)
    xs = inputs.kl_samples(55, 0, 8, 10)
    xd, itd, rrd, std, _ = gpu_solve(mesh, xs, 1e-8)
    xc, itc, rrc, stc, _ = gpu_solve(mesh, xs, 1e-8, flags=E.CG_COUPLED)
    assert stc == [0] * 8 and len(set(itc)) == 1
    # coupled iterations are never fewer than the slowest decoupled member
    assert itc[0] >= max(itd)
    rm, col, ov, ob = oracle_members(8, 10, xs)
    res2 = sum((rrc[e] * np.linalg.norm(ob[e])) ** 2 for e in range(8))
    assert math.sqrt(res2) <= 1.01e-8 * math.sqrt(sum(np.linalg.norm(v) ** 2 for v in ob))
    for e in range(8):
        xo, _, _, _ = O.cg(rm, col, ov[e], ob[e], tol=1e-12)
        assert np.linalg.norm(xc[:, e] - xo) <= 1e-6 * np.linalg.norm(xo)


def block_system(rm, col, vals, bs):
    """The s member systems as one block-diagonal CSR system (members in order)."""
    n = len(rm) - 1
    rmb = np.concatenate([np.asarray(rm[:-1]) + e * len(col) for e in range(len(vals))] +
                         [[len(col) * len(vals)]]).astype(np.int32)
    colb = np.concatenate([np.asarray(col) + e * n for e in range(len(vals))]).astype(np.int32)
    return rmb, colb, np.concatenate(vals), np.concatenate(bs)


@pytest.mark.parametrize("s", [4, 8])
def test_cg_coupled_is_cg_on_the_block_system(torch, s):
    """The coupled ensemble CG of Sects. 3.4 and 3.7 (alpha, beta and the stopping test
    from member-summed dots) is plain CG on the block-diagonal system of all
    members: the oracle's CG on that system gives the same iterates."""
    N, M = 9, 10
    mesh = E.Mesh(N, M)
    xs = inputs.kl_samples(57, 0, s, M)
    xc, itc, rrc, stc, _ = gpu_solve(mesh, xs, 1e-10, flags=E.CG_COUPLED)
    rm, col, ov, ob = oracle_members(N, M, xs)
    xo, ito, rro, sto = O.cg(*block_system(rm, col, ov, ob), tol=1e-10)
    assert stc == [0] * s and sto == 0 and len(set(itc)) == 1
    if itc[0] != ito:  # rounding decided the stopping test: compare at a fixed count
        assert abs(itc[0] - ito) == 1
        k = max(itc[0], ito)
        xc, itc, _, _, _ = gpu_solve(mesh, xs, 0.0, max_iter=k, flags=E.CG_COUPLED)
        xo, ito, _, _ = O.cg(*block_system(rm, col, ov, ob), tol=0.0, max_iter=k)
    Xo = xo.reshape(s, -1).T
    assert np.linalg.norm(xc - Xo) <= 1e-10 * np.linalg.norm(Xo)


def test_error_statuses(torch):
    mesh = E.Mesh(4, 3)
    x = torch.zeros(mesh.n * 4 + 1, dtype=torch.float64, device=gpu())
    y = torch.zeros(mesh.n * 4, dtype=torch.float64, device=gpu())
    vals, b = mesh.assemble(4, to_dev(inputs.ensemble_layout(inputs.kl_samples(1, 0, 4, 3))))
    with pytest.raises(E.EnsError) as ei:
        E.spmv(mesh.graph, 3, vals, x[:-1], y)
    assert ei.value.code == 2
    with pytest.raises(E.EnsError) as ei:
        E.spmv(mesh.graph, 4, vals, x[1:], y)
    assert ei.value.code == 3
    small = torch.empty(64, dtype=torch.uint8, device=gpu())
    with pytest.raises(E.EnsError) as ei:
        E.cg(mesh.graph, 4, vals, b, y, 1e-8, 10, small)
    assert ei.value.code == 9


# ------------------------------------------ full-size workload, sampled checks
def test_scale_64cubed_s32_sampled(torch):
    """64^3 cells, M = 10, s = 32, tol 1e-8: the benchmark's launch shape."""
    N, M, s = 64, 10, 32
    mesh = E.Mesh(N, M)
    xs = inputs.kl_samples(inputs.SEED_SCALE, 0, s, M)
    vals, b = mesh.assemble(s, to_dev(inputs.ensemble_layout(xs)))
    picks = [0, 17]
    rm, col, ov, ob = oracle_members(N, M, xs[picks])
    V = ens_cols(to_np(vals), s)
    for i, e in enumerate(picks):
        assert np.all(np.abs(V[:, e] - ov[i]) <= 1e-13 * np.abs(diag_of(rm, col, ov[i])))
    # SpMV at full size, all 32 members: oracle values of the picked samples tiled
    xm = [inputs.random_vector(1300 + e, mesh.n) for e in range(s)]
    vt = to_dev(O.to_ensemble([ov[e % 2] for e in range(s)]))
    y = torch.empty(mesh.n * s, dtype=torch.float64, device=gpu())
    E.spmv(mesh.graph, s, vt, to_dev(O.to_ensemble(xm)), y)
    Y = ens_cols(to_np(y), s)
    for e in range(s):
        ref = O.spmv(rm, col, ov[e % 2], xm[e])
        assert np.all(np.abs(Y[:, e] - ref) <= spmv_bound(rm, col, ov[e % 2], xm[e])), e
    # CG of the whole ensemble; two members against oracle solves
    oracle_sol = [O.cg(rm, col, ov[i], ob[i], tol=1e-8) for i in range(len(picks))]
    for flags, presplit in ((0, False), (E.CG_DF64, False), (E.CG_SPLIT64, False), (0, True)):
        xg, it, rr, st, _ = gpu_solve(mesh, xs, 1e-8, flags=flags, presplit=presplit)
        assert st == [0] * s and max(rr) < 2e-8
        compare_cg_picked(mesh, xs, picks, rm, col, ov, ob, oracle_sol, xg, it, flags, presplit)


def compare_cg_picked(mesh, xs, picks, rm, col, ov, ob, oracle_sol, xg, it, flags, presplit):
    """Members `picks` against oracle solves: 1e-8 at equal iteration counts;
    else both sides re-run for max(counts) iterations and compared at 1e-10."""
    for i, e in enumerate(picks):
        xo, ito, rro, sto = oracle_sol[i]
        assert sto == 0 and abs(it[e] - ito) <= 1, (e, it[e], ito)
        if it[e] == ito:
            err = np.linalg.norm(xg[:, e] - xo) / np.linalg.norm(xo)
            assert err <= 1e-8, (e, err)
        else:
            k = max(it[e], ito)
            xo2, _, _, _ = O.cg(rm, col, ov[i], ob[i], tol=0.0, max_iter=k)
            xg2, it2, _, _, _ = gpu_solve(mesh, xs, 0.0, max_iter=k, flags=flags, presplit=presplit)
            assert it2[e] == k
            assert np.linalg.norm(xg2[:, e] - xo2) <= 1e-10 * np.linalg.norm(xo2), e


# ------------------------------------ extreme magnitudes (float-pair ranges)
@pytest.mark.parametrize("scale", [1e-20, 2.0 ** -100, 1e25, 2.0 ** 90])
@pytest.mark.parametrize("form", ["f64", "df", "split", "dfv"])
def test_cg_rhs_scaled_far_outside_fp32_range(torch, scale, form):
    """CG with b scaled far below and above FP32's range: the float-pair r.r of
    K2 and the double-float SpMV products leave FP32's normal range, and must
    fall back to FP64 rather than stop early (underflow) or break down
    (overflow).  Status, iteration counts and solutions against the oracle's
    CG on the same scaled system."""
    N, M, s = 9, 10, 4
    mesh = E.Mesh(N, M)
    xs = inputs.kl_samples(1500, 0, s, M)
    vals, b = mesh.assemble(s, to_dev(inputs.ensemble_layout(xs)))
    b *= scale
    vdf = None
    if form == "dfv":
        vdf = torch.empty(2 * vals.numel(), dtype=torch.float32, device=gpu())
        E.convert_values(mesh.graph, s, vals, vdf, dtype=E.F64_DF)
    flags = {"f64": 0, "df": E.CG_DF64, "split": E.CG_SPLIT64, "dfv": 0}[form]
    work = torch.empty(E.cg_workspace_size(mesh.n, s), dtype=torch.uint8, device=gpu())

    def run(tol, max_iter):
        x = torch.zeros(mesh.n * s, dtype=torch.float64, device=gpu())
        it, rr, st, _ = E.cg(mesh.graph, s, vals, b, x, tol, max_iter, work, flags=flags, values_df=vdf)
        return ens_cols(to_np(x), s), it, rr, st

    xg, it, rr, st = run(1e-8, 5000)
    assert st == [0] * s, st
    rm, col, ov, ob = oracle_members(N, M, xs)
    for e in range(s):
        bo = ob[e] * scale
        xo, ito, rro, sto = O.cg(rm, col, ov[e], bo, tol=1e-8)
        assert sto == 0 and abs(it[e] - ito) <= 1, (e, it[e], ito)
        assert rr[e] <= 2e-8, (e, rr[e])
        if it[e] == ito:
            assert np.linalg.norm(xg[:, e] - xo) <= 1e-8 * np.linalg.norm(xo), e
        else:  # stopping decided by rounding: compare at a fixed iteration count
            k = max(it[e], ito)
            xo2, _, _, _ = O.cg(rm, col, ov[e], bo, tol=0.0, max_iter=k)
            xg2, it2, _, _ = run(0.0, k)
            assert it2[e] == k
            assert np.linalg.norm(xg2[:, e] - xo2) <= 1e-10 * np.linalg.norm(xo2), e


@pytest.mark.parametrize("s", [1, 4, 32])
@pytest.mark.parametrize("form", ["df", "split", "dfv"])
@pytest.mark.parametrize("vscale,xscale", [(1.0, 2.0 ** -100), (2.0 ** -30, 2.0 ** -100),
                                           (2.0 ** -60, 2.0 ** -90), (1.0, 2.0 ** -120)])
def test_spmv_df_products_below_fp32_normal_range(torch, s, form, vscale, xscale):
    """Products a_j x_j below 2^-96 (here down to FP32's subnormals and below
    them) with values and x inside the split range, and x below the split range
    (2^-120): the double-float forms recompute such members in FP64 and stay
    inside the 1e-12 componentwise bound; rows of ordinary magnitude in the
    same launch are unaffected.  Members whose every product is below 2^-149
    may return 0: the documented absolute floor 27 * 2^-149."""
    N, M = 5, 10
    xs = inputs.kl_samples(1510, 0, 1, M)
    rm, col, ov, _ = oracle_members(N, M, xs)
    n = len(rm) - 1
    vals = [ov[0] * (1.0 + 0.01 * e) * vscale for e in range(s)]
    xm = []
    for e in range(s):
        v = inputs.random_vector(1520 + e, n, 0.5, 1.0) * np.where(np.arange(n) % 2, 1.0, -1.0)
        v[(np.arange(n) % 3) != 0] *= xscale      # two thirds of the entries tiny
        if e % 2:
            v *= xscale                            # odd members: every entry tiny
        xm.append(v)
    y = torch.empty(n * s, dtype=torch.float64, device=gpu())
    graph = E.Graph(to_dev(rm), to_dev(col))
    spmv_form(torch, graph, s, to_dev(O.to_ensemble(vals)), to_dev(O.to_ensemble(xm)), y, form)
    Y = ens_cols(to_np(y), s)
    for e in range(s):
        ref = O.spmv(rm, col, vals[e], xm[e])
        bound = np.maximum(spmv_bound(rm, col, vals[e], xm[e]), 27 * 2.0 ** -149)
        assert np.all(np.abs(Y[:, e] - ref) <= bound), e
        if vscale * xscale >= 2.0 ** -130:   # products above FP32's subnormal floor: the plain bar
            assert np.all(np.abs(Y[:, e] - ref) <= spmv_bound(rm, col, vals[e], xm[e])), e


@pytest.mark.parametrize("s", [1, 4, 32])
def test_cg_df_tiny_products_bitwise_equals_df64(torch, s):
    """The pre-split form and the df form take the same FP64 decision for
    members with tiny products, so ens_cg_df stays bitwise ens_cg with
    ENS_CG_DF64 (b scaled by 2^-100, fixed iteration count)."""
    N, M = 7, 10
    mesh = E.Mesh(N, M)
    xs = inputs.kl_samples(1530 + s, 0, s, M)
    vals, b = mesh.assemble(s, to_dev(inputs.ensemble_layout(xs)))
    b *= 2.0 ** -100
    vdf = torch.empty(2 * vals.numel(), dtype=torch.float32, device=gpu())
    E.convert_values(mesh.graph, s, vals, vdf, dtype=E.F64_DF)
    work = torch.empty(E.cg_workspace_size(mesh.n, s), dtype=torch.uint8, device=gpu())
    out = []
    for flags, vd in ((E.CG_DF64, None), (0, vdf)):
        x = torch.zeros(mesh.n * s, dtype=torch.float64, device=gpu())
        it, rr, st, _ = E.cg(mesh.graph, s, vals, b, x, 0.0, 40, work, flags=flags, values_df=vd)
        out.append((to_np(x), it, rr))
    assert out[0][1] == out[1][1] and out[0][2] == out[1][2]
    assert np.array_equal(out[0][0], out[1][0])
