"""Multigrid-preconditioned ensemble CG against the FP64 oracle (oracle/multigrid.py).

Bars: iteration counts within one of the oracle's MG-PCG on the same
hierarchy, solutions to 1e-8 relative; member results bitwise independent of
s; graph replay bitwise equal to direct launches; a mesh-independent
iteration count.
"""
import numpy as np
import pytest

from oracle import multigrid as G
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


def start(l, e, n):
    return inputs.random_vector(600 + 100 * l + e, n)


def gpu_mg(torch, mg, xs, tol=1e-10, flags=0, degree=2, ratio=5.0, check_every=4, presplit=False, f32=False,
           power_iters=10):
    """presplit: level 0 assembled in double-float with its pre-split copy, so
    that the level-0 SpMVs (K1 and the V-cycle's) run in double-float."""
    s = xs.shape[0]
    if presplit == "all":   # every level pre-split
        vdf = [torch.empty(2 * m.nnz * s, dtype=torch.float32, device=gpu()) for m in mg.meshes]
    else:
        vdf = torch.empty(2 * mg.meshes[0].nnz * s, dtype=torch.float32, device=gpu()) if presplit else None
    vals, b = mg.assemble(s, to_dev(inputs.ensemble_layout(xs)), values_df=vdf)
    starts = [to_dev(np.stack([start(l, e, m.n) for e in range(s)], axis=1).reshape(-1))
              for l, m in enumerate(mg.meshes)]
    x = torch.zeros(mg.meshes[0].n * s, dtype=torch.float64, device=gpu())
    v32 = mg.to_f32(s, vals) if f32 else None
    work = torch.empty(mg.workspace_size(s, vals, starts, vdf, v32), dtype=torch.uint8, device=gpu())
    it, rr, st, stats = mg.solve(s, vals, b, x, tol, 200, work, starts, degree=degree, ratio=ratio, flags=flags,
                                 check_every=check_every, values_df=vdf, values_f32=v32, power_iters=power_iters)
    return to_np(x).reshape(-1, s), it, rr, st


@pytest.mark.parametrize("presplit", [False, True, "all"])
@pytest.mark.parametrize("s", [1, 4, 32])
def test_mg_pcg_matches_oracle(torch, s, presplit):
    N, M = 16, 10
    mg = E.Multigrid(N, M)
    assert mg.sizes == [16, 8, 4]
    xs = inputs.kl_samples(800 + s, 0, s, M)
    X, it, rr, st = gpu_mg(torch, mg, xs, presplit=presplit)
    assert st == [0] * s and max(rr) <= 1.01e-10
    for e in ([0, s - 1] if s > 2 else range(s)):
        starts = [start(l, e, (n + 1) ** 3) for l, n in enumerate(G.level_sizes(N))]
        lv = G.hierarchy(N, M, xs[e], starts)
        xo, ito, rro, sto = G.mg_pcg(lv, lv[0].load, tol=1e-10)
        assert sto == 0 and abs(it[e] - ito) <= 1, (e, it[e], ito)
        assert np.linalg.norm(X[:, e] - xo) <= 1e-8 * np.linalg.norm(xo), e


@pytest.mark.parametrize("presplit", [False, True, "all"])
def test_mg_member_independent_of_s_and_graph(torch, presplit):
    mg = E.Multigrid(8, 10)
    xs = inputs.kl_samples(820, 0, 32, 10)
    ref = None
    for s in (1, 4, 32):
        X, it, rr, st = gpu_mg(torch, mg, xs[:s], presplit=presplit)
        cur = (X[:, 0].copy(), it[0])
        ref = cur if ref is None else ref
        assert np.array_equal(cur[0], ref[0]) and cur[1] == ref[1], s
    Xg, itg, _, _ = gpu_mg(torch, mg, xs[:8], flags=E.CG_GRAPH, presplit=presplit)
    Xd, itd, _, _ = gpu_mg(torch, mg, xs[:8], presplit=presplit)
    assert itg == itd and np.array_equal(Xg, Xd)


def test_mg_iterations_do_not_grow_with_the_mesh(torch):
    its = []
    for N in (16, 32):
        mg = E.Multigrid(N, 10)
        xs = inputs.kl_samples(830, 0, 4, 10)
        X, it, rr, st = gpu_mg(torch, mg, xs, tol=1e-8)
        assert st == [0] * 4
        its.append(max(it))
    assert its[0] <= 8 and its[1] <= its[0] + 1, its


def test_mg_argument_errors(torch):
    with pytest.raises(E.EnsError):
        E.Multigrid(7, 10)          # no halving down to N <= 4
    mg = E.Multigrid(8, 10)
    xs = inputs.kl_samples(840, 0, 4, 10)
    vals, b = mg.assemble(4, to_dev(inputs.ensemble_layout(xs)))
    starts = [torch.zeros(m.n * 4, dtype=torch.float64, device=gpu()) for m in mg.meshes]
    c = mg._levels(4, vals, starts)
    c[1].N = 3                       # not half of level 0
    import ctypes
    v = ctypes.c_size_t()
    assert E.lib().ens_mg_workspace_size(2, c, 4, ctypes.byref(v)) == 1


def test_mg_64cubed_s32_sampled(torch):
    """The benchmark's shape: 64^3 cells, M = 10, s = 32, every level
    pre-split, tol 1e-8; two members against oracle MG-PCG solves."""
    N, M, s = 64, 10, 32
    mg = E.Multigrid(N, M)
    xs = inputs.kl_samples(inputs.SEED_SCALE, 0, s, M)
    X, it, rr, st = gpu_mg(torch, mg, xs, tol=1e-8, presplit="all")
    assert st == [0] * s and max(rr) <= 1.01e-8 and max(it) <= 8
    for e in (0, 17):
        starts = [start(l, e, (n + 1) ** 3) for l, n in enumerate(G.level_sizes(N))]
        lv = G.hierarchy(N, M, xs[e], starts)
        xo, ito, rro, sto = G.mg_pcg(lv, lv[0].load, tol=1e-8)
        assert sto == 0 and abs(it[e] - ito) <= 1, (e, it[e], ito)
        err = np.linalg.norm(X[:, e] - xo) / np.linalg.norm(xo)
        assert err <= 1e-8 or it[e] != ito, (e, err)


@pytest.mark.parametrize("s,presplit", [(1, False), (4, False), (32, False), (32, "all")])
def test_mg_fp32_vcycle_matches_oracle(torch, s, presplit):
    """The FP32 V-cycle (a mixed-precision preconditioner of the FP64 CG):
    the same tolerance reached in at most one iteration more than the
    oracle's FP64 MG-PCG, solutions to 1e-8."""
    N, M = 16, 10
    mg = E.Multigrid(N, M)
    xs = inputs.kl_samples(850 + s, 0, s, M)
    X, it, rr, st = gpu_mg(torch, mg, xs, presplit=presplit, f32=True)
    assert st == [0] * s and max(rr) <= 1.01e-10
    for e in ([0, s - 1] if s > 2 else range(s)):
        starts = [start(l, e, (n + 1) ** 3) for l, n in enumerate(G.level_sizes(N))]
        lv = G.hierarchy(N, M, xs[e], starts)
        xo, ito, rro, sto = G.mg_pcg(lv, lv[0].load, tol=1e-10)
        assert sto == 0 and ito - 1 <= it[e] <= ito + 1, (e, it[e], ito)
        assert np.linalg.norm(X[:, e] - xo) <= 1e-8 * np.linalg.norm(xo), e


def test_mg_fp32_vcycle_member_independent_of_s_and_graph(torch):
    mg = E.Multigrid(8, 10)
    xs = inputs.kl_samples(870, 0, 32, 10)
    ref = None
    for s in (1, 4, 32):
        X, it, rr, st = gpu_mg(torch, mg, xs[:s], f32=True)
        cur = (X[:, 0].copy(), it[0])
        ref = cur if ref is None else ref
        assert np.array_equal(cur[0], ref[0]) and cur[1] == ref[1], s
    Xg, itg, _, _ = gpu_mg(torch, mg, xs[:8], flags=E.CG_GRAPH, f32=True)
    Xd, itd, _, _ = gpu_mg(torch, mg, xs[:8], f32=True)
    assert itg == itd and np.array_equal(Xg, Xd)


@pytest.mark.parametrize("presplit", [False, "all"])
@pytest.mark.parametrize("s", [1, 4, 32])
def test_mg_pcg_lanczos_matches_oracle(torch, s, presplit):
    """ENS_PC_LANCZOS: every level's smoother bound from 5 Lanczos steps (FP64
    or pre-split SpMVs) against the oracle's MG-PCG on the hierarchy with the
    same Lanczos estimates: iterations within one, solutions to 1e-8."""
    N, M = 16, 10
    mg = E.Multigrid(N, M)
    xs = inputs.kl_samples(850 + s, 0, s, M)
    X, it, rr, st = gpu_mg(torch, mg, xs, presplit=presplit, flags=E.PC_LANCZOS, power_iters=5)
    assert st == [0] * s and max(rr) <= 1.01e-10
    for e in ([0, s - 1] if s > 2 else range(s)):
        starts = [start(l, e, (n + 1) ** 3) for l, n in enumerate(G.level_sizes(N))]
        lv = G.hierarchy(N, M, xs[e], starts, power_iters=5, lanczos=True)
        xo, ito, rro, sto = G.mg_pcg(lv, lv[0].load, tol=1e-10)
        assert sto == 0 and abs(it[e] - ito) <= 1, (e, it[e], ito)
        assert np.linalg.norm(X[:, e] - xo) <= 1e-8 * np.linalg.norm(xo), e


def test_mg_lanczos_member_independent_of_s_and_fp32_converges(torch):
    mg = E.Multigrid(8, 10)
    xs = inputs.kl_samples(860, 0, 32, 10)
    ref = None
    for s in (1, 4, 32):
        X, it, rr, st = gpu_mg(torch, mg, xs[:s], presplit="all", flags=E.PC_LANCZOS, power_iters=5)
        cur = (X[:, 0].copy(), it[0])
        ref = cur if ref is None else ref
        assert np.array_equal(cur[0], ref[0]) and cur[1] == ref[1], s
    # the FP32 V-cycle with its Lanczos bound on the FP32 values: converges
    # to the same FP64 tolerance, close to the FP64 hierarchy's count
    X32, it32, rr32, st32 = gpu_mg(torch, mg, xs[:4], f32=True, flags=E.PC_LANCZOS, power_iters=5)
    X64, it64, rr64, st64 = gpu_mg(torch, mg, xs[:4], flags=E.PC_LANCZOS, power_iters=5)
    assert st32 == [0] * 4 and max(rr32) <= 1.01e-10
    assert max(abs(a - b) for a, b in zip(it32, it64)) <= 1
