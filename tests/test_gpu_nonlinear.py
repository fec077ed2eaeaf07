"""Newton-GMRES for the nonlinear advection-diffusion problem against the FP64
oracle (oracle/nonlinear.py).

Bars: the advection matrix, the Jacobian and the residual to 1e-14 of their
scale; GMRES iteration counts within one of the oracle's (two with restarts)
and solutions to 1e-8 relative; Newton step counts equal to the oracle's,
GMRES steps per solve within one per Newton step, solutions to 1e-8; member
results bitwise independent of s.
"""
import numpy as np
import pytest

import oracle as O
from oracle import multigrid as G
from oracle import nonlinear as NL
import paper_1511_03703_gb300 as E
from paper_1511_03703_gb300 import inputs
from helpers import gpu, to_dev, to_np

pytestmark = pytest.mark.gpu

V = (1.0, 1.0, 1.0)


@pytest.fixture(scope="module")
def torch():
    import torch as T
    assert T.cuda.is_available()
    E.lib()
    return T


def start(l, e, n):
    return inputs.random_vector(600 + 100 * l + e, n)


def dev_starts(nl, s):
    return [to_dev(np.stack([start(l, e, m.n) for e in range(s)], axis=1).reshape(-1))
            for l, m in enumerate(nl.meshes)]


def zero_boundary_field(seed, mesh_o, s, scale=0.3):
    return [scale * inputs.random_vector(seed + e, mesh_o.n) * ~mesh_o.bm for e in range(s)]


def test_advection_matches_oracle(torch):
    N, v = 7, (0.7, -1.3, 2.1)
    mesh = E.Mesh(N, 3)
    C = to_np(E.nl_advection(mesh, v))
    ref = NL.advection_values(NL.Mesh(N), v)
    assert np.max(np.abs(C - ref)) <= 1e-15 * np.max(np.abs(ref))


@pytest.mark.parametrize("s", [1, 4, 32])
def test_jacobian_and_residual_match_oracle(torch, s):
    N, M, alpha, beta = 6, 4, 5.0, 10.0
    mesh = E.Mesh(N, M)
    xs = inputs.kl_samples(900 + s, 0, s, M)
    A, b = mesh.assemble(s, to_dev(inputs.ensemble_layout(xs)))
    C = E.nl_advection(mesh, V)
    mo = NL.Mesh(N)
    us = zero_boundary_field(910, mo, s)
    J, F = E.nl_jacobian(mesh, s, A, C, alpha, beta, b, to_dev(O.to_ensemble(us)))
    J, F = to_np(J).reshape(-1, s), to_np(F).reshape(-1, s)
    for e in ([0, s - 1] if s > 2 else range(s)):
        prob = NL.Problem(N, M, xs[e], alpha, beta, v=V)
        Jo, Fo = prob.jacobian(us[e]), prob.residual(us[e])
        assert np.max(np.abs(J[:, e] - Jo)) <= 1e-14 * np.max(np.abs(Jo)), e
        # F's scale: the terms it sums, |J| |u| + |b|
        scale = np.max(O.spmv(mo.rm, mo.col, np.abs(Jo), np.abs(us[e])) + np.abs(prob.b))
        assert np.max(np.abs(F[:, e] - Fo)) <= 1e-14 * scale, e


def gmres_case(torch, s, precond, restart, N=8, seed=920):
    M = 10
    nl = E.Nonlinear(N, M, v=V, precond=precond)
    xs = inputs.kl_samples(seed, 0, s, M)
    vals, b = nl.assemble(s, to_dev(inputs.ensemble_layout(xs)))
    mo = NL.Mesh(N)
    us = zero_boundary_field(seed + 50, mo, s)
    J, _ = E.nl_jacobian(nl.mesh, s, vals[0], nl.C, 5.0, 10.0, b, to_dev(O.to_ensemble(us)))
    rhs = [inputs.random_vector(seed + 100 + e, mo.n) for e in range(s)]
    starts = dev_starts(nl, s) if precond == E.NL_PRECOND_MG else None
    x = torch.empty(mo.n * s, dtype=torch.float64, device=gpu())
    work = torch.empty(nl.gmres_workspace_size(s, vals, starts, restart), dtype=torch.uint8, device=gpu())
    it, rr, st, stats = nl.gmres(s, vals, J, to_dev(O.to_ensemble(rhs)), x, work, starts, 1e-10, restart=restart,
                                 max_iter=400)
    return nl, xs, us, rhs, to_np(J).reshape(-1, s), to_np(x).reshape(-1, s), it, rr, st


@pytest.mark.parametrize("s", [1, 4, 8, 16, 32])
@pytest.mark.parametrize("precond", [E.NL_PRECOND_NONE, E.NL_PRECOND_MG])
def test_gmres_matches_oracle(torch, s, precond):
    nl, xs, us, rhs, J, X, it, rr, st = gmres_case(torch, s, precond, 30)
    assert st == [0] * s and max(rr) <= 1.01e-10
    mo = NL.Mesh(8)
    for e in ([0, s - 1] if s > 2 else range(s)):
        pre = None
        if precond == E.NL_PRECOND_MG:
            lv = G.hierarchy(8, 10, xs[e], [start(l, e, (n + 1) ** 3) for l, n in enumerate(G.level_sizes(8))])
            pre = lambda r, lv=lv: G.vcycle(lv, r)
        xo, ito, rro, sto = NL.gmres(mo.rm, mo.col, J[:, e], rhs[e], pre, restart=30, tol=1e-10, max_iter=400)
        assert sto == 0 and abs(it[e] - ito) <= 1, (e, it[e], ito)
        assert np.linalg.norm(X[:, e] - xo) <= 1e-8 * np.linalg.norm(xo), e


def test_gmres_restarts_match_oracle(torch):
    s = 4
    nl, xs, us, rhs, J, X, it, rr, st = gmres_case(torch, s, E.NL_PRECOND_NONE, 5, N=6, seed=940)
    assert st == [0] * s and max(rr) <= 1.01e-10
    mo = NL.Mesh(6)
    for e in range(s):
        xo, ito, rro, sto = NL.gmres(mo.rm, mo.col, J[:, e], rhs[e], None, restart=5, tol=1e-10, max_iter=400)
        assert sto == 0 and ito > 5 and abs(it[e] - ito) <= 2, (e, it[e], ito)
        assert np.linalg.norm(X[:, e] - xo) <= 1e-8 * np.linalg.norm(xo), e


def test_gmres_longest_restart_and_no_iterations(torch):
    s = 4
    nl, xs, us, rhs, J, X, it, rr, st = gmres_case(torch, s, E.NL_PRECOND_NONE, 64, N=6, seed=950)
    assert st == [0] * s and max(rr) <= 1.01e-10
    mo = NL.Mesh(6)
    for e in range(s):
        xo, ito, rro, sto = NL.gmres(mo.rm, mo.col, J[:, e], rhs[e], None, restart=400, tol=1e-10)
        assert ito <= 64 and abs(it[e] - ito) <= 1, (e, it[e], ito)
        assert np.linalg.norm(X[:, e] - xo) <= 1e-8 * np.linalg.norm(xo), e
    # max_iter = 0: x stays 0 and every member with b != 0 is reported not converged
    vals, _ = nl.assemble(s, to_dev(inputs.ensemble_layout(xs)))
    x = torch.full((mo.n * s,), 7.0, dtype=torch.float64, device=gpu())
    work = torch.empty(nl.gmres_workspace_size(s, vals, None, 8), dtype=torch.uint8, device=gpu())
    it0, rr0, st0, _ = nl.gmres(s, vals, to_dev(J.reshape(-1)), to_dev(O.to_ensemble(rhs)), x, work, None,
                                1e-10, restart=8, max_iter=0)
    assert it0 == [0] * s and st0 == [E.ERR_NOT_CONVERGED] * s and not torch.any(x != 0)


def newton_case(torch, s, N, alpha, beta, precond=E.NL_PRECOND_MG, seed=960, presplit=False, f32=False, **kw):
    M = 10
    nl = E.Nonlinear(N, M, v=V, precond=precond)
    xs = inputs.kl_samples(seed, 0, s, M)
    if presplit == "all":
        vdf = [torch.empty(2 * m.nnz * s, dtype=torch.float32, device=gpu()) for m in nl.meshes]
    else:
        vdf = torch.empty(2 * nl.mesh.nnz * s, dtype=torch.float32, device=gpu()) if presplit else None
    vals, b = nl.assemble(s, to_dev(inputs.ensemble_layout(xs)), values_df=vdf)
    starts = dev_starts(nl, s) if precond == E.NL_PRECOND_MG else None
    p = nl.params(alpha, beta, **kw)
    u = torch.zeros(nl.mesh.n * s, dtype=torch.float64, device=gpu())
    v32 = nl.mg.to_f32(s, vals) if f32 else None
    work = torch.empty(nl.workspace_size(s, vals, starts, p, vdf, v32), dtype=torch.uint8, device=gpu())
    ni, li, rr, st, stats = nl.solve(s, vals, b, u, work, starts, p, values_df=vdf, values_f32=v32)
    return xs, to_np(u).reshape(-1, s), ni, li, rr, st


@pytest.mark.parametrize("s,presplit", [(1, False), (4, False), (8, False), (16, True), (32, False), (4, True),
                                        (32, True), (32, "all")])
def test_newton_matches_oracle(torch, s, presplit):
    N, alpha, beta, tol, lin_tol = 8, 1.0, 10.0, 1e-10, 1e-11
    xs, U, ni, li, rr, st = newton_case(torch, s, N, alpha, beta, tol=tol, lin_tol=lin_tol, presplit=presplit)
    assert st == [0] * s and max(rr) <= tol
    for e in ([0, s - 1] if s > 2 else range(s)):
        prob = NL.Problem(N, 10, xs[e], alpha, beta, v=V)
        lv = G.hierarchy(N, 10, xs[e], [start(l, e, (n + 1) ** 3) for l, n in enumerate(G.level_sizes(N))])
        uo, ko, lino, hist, sto = NL.newton(prob, tol=tol, lin_tol=lin_tol, precond=lambda r, lv=lv: G.vcycle(lv, r))
        assert sto == 0 and ni[e] == ko, (e, ni[e], ko)
        assert abs(li[e] - sum(lino)) <= ko, (e, li[e], lino)
        assert np.linalg.norm(U[:, e] - uo) <= 1e-8 * np.linalg.norm(uo), e


@pytest.mark.parametrize("s,presplit", [(4, False), (32, "all")])
def test_newton_lanczos_bound_matches_oracle(torch, s, presplit):
    """ENS_PC_LANCZOS in the Newton parameters: the V-cycle's eigenvalue bounds
    by 5 Lanczos steps; against the oracle's Newton with the same hierarchy."""
    N, alpha, beta, tol, lin_tol = 8, 1.0, 10.0, 1e-10, 1e-11
    xs, U, ni, li, rr, st = newton_case(torch, s, N, alpha, beta, tol=tol, lin_tol=lin_tol, presplit=presplit,
                                        power_iters=5, flags=E.PC_LANCZOS)
    assert st == [0] * s and max(rr) <= tol
    for e in ([0, s - 1] if s > 2 else range(s)):
        prob = NL.Problem(N, 10, xs[e], alpha, beta, v=V)
        lv = G.hierarchy(N, 10, xs[e], [start(l, e, (n + 1) ** 3) for l, n in enumerate(G.level_sizes(N))],
                         power_iters=5, lanczos=True)
        uo, ko, lino, hist, sto = NL.newton(prob, tol=tol, lin_tol=lin_tol, precond=lambda r, lv=lv: G.vcycle(lv, r))
        assert sto == 0 and ni[e] == ko, (e, ni[e], ko)
        assert abs(li[e] - sum(lino)) <= ko, (e, li[e], lino)
        assert np.linalg.norm(U[:, e] - uo) <= 1e-8 * np.linalg.norm(uo), e


def test_newton_member_independent_of_s(torch):
    ref = None
    for s in (1, 4, 32):
        xs, U, ni, li, rr, st = newton_case(torch, s, 8, 1.0, 10.0, seed=980, tol=1e-10, lin_tol=1e-11)
        cur = (U[:, 0].copy(), ni[0], li[0])
        ref = cur if ref is None else ref
        assert np.array_equal(cur[0], ref[0]) and cur[1:] == ref[1:], s


def test_newton_linear_case_is_one_solve(torch):
    s, N = 4, 8
    xs, U, ni, li, rr, st = newton_case(torch, s, N, 0.0, 0.0, precond=E.NL_PRECOND_NONE, tol=1e-10,
                                        lin_tol=1e-12, restart=60)
    assert st == [0] * s and ni == [1] * s
    rm, col = O.graph(N)
    for e in range(s):
        v, bo = O.assemble(N, 10, xs[e], rm, col)
        xo, _, _, _ = O.cg(rm, col, v, bo, tol=1e-12)
        assert np.linalg.norm(U[:, e] - xo) <= 1e-9 * np.linalg.norm(xo), e


def test_newton_argument_errors(torch):
    nl = E.Nonlinear(8, 10, v=V, precond=E.NL_PRECOND_NONE)
    xs = inputs.kl_samples(990, 0, 4, 10)
    vals, b = nl.assemble(4, to_dev(inputs.ensemble_layout(xs)))
    u = torch.zeros(nl.mesh.n * 4, dtype=torch.float64, device=gpu())
    for kw in ({"restart": 0}, {"restart": 65}, {"check_every": 0}):
        p = nl.params(1.0, 1.0, **kw)
        with pytest.raises(E.EnsError):
            nl.workspace_size(4, vals, None, p) if "restart" in kw else nl.solve(
                4, vals, b, u, torch.empty(1 << 20, dtype=torch.uint8, device=gpu()), None, p)
    p = nl.params(1.0, 1.0)
    small = torch.empty(1024, dtype=torch.uint8, device=gpu())
    with pytest.raises(E.EnsError) as ei:
        nl.solve(4, vals, b, u, small, None, p)
    assert ei.value.code == E.ERR_WORKSPACE


def test_newton_64cubed_s32_sampled(torch):
    """The benchmark's shape: 64^3 cells, s = 32, alpha = 1, beta = 10, Newton
    to 1e-8, GMRES(30) to 1e-6 per step, V-cycle with level 0 pre-split; two
    members against oracle Newton solves, and their residuals re-evaluated by
    the oracle."""
    N, s, tol, lin_tol = 64, 32, 1e-8, 1e-6
    xs, U, ni, li, rr, st = newton_case(torch, s, N, 1.0, 10.0, seed=inputs.SEED_SCALE, presplit="all", tol=tol,
                                        lin_tol=lin_tol, restart=30, max_lin=300)
    assert st == [0] * s and max(rr) <= tol
    for e in (0, 31):
        prob = NL.Problem(N, 10, xs[e], 1.0, 10.0, v=V)
        f0 = np.linalg.norm(prob.b)
        assert np.linalg.norm(prob.residual(U[:, e])) <= 1.01 * tol * f0, e
        lv = G.hierarchy(N, 10, xs[e], [start(l, e, (n + 1) ** 3) for l, n in enumerate(G.level_sizes(N))])
        uo, ko, lino, hist, sto = NL.newton(prob, tol=tol, lin_tol=lin_tol, restart=30, max_lin=300,
                                            precond=lambda r, lv=lv: G.vcycle(lv, r))
        assert sto == 0 and ni[e] == ko, (e, ni[e], ko)
        assert abs(li[e] - sum(lino)) <= ko, (e, li[e], lino)
        assert np.linalg.norm(U[:, e] - uo) <= 1e-7 * np.linalg.norm(uo), e


def test_gmres_zero_rhs_member_and_newton_step_limit(torch):
    """A member with b = 0 is solved by x = 0 at once while the others iterate;
    Newton stopped by max_newton reports not converged after that many steps."""
    s = 4
    nl = E.Nonlinear(6, 10, v=V, precond=E.NL_PRECOND_NONE)
    xs = inputs.kl_samples(970, 0, s, 10)
    vals, b = nl.assemble(s, to_dev(inputs.ensemble_layout(xs)))
    mo = NL.Mesh(6)
    us = zero_boundary_field(975, mo, s)
    J, _ = E.nl_jacobian(nl.mesh, s, vals[0], nl.C, 5.0, 10.0, b, to_dev(O.to_ensemble(us)))
    rhs = [inputs.random_vector(980 + e, mo.n) for e in range(s)]
    rhs[2] = np.zeros(mo.n)
    x = torch.full((mo.n * s,), 3.0, dtype=torch.float64, device=gpu())
    work = torch.empty(nl.gmres_workspace_size(s, vals, None, 10), dtype=torch.uint8, device=gpu())
    it, rr, st, _ = nl.gmres(s, vals, J, to_dev(O.to_ensemble(rhs)), x, work, None, 1e-10, restart=10,
                             max_iter=400)
    X = to_np(x).reshape(-1, s)
    Jn = to_np(J).reshape(-1, s)
    assert st == [0] * s and it[2] == 0 and rr[2] == 0.0 and not np.any(X[:, 2])
    for e in (0, 1, 3):
        xo, ito, _, sto = NL.gmres(mo.rm, mo.col, Jn[:, e], rhs[e], None, restart=10, tol=1e-10, max_iter=400)
        assert abs(it[e] - ito) <= 2 and np.linalg.norm(X[:, e] - xo) <= 1e-8 * np.linalg.norm(xo), e
    xs2, U, ni, li, rr2, st2 = newton_case(torch, 4, 8, 1.0, 10.0, precond=E.NL_PRECOND_NONE, tol=1e-14,
                                           lin_tol=1e-3, max_newton=1, restart=30)
    assert ni == [1] * 4 and st2 == [E.ERR_NOT_CONVERGED] * 4 and min(rr2) > 1e-14


@pytest.mark.parametrize("s,presplit", [(4, False), (32, "all")])
def test_newton_fp32_vcycle_matches_oracle(torch, s, presplit):
    """Newton with the FP32 V-cycle inside the flexible GMRES: the same Newton
    steps as the oracle (FP64 V-cycle), GMRES steps within one per Newton step
    more or less, solutions to 1e-8."""
    N, alpha, beta, tol, lin_tol = 8, 1.0, 10.0, 1e-10, 1e-11
    xs, U, ni, li, rr, st = newton_case(torch, s, N, alpha, beta, tol=tol, lin_tol=lin_tol, presplit=presplit,
                                        f32=True)
    assert st == [0] * s and max(rr) <= tol
    for e in ([0, s - 1] if s > 2 else range(s)):
        prob = NL.Problem(N, 10, xs[e], alpha, beta, v=V)
        lv = G.hierarchy(N, 10, xs[e], [start(l, e, (n + 1) ** 3) for l, n in enumerate(G.level_sizes(N))])
        uo, ko, lino, hist, sto = NL.newton(prob, tol=tol, lin_tol=lin_tol, precond=lambda r, lv=lv: G.vcycle(lv, r))
        assert sto == 0 and ni[e] == ko, (e, ni[e], ko)
        assert abs(li[e] - sum(lino)) <= ko, (e, li[e], lino)
        assert np.linalg.norm(U[:, e] - uo) <= 1e-8 * np.linalg.norm(uo), e
