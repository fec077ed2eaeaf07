"""Preconditioned ensemble CG (Jacobi, Chebyshev) against the FP64 oracle.

Bars: the largest-eigenvalue estimates to 1e-10 relative; iteration counts
within one of the oracle's PCG with the same preconditioner and solutions to
1e-8 relative; member results bitwise independent of s; graph replay bitwise
equal to direct launches.
"""
import numpy as np
import pytest

import oracle as O
from oracle import precond as P
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


def starts(n, s, seed=500):
    return [inputs.random_vector(seed + e, n) for e in range(s)]


def gpu_pcg(torch, mesh, xs, precond, degree=2, tol=1e-10, iters=10, flags=0, check_every=4):
    s = xs.shape[0]
    vals, b = mesh.assemble(s, to_dev(inputs.ensemble_layout(xs)))
    x = torch.zeros(mesh.n * s, dtype=torch.float64, device=gpu())
    work = torch.empty(E.pcg_workspace_size(mesh.n, s), dtype=torch.uint8, device=gpu())
    v0 = to_dev(O.to_ensemble(starts(mesh.n, s)))
    it, rr, st, lam, stats = E.pcg(mesh.graph, s, vals, b, x, tol, 5000, work, precond=precond, degree=degree,
                                   power_iters=iters, power_start=v0, flags=flags, check_every=check_every)
    return to_np(x).reshape(-1, s), it, rr, st, lam


CASES = [("jacobi", E.PC_JACOBI, 0), ("cheb1", E.PC_CHEBYSHEV, 1), ("cheb2", E.PC_CHEBYSHEV, 2),
         ("cheb3", E.PC_CHEBYSHEV, 3)]


@pytest.mark.parametrize("s", [1, 4, 32])
@pytest.mark.parametrize("name,pc,deg", CASES)
def test_pcg_matches_oracle(torch, s, name, pc, deg):
    N, M = 13, 10
    mesh = E.Mesh(N, M)
    xs = inputs.kl_samples(700 + s, 0, s, M)
    X, it, rr, st, lam = gpu_pcg(torch, mesh, xs, pc, degree=max(deg, 1))
    assert st == [0] * s and max(rr) <= 1.01e-10
    rm, col, ov, ob = oracle_members(N, M, xs)
    v0 = starts(mesh.n, s)
    for e in ([0, s - 1] if s > 2 else range(s)):
        d = P.diagonal(rm, col, ov[e])
        if pc == E.PC_JACOBI:
            pre = lambda r, d=d: r / d
        else:
            lo = P.lam_max(rm, col, ov[e], v0[e], 10)
            assert abs(lam[e] - lo) <= 1e-10 * lo, (e, lam[e], lo)
            pre = lambda r, v=ov[e], lo=lo: P.chebyshev(rm, col, v, r, 1.1 * lo, 30.0, deg)
        xo, ito, rro, sto = P.pcg(rm, col, ov[e], ob[e], pre, tol=1e-10)
        assert sto == 0 and abs(it[e] - ito) <= 1, (e, it[e], ito)
        assert np.linalg.norm(X[:, e] - xo) <= 1e-8 * np.linalg.norm(xo), e


@pytest.mark.parametrize("name,pc,deg", [CASES[0], CASES[2]])
def test_pcg_member_independent_of_s_and_graph(torch, name, pc, deg):
    mesh = E.Mesh(9, 10)
    xs = inputs.kl_samples(720, 0, 32, 10)
    ref = None
    for s in (1, 4, 32):
        X, it, rr, st, lam = gpu_pcg(torch, mesh, xs[:s], pc, degree=deg)
        cur = (X[:, 0].copy(), it[0], lam[0])
        ref = cur if ref is None else ref
        assert np.array_equal(cur[0], ref[0]) and cur[1:] == ref[1:], s
    Xg, itg, _, _, _ = gpu_pcg(torch, mesh, xs[:8], pc, degree=deg, flags=E.CG_GRAPH)
    Xd, itd, _, _, _ = gpu_pcg(torch, mesh, xs[:8], pc, degree=deg)
    assert itg == itd and np.array_equal(Xg, Xd)


def test_pcg_saves_iterations_and_rejects_bad_arguments(torch):
    mesh = E.Mesh(16, 10)
    xs = inputs.kl_samples(730, 0, 4, 10)
    _, it_j, _, _, _ = gpu_pcg(torch, mesh, xs, E.PC_JACOBI, tol=1e-8)
    _, it_c, _, _, _ = gpu_pcg(torch, mesh, xs, E.PC_CHEBYSHEV, degree=3, tol=1e-8)
    vals, b = mesh.assemble(4, to_dev(inputs.ensemble_layout(xs)))
    x = torch.zeros(mesh.n * 4, dtype=torch.float64, device=gpu())
    work = torch.empty(E.cg_workspace_size(mesh.n, 4), dtype=torch.uint8, device=gpu())
    it0, _, _, _ = E.cg(mesh.graph, 4, vals, b, x, 1e-8, 5000, work)
    assert max(it_c) < 0.6 * min(it0) and max(it_j) <= max(it0)
    pw = torch.empty(E.pcg_workspace_size(mesh.n, 4), dtype=torch.uint8, device=gpu())
    for kw, code in (({"precond": 7}, 2), ({"precond": E.PC_CHEBYSHEV, "degree": 9}, 1),
                     ({"precond": E.PC_CHEBYSHEV, "power_start": None}, 1)):
        with pytest.raises(E.EnsError) as ei:
            E.pcg(mesh.graph, 4, vals, b, x, 1e-8, 100, pw, **kw)
        assert ei.value.code == code


@pytest.mark.parametrize("s", [1, 4, 32])
@pytest.mark.parametrize("steps", [5, 8, 12])
def test_pcg_lanczos_bound_matches_oracle(torch, s, steps):
    """ENS_PC_LANCZOS: the Lanczos estimate of the largest eigenvalue of D^-1 A
    (largest Ritz value of the tridiagonal, by bisection on the device) against
    the oracle's (LAPACK on the same tridiagonal) to 1e-10, and the Chebyshev
    PCG built on it against the oracle's.  (One step gives only the start
    vector's Rayleigh quotient, about 2/3 of the largest eigenvalue: the
    Chebyshev polynomial is then not positive on the spectrum and PCG breaks
    down, as it does with too few power steps.)"""
    N, M, deg = 13, 10, 2
    mesh = E.Mesh(N, M)
    xs = inputs.kl_samples(760 + s, 0, s, M)
    X, it, rr, st, lam = gpu_pcg(torch, mesh, xs, E.PC_CHEBYSHEV, degree=deg, iters=steps, flags=E.PC_LANCZOS)
    assert st == [0] * s and max(rr) <= 1.01e-10
    rm, col, ov, ob = oracle_members(N, M, xs)
    v0 = starts(mesh.n, s)
    for e in ([0, s - 1] if s > 2 else range(s)):
        lo = P.lam_max_lanczos(rm, col, ov[e], v0[e], steps)
        assert abs(lam[e] - lo) <= 1e-10 * lo, (e, lam[e], lo)
        pre = lambda r, v=ov[e], lo=lo: P.chebyshev(rm, col, v, r, 1.1 * lo, 30.0, deg)
        xo, ito, rro, sto = P.pcg(rm, col, ov[e], ob[e], pre, tol=1e-10)
        assert sto == 0 and abs(it[e] - ito) <= 1, (e, it[e], ito)
        assert np.linalg.norm(X[:, e] - xo) <= 1e-8 * np.linalg.norm(xo), e


def test_pcg_lanczos_steps_limit(torch):
    mesh = E.Mesh(5, 10)
    xs = inputs.kl_samples(770, 0, 4, 10)
    with pytest.raises(E.EnsError):
        gpu_pcg(torch, mesh, xs, E.PC_CHEBYSHEV, iters=33, flags=E.PC_LANCZOS)
