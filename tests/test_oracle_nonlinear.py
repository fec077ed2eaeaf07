"""Pins for the nonlinear advection-diffusion oracle (oracle/nonlinear.py).

Independent of the oracle's own quadrature: the advection and mass matrices
against their tensor-product closed forms (1-D integrals of hat functions),
the integration-by-parts skew symmetry of C, the quadratic term against the
exact integral of a hat function times x^2, the Jacobian against central
differences of the residual (exact for a quadratic F), GMRES against a sparse
direct solve and its finite termination on a matrix with k distinct
eigenvalues, Newton against a direct linear solve when alpha = beta = 0 and
against MINPACK's hybrid root finder (scipy.optimize.root) on a small mesh.
"""
import numpy as np
import pytest
import scipy.optimize as opt
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle as O
from oracle import multigrid as G
from oracle import nonlinear as NL
from paper_1511_03703_gb300 import inputs

M1 = {0: 2.0 / 3.0, 1: 1.0 / 6.0, -1: 1.0 / 6.0}      # 1-D mass of two hats / h
G1 = {0: 0.0, 1: 0.5, -1: -0.5}                        # 1-D int hat_i hat_j'


def coords(N):
    n1 = N + 1
    t = np.arange(n1 ** 3)
    return np.stack([t % n1, (t // n1) % n1, t // (n1 * n1)], axis=1)


def entry_offsets(mesh):
    c = coords(mesh.N)
    return c[mesh.col] - c[mesh.row]


def interior_pairs(mesh):
    return ~mesh.bm[mesh.row] & ~mesh.bm[mesh.col]


def test_advection_matches_closed_form_and_is_skew():
    N, v = 6, (0.7, -1.3, 2.1)
    mesh = NL.Mesh(N)
    C = NL.advection_values(mesh, v)
    h = 1.0 / N
    off = entry_offsets(mesh)
    ref = np.array([h * h * sum(v[d] * G1[o[d]] * np.prod([M1[o[e]] for e in range(3) if e != d])
                                for d in range(3)) for o in off])
    ip = interior_pairs(mesh)
    assert np.max(np.abs(C[ip] - ref[ip])) <= 1e-15
    assert np.all(C[~ip] == 0.0)
    Cs = sp.csr_matrix((C, mesh.col, mesh.rm)).toarray()
    assert np.max(np.abs(Cs + Cs.T)) <= 1e-16


def test_mass_of_unit_field_is_the_consistent_mass_matrix():
    N = 5
    mesh = NL.Mesh(N)
    Mv = NL.mass_u_values(mesh, np.ones(mesh.n))
    h = 1.0 / N
    ref = np.array([h ** 3 * np.prod([M1[t] for t in o]) for o in entry_offsets(mesh)])
    ip = interior_pairs(mesh)
    assert np.max(np.abs(Mv[ip] - ref[ip])) <= 1e-17
    assert np.all(Mv[~ip] == 0.0)


def test_quadratic_and_advection_terms_of_a_linear_field():
    N, v = 6, (0.4, 1.0, -2.0)
    mesh = NL.Mesh(N)
    h = 1.0 / N
    x = coords(N)[:, 0] * h
    inside = ~mesh.bm
    q = NL.quadratic_term(mesh, x)
    ref = h * h * (h * x * x + h ** 3 / 6.0)               # int hat_i(x) x^2 dx * h * h
    assert np.max(np.abs(q[inside] - ref[inside])) <= 1e-16
    a = NL.advection_term(mesh, x, v)
    assert np.max(np.abs(a[inside] - v[0] * h ** 3)) <= 1e-16


def test_terms_agree_with_their_matrices():
    N, v = 6, (1.0, 1.0, 1.0)
    mesh = NL.Mesh(N)
    u = inputs.random_vector(11, mesh.n) * ~mesh.bm
    inside = ~mesh.bm
    Mu = O.spmv(mesh.rm, mesh.col, NL.mass_u_values(mesh, u), u)
    assert np.max(np.abs(Mu[inside] - NL.quadratic_term(mesh, u)[inside])) <= 1e-15
    Cu = O.spmv(mesh.rm, mesh.col, NL.advection_values(mesh, v), u)
    assert np.max(np.abs(Cu[inside] - NL.advection_term(mesh, u, v)[inside])) <= 1e-15


@pytest.mark.parametrize("alpha,beta", [(0.0, 0.0), (3.0, 0.0), (0.0, 7.0), (10.0, 10.0)])
def test_jacobian_is_the_derivative_of_the_residual(alpha, beta):
    N, M = 6, 4
    xi = inputs.kl_samples(21, 0, 1, M)[0]
    prob = NL.Problem(N, M, xi, alpha, beta)
    mesh = prob.mesh
    u = 0.3 * inputs.random_vector(12, mesh.n) * ~mesh.bm
    d = inputs.random_vector(13, mesh.n) * ~mesh.bm
    eps = 1e-2
    fd = (prob.residual(u + eps * d) - prob.residual(u - eps * d)) / (2 * eps)  # exact: F is quadratic
    Jd = O.spmv(mesh.rm, mesh.col, prob.jacobian(u), d)
    assert np.max(np.abs(fd - Jd)) <= 1e-12 * np.max(np.abs(Jd))


def small_nonsymmetric(N=6, seed=30):
    xi = inputs.kl_samples(seed, 0, 1, 4)[0]
    prob = NL.Problem(N, 4, xi, 40.0, 10.0)
    u = 0.5 * inputs.random_vector(seed + 1, prob.mesh.n) * ~prob.mesh.bm
    return prob, prob.jacobian(u)


def test_gmres_matches_direct_solve_with_and_without_restarts():
    prob, J = small_nonsymmetric()
    m = prob.mesh
    Js = sp.csr_matrix((J, m.col, m.rm))
    assert abs(Js - Js.T).max() > 1e-3                       # really non-symmetric
    b = inputs.random_vector(40, m.n)
    xd = spla.spsolve(Js.tocsc(), b)
    x1, it1, rr1, st1 = NL.gmres(m.rm, m.col, J, b, restart=400, tol=1e-12)
    x2, it2, rr2, st2 = NL.gmres(m.rm, m.col, J, b, restart=7, tol=1e-12, max_iter=5000)
    assert st1 == 0 and st2 == 0 and rr1 <= 1.01e-12 and rr2 <= 1.01e-12
    for x in (x1, x2):
        assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
    assert it2 > it1


def test_gmres_terminates_after_k_distinct_eigenvalues():
    n, k = 60, 5
    lam = np.array([1.0, 2.5, 4.0, 7.0, 11.0])
    diag = lam[np.arange(n) % k]
    T = sp.diags(diag) + sp.diags(0.0 * np.ones(n - 1), 1)    # keep a CRS with stored zeros
    T = sp.csr_matrix(T)
    b = 1.0 + inputs.random_vector(41, n) ** 2
    x, it, rr, st = NL.gmres(T.indptr.astype(np.int32), T.indices.astype(np.int32), T.data, b, tol=1e-13)
    assert st == 0 and it == k and rr <= 1e-12
    assert np.max(np.abs(x - b / diag)) <= 1e-13


def test_gmres_with_exact_preconditioner_takes_one_step():
    prob, J = small_nonsymmetric(5, 50)
    m = prob.mesh
    lu = spla.splu(sp.csr_matrix((J, m.col, m.rm)).tocsc())
    b = inputs.random_vector(42, m.n)
    x, it, rr, st = NL.gmres(m.rm, m.col, J, b, precond=lu.solve, tol=1e-12)
    assert st == 0 and it == 1 and rr <= 1e-13


def test_newton_is_one_linear_solve_when_linear():
    N, M = 6, 4
    xi = inputs.kl_samples(60, 0, 1, M)[0]
    prob = NL.Problem(N, M, xi, 0.0, 0.0)
    m = prob.mesh
    u, k, lin, hist, st = NL.newton(prob, tol=1e-10, lin_tol=1e-12, restart=200)
    ud = spla.spsolve(sp.csr_matrix((prob.A, m.col, m.rm)).tocsc(), prob.b)
    assert st == 0 and k == 1
    assert np.linalg.norm(u - ud) <= 1e-10 * np.linalg.norm(ud)


def test_newton_matches_minpack_root_and_converges_quadratically():
    N, M = 4, 4
    xi = inputs.kl_samples(61, 0, 1, M)[0]
    prob = NL.Problem(N, M, xi, 10.0, 400.0)
    m = prob.mesh
    u, k, lin, hist, st = NL.newton(prob, tol=1e-13, lin_tol=1e-14, restart=200)
    assert st == 0 and 3 <= k <= 8
    sol = opt.root(prob.residual, np.zeros(m.n), method="hybr", tol=1e-14)
    assert sol.success
    assert np.linalg.norm(u - sol.x) <= 1e-10 * np.linalg.norm(sol.x)
    # quadratic: ||F_{k+1}|| / ||F_k||^2 stays bounded while far above rounding
    h = np.array(hist) / hist[0]
    ratios = [h[i + 1] / h[i] ** 2 for i in range(len(h) - 1) if h[i + 1] > 1e-12]
    assert len(ratios) >= 2 and max(ratios[1:]) <= 10.0 * max(ratios[0], 1.0)


def test_newton_with_multigrid_preconditioner():
    N, M = 8, 10
    xi = inputs.kl_samples(62, 0, 1, M)[0]
    prob = NL.Problem(N, M, xi, 1.0, 10.0)
    starts = [inputs.random_vector(600 + l, (n + 1) ** 3) for l, n in enumerate(G.level_sizes(N))]
    levels = G.hierarchy(N, M, xi, starts)
    pre = lambda r: G.vcycle(levels, r)
    u1, k1, lin1, _, st1 = NL.newton(prob, tol=1e-10, lin_tol=1e-11, precond=pre)
    u0, k0, lin0, _, st0 = NL.newton(prob, tol=1e-10, lin_tol=1e-11, restart=200)
    assert st1 == 0 and st0 == 0 and k1 == k0
    assert np.linalg.norm(u1 - u0) <= 1e-9 * np.linalg.norm(u0)
    assert max(lin1) <= 12 and sum(lin1) < 0.5 * sum(lin0)
    assert np.linalg.norm(prob.residual(u1)) <= 1e-10 * np.linalg.norm(prob.b)
