"""Pins for the preconditioned-CG oracle (Jacobi, Chebyshev, power iteration, Lanczos).

The Chebyshev preconditioner against its closed form through the Chebyshev
polynomials T_k of the scaled spectrum (Saad, Sect. 12.3: the error after k
steps is T_k((theta - A')/delta) / T_k(theta/delta) times the initial error,
A' = D^-1 A); the eigenvalue estimate against a dense symmetric eigen-solve;
PCG against direct solves, its finite termination, and the plain CG when the
preconditioner is the identity.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from numpy.polynomial import chebyshev as C

import oracle as O
from oracle import precond as P
from paper_1511_03703_gb300 import inputs


def system(N=3, seed=5):
    rm, col = O.graph(N)
    v, b = O.assemble(N, 10, inputs.kl_samples(seed, 0, 1, 10)[0], rm, col)
    return rm, col, v, b


def dense(rm, col, v):
    return sp.csr_matrix((v, col, rm)).toarray()


def scaled_eig(rm, col, v):
    A = dense(rm, col, v)
    dh = 1.0 / np.sqrt(np.diag(A))
    lam, V = np.linalg.eigh(dh[:, None] * A * dh[None, :])
    return A, dh, lam, V


def test_diagonal_extracts_the_diagonal():
    rm, col, v, _ = system()
    assert np.array_equal(P.diagonal(rm, col, v), np.diag(dense(rm, col, v)))


def test_lam_max_converges_to_the_largest_scaled_eigenvalue():
    rm, col, v, _ = system(3)
    A, dh, lam, V = scaled_eig(rm, col, v)
    est = P.lam_max(rm, col, v, inputs.random_vector(7, len(rm) - 1), 20000)
    # the spectrum of D^-1 A is that of D^-1/2 A D^-1/2
    assert abs(est - lam[-1]) <= 1e-8 * lam[-1]
    # a few steps give a lower bound (Rayleigh quotient)
    assert P.lam_max(rm, col, v, inputs.random_vector(7, len(rm) - 1), 3) <= lam[-1] * (1 + 1e-14)


def test_chebyshev_matches_the_closed_form():
    rm, col, v, _ = system(3)
    A, dh, lam, V = scaled_eig(rm, col, v)
    r = inputs.random_vector(11, len(rm) - 1)
    e0 = np.linalg.solve(A, r)
    lmax = lam[-1] * 1.05
    for ratio in (10.0, 30.0):
        lmin = lmax / ratio
        theta, delta = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
        for k in (1, 2, 3, 5):
            Tk = C.Chebyshev.basis(k)
            ck = Tk((theta - lam) / delta) / Tk(theta / delta)
            # e_k = D^-1/2 V C_k(Lambda) V^T D^1/2 e_0,  z_k = e_0 - e_k
            ek = dh * (V @ (ck * (V.T @ (e0 / dh))))
            z = P.chebyshev(rm, col, v, r, lmax, ratio, k)
            assert np.max(np.abs(z - (e0 - ek))) <= 1e-10 * np.max(np.abs(e0)), (ratio, k)


def test_chebyshev_preconditioner_is_symmetric_positive():
    rm, col, v, _ = system(3)
    A, dh, lam, V = scaled_eig(rm, col, v)
    n = len(rm) - 1
    Mi = np.stack([P.chebyshev(rm, col, v, np.eye(n)[i], lam[-1] * 1.1, 30.0, 3) for i in range(n)], axis=1)
    assert np.max(np.abs(Mi - Mi.T)) <= 1e-12 * np.max(np.abs(Mi))
    assert np.linalg.eigvalsh(0.5 * (Mi + Mi.T)).min() > 0


def test_pcg_matches_direct_solves():
    rm, col, v, b = system(6, 9)
    xd = spla.spsolve(sp.csr_matrix((v, col, rm)).tocsc(), b)
    d = P.diagonal(rm, col, v)
    lm = P.lam_max(rm, col, v, inputs.random_vector(7, len(b)), 20)
    for name, pre in (("none", lambda r: r.copy()), ("jacobi", lambda r: r / d),
                      ("cheb2", lambda r: P.chebyshev(rm, col, v, r, 1.1 * lm, 30.0, 2)),
                      ("cheb3", lambda r: P.chebyshev(rm, col, v, r, 1.1 * lm, 30.0, 3))):
        x, it, rr, st = P.pcg(rm, col, v, b, pre, tol=1e-12)
        assert st == 0 and rr <= 1e-11, name
        assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd), name


def test_pcg_identity_is_the_plain_cg_and_jacobi_terminates():
    rm, col, v, b = system(5, 13)
    x1, it1, _, _ = P.pcg(rm, col, v, b, lambda r: r.copy(), tol=1e-10)
    x2, it2, _, _ = O.cg(rm, col, v, b, tol=1e-10)
    assert it1 == it2 and np.linalg.norm(x1 - x2) <= 1e-12 * np.linalg.norm(x2)
    # D^-1 A with two distinct eigenvalues: Jacobi-PCG ends in at most 2 steps.
    # S = 2 J + beta (I - J), J = 11^T / n, has unit diagonal and eigenvalues
    # 2 and beta; A = D^1/2 S D^1/2 has diagonal D and D^-1 A similar to S
    n = 40
    rng = np.random.default_rng(3)
    J = np.full((n, n), 1.0 / n)
    beta = (1.0 - 2.0 / n) / (1.0 - 1.0 / n)
    S = 2.0 * J + beta * (np.eye(n) - J)
    dd = 1.0 + rng.random(n)
    A = np.sqrt(dd)[:, None] * S * np.sqrt(dd)[None, :]
    Acsr = sp.csr_matrix(A)
    rmA, colA, vA = Acsr.indptr.astype(np.int32), Acsr.indices.astype(np.int32), Acsr.data
    bA = inputs.random_vector(17, n)
    x, it, rr, st = P.pcg(rmA, colA, vA, bA, lambda r: r / np.diag(A), tol=1e-12)
    assert st == 0 and it <= 2 and np.linalg.norm(A @ x - bA) <= 1e-11 * np.linalg.norm(bA)


def tridiag_laplacian(n):
    """1D tridiag(-1, 2, -1) as CSR: D = 2 I, and the eigenvalues of D^-1 A are
    1 - cos(k pi / (n + 1)), k = 1..n (closed form)."""
    rm, col, v = [0], [], []
    for i in range(n):
        for j, a in ((i - 1, -1.0), (i, 2.0), (i + 1, -1.0)):
            if 0 <= j < n:
                col.append(j)
                v.append(a)
        rm.append(len(col))
    return np.array(rm, np.int32), np.array(col, np.int32), np.array(v)


def test_lanczos_is_exact_on_the_whole_krylov_space():
    # n steps span the whole space: the largest Ritz value is the largest
    # eigenvalue, here the closed form 1 + cos(pi / (n + 1))
    n = 12
    rm, col, v = tridiag_laplacian(n)
    est = P.lam_max_lanczos(rm, col, v, inputs.random_vector(3, n), n)
    assert abs(est - (1.0 + np.cos(np.pi / (n + 1)))) <= 1e-12


def test_lanczos_terminates_after_the_distinct_eigenvalues():
    # D^-1 A with five distinct eigenvalues (two decoupled 2x2 blocks of one
    # kind, one of another, an isolated row): exact after 5 steps (finite
    # termination), and the repeated block adds no step
    rm = np.array([0, 2, 4, 6, 8, 10, 12, 13], np.int32)
    col = np.array([0, 1, 0, 1, 2, 3, 2, 3, 4, 5, 4, 5, 6], np.int32)
    v = np.array([2.0, -1.0, -1.0, 2.0, 2.0, -1.0, -1.0, 2.0, 4.0, 1.0, 1.0, 4.0, 3.0])
    # block [[2,-1],[-1,2]]/2: 1/2, 3/2; block [[4,1],[1,4]]/4: 3/4, 5/4; row: 1
    est = P.lam_max_lanczos(rm, col, v, inputs.random_vector(4, 7), 5)
    assert abs(est - 1.5) <= 1e-12


def test_lanczos_bounds_the_power_estimate_from_below_and_above():
    rm, col, v, _ = system(3)
    A, dh, lam, V = scaled_eig(rm, col, v)
    v0 = inputs.random_vector(7, len(rm) - 1)
    prev = 0.0
    for k in range(1, 9):
        est = P.lam_max_lanczos(rm, col, v, v0, k)
        # a Ritz value: never above the largest eigenvalue, never decreasing
        # with k, and never below the power estimate that uses k - 1 products
        # of the same start (its vector lies in the same Krylov space)
        assert est <= lam[-1] * (1 + 1e-13)
        assert est >= prev - 1e-13 * lam[-1]
        if k >= 2:
            assert est >= P.lam_max(rm, col, v, v0, k - 1) - 1e-13 * lam[-1]
        prev = est
    assert abs(P.lam_max_lanczos(rm, col, v, v0, 30) - lam[-1]) <= 1e-9 * lam[-1]
