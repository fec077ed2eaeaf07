"""Pins for the oracle's CRS SpMV (Fig. 2), inner product and CG (Sect. 3.4).

SpMV against a dense product; dot against exactly-rounded summation
(math.fsum); CG against a direct sparse solve, the finite-termination
property (k distinct eigenvalues -> at most k steps), a manufactured
discrete solution and its failure statuses.
"""
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle as O
from paper_1511_03703_gb300 import inputs


def test_spmv_matches_dense():
    N, M = 3, 10
    row_map, col = O.graph(N)
    vals, _ = O.assemble(N, M, inputs.kl_samples(11, 0, 1, M)[0], row_map, col)
    x = inputs.random_vector(12, len(row_map) - 1)
    D = sp.csr_matrix((vals, col, row_map)).toarray()
    z = O.spmv(row_map, col, vals, x)
    bound = 1e-15 * 30 * (np.abs(D) @ np.abs(x))
    assert np.all(np.abs(z - D @ x) <= bound)


def test_dot_within_summation_bound():
    for n in (1, 7, 1000, 100003):
        u = inputs.random_vector(21, n)
        v = inputs.random_vector(22, n, -3.0, 5.0)
        exact = math.fsum((u * v).tolist())
        gamma = n * 2.0 ** -53 / (1 - n * 2.0 ** -53)
        assert abs(O.dot(u, v) - exact) <= (gamma + 2.0 ** -53) * np.sum(np.abs(u * v))


def test_cg_finite_termination_three_eigenvalues():
    n = 50
    d = np.array([1.0, 2.0, 5.0])[np.arange(n) % 3]
    row_map = np.arange(n + 1, dtype=np.int32)
    col = np.arange(n, dtype=np.int32)
    b = inputs.random_vector(5, n)
    x, it, rr, st = O.cg(row_map, col, d, b, tol=1e-14)
    assert st == 0 and it <= 3 and np.max(np.abs(x - b / d)) < 1e-14


def test_cg_matches_direct_solve():
    N, M = 6, 10
    row_map, col = O.graph(N)
    vals, b = O.assemble(N, M, inputs.kl_samples(31, 0, 1, M)[0], row_map, col)
    x, it, rr, st = O.cg(row_map, col, vals, b, tol=1e-13)
    xd = spla.spsolve(sp.csr_matrix((vals, col, row_map)).tocsc(), b)
    assert st == 0 and rr <= 1e-12
    assert np.linalg.norm(x - xd) <= 1e-11 * np.linalg.norm(xd)


def test_cg_manufactured_solution_and_boundary_zero():
    N, M = 8, 3
    row_map, col = O.graph(N)
    vals, _ = O.assemble(N, M, inputs.kl_samples(inputs.SEED_SMALL, 0, 1, M)[0], row_map, col)
    bm = O.bmask(N)
    xs = inputs.random_vector(41, len(bm))
    xs[bm == 1] = 0.0
    b = O.spmv(row_map, col, vals, xs)
    x, it, rr, st = O.cg(row_map, col, vals, b, tol=1e-13)
    assert st == 0
    assert np.linalg.norm(x - xs) <= 1e-11 * np.linalg.norm(xs)
    assert np.all(x[bm == 1] == 0.0)


def test_cg_statuses():
    N = 4
    row_map, col = O.graph(N)
    vals, b = O.assemble(N, 3, np.zeros(3), row_map, col)
    _, it, rr, st = O.cg(row_map, col, vals, b, tol=1e-12, max_iter=2)
    assert st == 5 and it == 2 and rr > 1e-12
    x, it, rr, st = O.cg(row_map, col, vals, np.zeros_like(b), x0=np.ones_like(b))
    assert st == 0 and it == 0 and np.all(x == 0)
    # indefinite matrix -> breakdown detected on p'Ap <= 0
    n = 4
    rm = np.arange(n + 1, dtype=np.int32)
    c = np.arange(n, dtype=np.int32)
    _, it, rr, st = O.cg(rm, c, np.array([1.0, -1.0, 1.0, -1.0]), np.array([1.0, 1.0, 0.0, 0.0]))
    assert st == 6


def test_solve_samples_matches_single_calls():
    N, M = 4, 10
    xi = inputs.kl_samples(77, 0, 3, M)
    x, it, rr, st = O.solve_samples(N, M, xi, tol=1e-10, nthreads=2, want_x=True)
    row_map, col = O.graph(N)
    for j in range(3):
        vals, b = O.assemble(N, M, xi[j], row_map, col)
        xj, itj, rrj, stj = O.cg(row_map, col, vals, b, tol=1e-10)
        assert np.array_equal(x[j], xj) and it[j] == itj and st[j] == stj == 0


def test_splitmix64_published_vectors():
    # first five outputs of SplitMix64 seeded with 1234567, and the first for seed 0
    got = [int(v) for v in inputs.splitmix64(1234567, np.arange(1, 6))]
    assert got == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                   4593380528125082431, 16408922859458223821]
    assert int(inputs.splitmix64(0, 1)) == 0xE220A8397B1DCDAF
    xi = inputs.kl_samples(1001, 0, 4, 3)
    assert xi.shape == (4, 3) and np.all(np.abs(xi) <= 1.0)
    assert np.array_equal(inputs.kl_samples(1001, 2, 2, 3), xi[2:])
