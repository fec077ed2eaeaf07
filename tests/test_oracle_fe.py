"""Pins for the oracle's finite-element assembly (Algorithm 2, Sect. 4).

Trilinear (Q1) hex elements with 8 Gauss points; -div(a grad u) = 1 on the unit
cube with u = 0 on the boundary (symmetric elimination).  Checked against
closed forms (constant coefficient), a dense brute-force assembly written
independently here (gradients by exact central differences), bitwise
symmetry, positive definiteness and the PDE's own Fourier-series solution.
"""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from helpers import leading_mode_threshold


def dense(row_map, col, vals):
    n = len(row_map) - 1
    return sp.csr_matrix((vals, col, row_map), shape=(n, n)).toarray()


def test_element_matrix_constant_closed_form():
    for h in (1.0, 0.125, 1.0 / 64):
        K = O.element_matrix(h, np.ones(8))
        for a, b in itertools.product(range(8), repeat=2):
            ham = bin(a ^ b).count("1")
            expect = h * {0: 1 / 3, 1: 0.0, 2: -1 / 12, 3: -1 / 12}[ham]
            assert abs(K[a, b] - expect) < 1e-15 * max(h, 1e-300) * 10
        assert np.allclose(O.element_load(h), h ** 3 / 8, rtol=1e-15, atol=0)


def ref_basis(l, x):
    return np.prod([x[d] if (l >> d) & 1 else 1 - x[d] for d in range(3)])


def brute_element(h, a_q):
    """K_e from exact central differences of the trilinear basis (independent route)."""
    g = [0.5 - 0.5 / np.sqrt(3), 0.5 + 0.5 / np.sqrt(3)]
    K = np.zeros((8, 8))
    for q in range(8):
        x = np.array([g[q & 1], g[(q >> 1) & 1], g[(q >> 2) & 1]])
        B = np.zeros((8, 3))
        for l in range(8):
            for d in range(3):
                e = np.zeros(3)
                e[d] = 0.25
                B[l, d] = (ref_basis(l, x + e) - ref_basis(l, x - e)) / 0.5 / h
        K += a_q[q] * (h ** 3 / 8) * B @ B.T
    return K


def test_element_matrix_general_coefficient():
    rng = np.random.default_rng(7)
    for _ in range(5):
        a_q = rng.uniform(0.5, 1.5, 8)
        h = 1.0 / rng.integers(1, 100)
        K = O.element_matrix(h, a_q)
        assert np.array_equal(K, K.T)
        assert np.max(np.abs(K - brute_element(h, a_q))) < 1e-14 * h * 10
        assert np.max(np.abs(K.sum(axis=1))) < 1e-15 * h * 10   # constants in the kernel


@pytest.mark.parametrize("N", [2, 3])
def test_assembly_dense_brute_force(N):
    M = 10
    xi = np.array([0.7, -0.4, 0.9, -1.0, 0.2, 0.55, -0.35, 0.05, 0.8, -0.6])
    row_map, col = O.graph(N)
    vals, b = O.assemble(N, M, xi, row_map, col)
    h = 1.0 / N
    a_qp = O.kl_coeff_qp(N, M, xi)
    n = (N + 1) ** 3
    A = np.zeros((n, n))
    f = np.zeros(n)
    for ck, cj, ci in itertools.product(range(N), repeat=3):
        c = ci + N * (cj + N * ck)
        nodes = [(ci + (l & 1)) + (N + 1) * ((cj + ((l >> 1) & 1)) + (N + 1) * (ck + ((l >> 2) & 1)))
                 for l in range(8)]
        A[np.ix_(nodes, nodes)] += brute_element(h, a_qp[c])
        f[nodes] += h ** 3 / 8
    bnd = np.array([min(i, j, k) == 0 or max(i, j, k) == N
                    for k in range(N + 1) for j in range(N + 1) for i in range(N + 1)])
    A[bnd, :] = 0
    A[:, bnd] = 0
    A[bnd, bnd] = 1
    f[bnd] = 0
    D = dense(row_map, col, vals)
    assert np.max(np.abs(D - A)) < 1e-15 * 20
    assert np.max(np.abs(b - f)) < 1e-14 * h ** 3
    # the stored pattern covers all non-zeros and nothing else is touched
    pattern = dense(row_map, col, np.ones_like(vals)) > 0
    assert not np.any(A[~pattern])


@pytest.mark.parametrize("N", [2, 4, 8])
def test_assembly_constant_coefficient_stencil(N):
    row_map, col = O.graph(N)
    vals, b = O.assemble(N, 3, np.array([1.0, -1.0, 0.5]), row_map, col, sigma=0.0)
    h = 1.0 / N
    bm = O.bmask(N)
    coords = np.array([(i, j, k) for k in range(N + 1) for j in range(N + 1) for i in range(N + 1)])
    for I in range(len(bm)):
        for e in range(row_map[I], row_map[I + 1]):
            J = col[e]
            if bm[I]:
                expect = 1.0 if I == J else 0.0
            elif bm[J]:
                expect = 0.0
            else:
                ham = int(np.sum(coords[I] != coords[J]))
                expect = h * {0: 8 / 3, 1: 0.0, 2: -1 / 6, 3: -1 / 12}[ham]
            assert abs(vals[e] - expect) < 1e-14 * h, (I, J)
        assert (b[I] == 0.0) if bm[I] else abs(b[I] - h ** 3) < 1e-15 * h ** 3


def test_assembly_bitwise_symmetric_and_spd():
    N, M = 4, 10
    xi = np.linspace(-1, 1, M)
    row_map, col = O.graph(N)
    vals, _ = O.assemble(N, M, xi, row_map, col)
    D = dense(row_map, col, vals)
    assert np.array_equal(D, D.T)
    np.linalg.cholesky(D)  # raises if not SPD


def centre_value_series(terms=2001):
    l = np.arange(1, terms + 1, 2, dtype=np.float64)
    sg = np.where(((l - 1) / 2) % 2 == 0, 1.0, -1.0)
    tot = 0.0
    for i, li in enumerate(l):
        k = np.pi * np.sqrt(li ** 2 + l ** 2)
        with np.errstate(over="ignore"):
            w = (1 - 1 / np.cosh(k / 2)) / k ** 2
        tot += np.sum(16 / (np.pi ** 2 * li * l) * sg[i] * sg * w)
    return tot


def test_pde_centre_value_converges_second_order():
    # -Laplace u = 1, u = 0 on the boundary: double sine series in (x, y) with
    # the exact 1D solve in z gives u(1/2,1/2,1/2) = 0.0562128...
    exact = centre_value_series()
    assert abs(exact - 0.0562128298) < 1e-9
    errs = []
    for N in (8, 16, 32):
        row_map, col = O.graph(N)
        vals, b = O.assemble(N, 3, np.zeros(3), row_map, col, sigma=0.0)
        x, it, rr, st = O.cg(row_map, col, vals, b, tol=1e-12)
        assert st == 0 and rr < 1e-11
        c = N // 2
        errs.append(abs(x[c + (N + 1) * (c + (N + 1) * c)] - exact))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.7 < r2 < 4.3, errs


@pytest.mark.parametrize("N", [3, 4, 7])
def test_assembly_reports_a_nonpositive_coefficient_at_the_closed_form_threshold(N):
    """Sect. 4's coefficient must be positive for an elliptic problem: the
    oracle's assembly reports a(x_q) <= 0 exactly past the threshold the
    closed-form leading mode gives, and a positive mode never trips it."""
    rm, col = O.graph(N)
    sstar = leading_mode_threshold(N)
    O.assemble(N, 1, [-1.0], rm, col, sigma=sstar * (1 - 1e-9))
    assert O.coeff_min(N, 1, [-1.0], sigma=sstar * (1 - 1e-9)) > 0
    with pytest.raises(O.NonPositiveCoefficient):
        O.assemble(N, 1, [-1.0], rm, col, sigma=sstar * (1 + 1e-9))
    assert O.coeff_min(N, 1, [-1.0], sigma=sstar * (1 + 1e-9)) < 0
    O.assemble(N, 1, [1.0], rm, col, sigma=50 * sstar)          # kappa_1 > 0: a > kappa0
    with pytest.raises(O.NonPositiveCoefficient):
        O.assemble(N, 1, [1.0], rm, col, sigma=float("nan"))   # NaN is not positive
    # unchecked: the values are still those of the assembly
    v, b = O.assemble(N, 1, [-1.0], rm, col, sigma=2 * sstar, check=False)
    assert np.all(np.isfinite(v)) and np.all(np.isfinite(b))


def test_workload_coefficient_stays_positive():
    """The workloads' KL variables lie in [-1, 1] with sigma = 0.1 and M = 10:
    the coefficient stays well above zero (about 0.7 at worst)."""
    from paper_1511_03703_gb300 import inputs
    xs = inputs.kl_samples(1002, 0, 64, 10)
    amin = min(O.coeff_min(8, 10, x) for x in xs)
    assert 0.5 < amin < 1.0
    # the same draws with sigma large enough make the problem indefinite
    assert min(O.coeff_min(8, 10, x, sigma=2.0) for x in xs) < 0
