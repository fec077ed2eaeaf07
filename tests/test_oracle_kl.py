"""Pins for the oracle's Karhunen-Loeve expansion (Sect. 4, Eq. 9-10).

The paper states only the covariance C(x,x') = sigma^2 exp(-|x-x'|_1 / L) on
[0,1]^3 and that its eigenfunctions are tensor products of sines and cosines.
These tests check the oracle's eigenpairs against the integral equation
itself (evaluated by quadrature split at the kink), orthonormality, the trace
identity, an independent Nystrom discretisation, and the mode ordering rule.
"""
import numpy as np
import pytest

import oracle as O


def gl01(n, a=0.0, b=1.0):
    x, w = np.polynomial.legendre.leggauss(n)
    return a + (b - a) * (x + 1) / 2, w * (b - a) / 2


@pytest.mark.parametrize("L", [1.0, 0.5])
def test_kl_1d_integral_equation(L):
    om, lam = O.kl_1d(8, L)
    for p in range(8):
        for x in (0.0, 0.13, 0.5, 0.77, 1.0):
            s = 0.0
            for a, b in ((0.0, x), (x, 1.0)):
                if b > a:
                    t, w = gl01(40, a, b)
                    s += np.sum(w * np.exp(-np.abs(x - t) / L) * O.kl_phi1d(p, om[p], t, L))
            assert abs(s - lam[p] * O.kl_phi1d(p, om[p], [x], L)[0]) < 1e-13, (p, x)


def test_kl_1d_orthonormal_and_ordered():
    om, lam = O.kl_1d(12)
    t, w = gl01(80)
    phi = np.array([O.kl_phi1d(p, om[p], t) for p in range(12)])
    G = (phi * w) @ phi.T
    assert np.max(np.abs(G - np.eye(12))) < 1e-13
    assert np.all(np.diff(lam) < 0) and np.all(lam > 0)
    # alternating parity about x = 1/2: even p symmetric, odd p antisymmetric
    for p in range(12):
        f = O.kl_phi1d(p, om[p], [0.2, 0.8])
        assert abs(f[0] - (1 if p % 2 == 0 else -1) * f[1]) < 1e-14


def test_kl_1d_trace_identity():
    # sum of all eigenvalues = int_0^1 C(x,x) dx = 1; tail ~ sum 2c/omega^2
    om, lam = O.kl_1d(4000)
    s = lam.sum()
    assert s < 1.0 and 1.0 - s < 2.0 / (np.pi ** 2 * 4000) * 1.2


def test_kl_1d_against_nystrom():
    n = 1500
    t, w = gl01(n)
    K = np.exp(-np.abs(t[:, None] - t[None, :]))
    sw = np.sqrt(w)
    ev = np.linalg.eigvalsh(sw[:, None] * K * sw[None, :])[::-1]
    _, lam = O.kl_1d(5)
    assert np.max(np.abs(ev[:5] - lam) / lam) < 1e-5


def test_kl_mode_order_M3_M10():
    pqr3, lam3 = O.kl_modes(3)
    assert pqr3.tolist() == [[0, 0, 0], [0, 0, 1], [0, 1, 0]]
    pqr, lam = O.kl_modes(10)
    assert pqr.tolist() == [[0, 0, 0], [0, 0, 1], [0, 1, 0], [1, 0, 0], [0, 0, 2],
                            [0, 2, 0], [2, 0, 0], [0, 1, 1], [1, 0, 1], [1, 1, 0]]
    # tie groups are exact ties, groups strictly decreasing
    assert lam[1] == lam[2] == lam[3] and lam[4] == lam[5] == lam[6] and lam[7] == lam[8] == lam[9]
    assert lam[0] > lam[1] > lam[4] > lam[7]
    _, l1 = O.kl_1d(4)
    assert abs(lam[0] - l1[0] ** 3) < 1e-16 and abs(lam[7] - l1[0] * l1[1] ** 2) < 1e-16
    # the 11th mode, (0,0,3), is strictly smaller: M = 10 ends on a whole tie group
    pqr11, lam11 = O.kl_modes(11)
    assert pqr11[10].tolist() == [0, 0, 3] and lam11[10] < lam[9]


def kappa_mode(k, M, x):
    xi = np.zeros(M)
    xi[k] = 1.0
    return O.kl_coeff_at(M, xi, np.asarray(x, float), sigma=1.0, kappa0=0.0)


def test_kl_3d_integral_equation_and_axes():
    M = 10
    _, lam = O.kl_modes(M)
    x = np.array([0.31, 0.62, 0.17])
    n = 8
    for k in (0, 1, 3, 7, 9):
        tot = 0.0
        segs = [((0.0, x[d]), (x[d], 1.0)) for d in range(3)]
        for sx in segs[0]:
            tx, wx = gl01(n, *sx)
            for sy in segs[1]:
                ty, wy = gl01(n, *sy)
                for sz in segs[2]:
                    tz, wz = gl01(n, *sz)
                    for a in range(n):
                        for b in range(n):
                            for c in range(n):
                                t = (tx[a], ty[b], tz[c])
                                C = np.exp(-(abs(x[0] - t[0]) + abs(x[1] - t[1]) + abs(x[2] - t[2])))
                                tot += wx[a] * wy[b] * wz[c] * C * kappa_mode(k, M, t)
        # kappa_k = sqrt(lambda_k) phi_k is an eigenfunction with eigenvalue lambda_k
        assert abs(tot - lam[k] * kappa_mode(k, M, x)) < 1e-9 * max(1.0, abs(tot)), k
    # axis convention: mode 1 = (0,0,1) is odd in z and even in x; mode 3 = (1,0,0) odd in x
    p = np.array([0.2, 0.3, 0.4])
    assert abs(kappa_mode(1, M, p) + kappa_mode(1, M, [0.2, 0.3, 0.6])) < 1e-14
    assert abs(kappa_mode(1, M, p) - kappa_mode(1, M, [0.8, 0.3, 0.4])) < 1e-14
    assert abs(kappa_mode(3, M, p) + kappa_mode(3, M, [0.8, 0.3, 0.4])) < 1e-14


def test_kl_3d_orthogonality():
    M = 10
    _, lam = O.kl_modes(M)
    t, w = gl01(14)
    pts = [(a, b, c) for a in range(14) for b in range(14) for c in range(14)]
    F = np.array([[kappa_mode(k, M, (t[a], t[b], t[c])) for (a, b, c) in pts] for k in range(M)])
    W = np.array([w[a] * w[b] * w[c] for (a, b, c) in pts])
    G = (F * W) @ F.T
    assert np.max(np.abs(G - np.diag(lam))) < 1e-12


def test_kl_coefficient_at_quadrature_points():
    N, M = 4, 10
    xi = np.linspace(-0.9, 0.8, M)
    a = O.kl_coeff_qp(N, M, xi)
    g = [0.5 - 0.5 / np.sqrt(3), 0.5 + 0.5 / np.sqrt(3)]
    h = 1.0 / N
    for (ci, cj, ck) in [(0, 0, 0), (3, 1, 2), (1, 3, 3)]:
        c = ci + N * (cj + N * ck)
        for q in range(8):
            x = [(ci + g[q & 1]) * h, (cj + g[(q >> 1) & 1]) * h, (ck + g[(q >> 2) & 1]) * h]
            assert abs(a[c, q] - O.kl_coeff_at(M, xi, x)) < 1e-15
    # mean and bounds: kappa0 = 1, sigma = 0.1; |xi| <= 1 keeps a well inside (0.5, 1.5)
    assert 0.5 < a.min() and a.max() < 1.5
    assert np.all(O.kl_coeff_qp(N, M, np.zeros(M)) == 1.0)
