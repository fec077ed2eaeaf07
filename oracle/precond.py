"""CPU oracle of the preconditioned ensemble CG (Jacobi and Chebyshev), FP64.

TEST INFRASTRUCTURE ONLY: only `tests/`, `__graft_entry__.smoke()` and the
benchmark's CPU-baseline leg may import this module.  It shares no code with
the CUDA library; the SpMV is the C oracle's (Fig. 2 row loop).

The paper's solver is CG preconditioned by multigrid whose smoothers are
order-2 Chebyshev polynomials (Sect. 3.5); this module states the two
SpMV-based preconditioners used on their own, per sample, in textbook form:

  D         the diagonal of A; Jacobi:  z = D^-1 r.
  lam_max   estimate of the largest eigenvalue of D^-1 A: from a given start
            vector v_0, v_{k+1} = D^-1 A v_k / ||D^-1 A v_k||, and after
            `iters` steps the generalized Rayleigh quotient
            (v.A v) / (v.D v) of the last vector.
  lam_max_lanczos
            the same bound from `steps` Lanczos steps on D^-1 A, which is
            self-adjoint in the D inner product <x, y> = x.D y (Lanczos 1950;
            Saad, Iterative Methods, Sect. 6.6): q_1 = v_0 / ||v_0||_D,
            beta_0 = 0, and for j = 1 .. steps
              y = A q_j,  alpha_j = q_j.y,
              u = D^-1 y - alpha_j q_j - beta_{j-1} q_{j-1},
              beta_j = ||u||_D,  q_{j+1} = u / beta_j (0 when beta_j = 0);
            the estimate is the largest eigenvalue of the tridiagonal T with
            diagonal alpha_1..alpha_steps and off-diagonal beta_1..beta_{steps-1}
            (a Ritz value: a lower bound that no power estimate from the same
            start with fewer matrix products exceeds).
  Chebyshev z = p(D^-1 A) D^-1 r: `degree` steps of Chebyshev iteration for
            A z = r from z = 0 on the interval [lam_max / ratio, lam_max]
            (theta = centre, delta = half width, sigma = theta / delta):
              rho_0 = 1 / sigma,  d_0 = D^-1 r / theta,  z = d_0
              rho_k = 1 / (2 sigma - rho_{k-1}),
              d_k = rho_k rho_{k-1} d_{k-1} + (2 rho_k / delta) D^-1 (r - A z),
              z  += d_k                                  (k = 1 .. degree-1)
            (Saad, Iterative Methods for Sparse Linear Systems, Sect. 12.3).
  PCG       Hestenes-Stiefel with z = M^-1 r: alpha = (r.z) / (p.Ap),
            beta = (r.z)_new / (r.z)_old, p = z + beta p; stop when
            ||r|| <= tol ||b|| (recursive residual), as the plain CG.

Pins: tests/test_oracle_precond.py.
"""
import numpy as np

import oracle as O


def diagonal(row_map, col, values):
    n = len(row_map) - 1
    rows = np.repeat(np.arange(n), np.diff(row_map))
    d = np.zeros(n)
    sel = np.asarray(col) == rows
    d[rows[sel]] = np.asarray(values)[sel]
    return d


def lam_max(row_map, col, values, v0, iters):
    """Power-iteration estimate of the largest eigenvalue of D^-1 A."""
    d = diagonal(row_map, col, values)
    v = np.asarray(v0, dtype=np.float64).copy()
    for _ in range(iters):
        y = O.spmv(row_map, col, values, v) / d
        v = y / np.linalg.norm(y)
    av = O.spmv(row_map, col, values, v)
    return float(np.dot(v, av) / np.dot(v, d * v))


def lam_max_lanczos(row_map, col, values, v0, steps):
    """Lanczos estimate of the largest eigenvalue of D^-1 A (largest Ritz value)."""
    d = diagonal(row_map, col, values)
    v = np.asarray(v0, dtype=np.float64)
    q = v / np.sqrt(np.dot(v, d * v))
    q_prev = np.zeros_like(q)
    beta = 0.0
    alphas, betas = [], []
    for _ in range(steps):
        y = O.spmv(row_map, col, values, q)
        alpha = float(np.dot(q, y))
        u = y / d - alpha * q - beta * q_prev
        beta = float(np.sqrt(np.dot(u, d * u)))
        alphas.append(alpha)
        betas.append(beta)
        q_prev, q = q, (u / beta if beta > 0.0 else np.zeros_like(u))
    T = np.diag(alphas) + np.diag(betas[:-1], 1) + np.diag(betas[:-1], -1)
    return float(np.linalg.eigvalsh(T)[-1])


def chebyshev(row_map, col, values, r, lmax, ratio, degree):
    """z = p(D^-1 A) D^-1 r by `degree` Chebyshev steps from z = 0."""
    d = diagonal(row_map, col, values)
    lmin = lmax / ratio
    theta, delta = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    sigma = theta / delta
    rho = 1.0 / sigma
    dk = r / d / theta
    z = dk.copy()
    for _ in range(1, degree):
        rho_new = 1.0 / (2.0 * sigma - rho)
        res = r - O.spmv(row_map, col, values, z)
        dk = rho_new * rho * dk + (2.0 * rho_new / delta) * (res / d)
        z = z + dk
        rho = rho_new
    return z


def pcg(row_map, col, values, b, precond, tol=1e-10, max_iter=10000, x0=None):
    """Returns (x, iters, relres_true, status); precond(r) -> z."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    r = b - O.spmv(row_map, col, values, x)
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return np.zeros_like(b), 0, 0.0, O.STATUS_OK
    z = precond(r)
    p = z.copy()
    rz = float(np.dot(r, z))
    it, status = 0, O.STATUS_OK
    while np.linalg.norm(r) > tol * bn:
        if it >= max_iter:
            status = O.STATUS_NOT_CONVERGED
            break
        q = O.spmv(row_map, col, values, p)
        pq = float(np.dot(p, q))
        if not (pq > 0.0) or not np.isfinite(pq):
            status = O.STATUS_BREAKDOWN
            break
        alpha = rz / pq
        x += alpha * p
        r -= alpha * q
        it += 1
        if np.linalg.norm(r) <= tol * bn:
            break
        z = precond(r)
        rz_new = float(np.dot(r, z))
        p = z + (rz_new / rz) * p
        rz = rz_new
    rel = np.linalg.norm(b - O.spmv(row_map, col, values, x)) / bn
    return x, it, float(rel), status
