"""CPU oracle of the nonlinear advection-diffusion problem, FP64, per sample.

TEST INFRASTRUCTURE ONLY: only `tests/`, `__graft_entry__.smoke()` and the
benchmark's CPU-baseline leg may import this module.  It shares no code with
the CUDA library.

The paper's model problem (Sect. 4, Eq. 7) adds an advection term
alpha v.grad(u) and a reaction term beta u^2 to the KL diffusion operator; its
experiments set alpha = beta = 0, where one Newton step (Eq. 10) is the linear
solve.  For alpha, beta != 0 this oracle states, on the Q1 hex mesh of the
linear problem (source 1, u = 0 on the boundary):

  F_i(u) = (A u)_i + alpha int phi_i v.grad(u_h) + beta int phi_i u_h^2 - b_i
                                                       (interior node i)
  F_i(u) = u_i                                         (boundary node i)
  J(u)   = dF/du = A + alpha C + 2 beta M(u),
           C_ij = int phi_i v.grad(phi_j),  M(u)_ij = int phi_i phi_j u_h,
           boundary rows of J: identity; boundary columns of interior rows: 0
with A, b the diffusion matrix and load of the linear problem (oracle.assemble).
Every integral uses the 2x2x2 Gauss rule, which is exact here: each integrand
has degree <= 3 in each coordinate.  v is a constant velocity.

  Newton (Eq. 10): u <- u + du with J(u) du = -F(u), from u = 0, until
      ||F(u)|| <= tol ||F(0)|| (= tol ||b||).
  GMRES: restarted GMRES(m) with right preconditioning (Saad, Iterative
      Methods for Sparse Linear Systems, Sect. 6.5 and 9.3.2): Arnoldi by
      modified Gram-Schmidt, Givens rotations, stop when the residual
      estimate |g_{j+1}| <= lin_tol ||r_0||.  Preconditioner: none, or the
      multigrid V-cycle of the diffusion operator A of the same sample
      (oracle.multigrid), fixed through all Newton steps.

Pins: tests/test_oracle_nonlinear.py.
"""
import numpy as np

import oracle as O

STATUS_OK, STATUS_NOT_CONVERGED = 0, 5

_G1 = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])  # Gauss points on [0, 1]


def _reference_tables():
    """phi[q, a] and ref_grad[q, a, d] of the trilinear basis at the 8 Gauss
    points; node a has offsets (a & 1, a >> 1 & 1, a >> 2 & 1), point q the
    same bit layout over the two 1-D Gauss points."""
    phi = np.empty((8, 8))
    grad = np.empty((8, 8, 3))
    for q in range(8):
        xq = [_G1[(q >> d) & 1] for d in range(3)]
        for a in range(8):
            o = [(a >> d) & 1 for d in range(3)]
            L = [xq[d] if o[d] else 1.0 - xq[d] for d in range(3)]
            dL = [1.0 if o[d] else -1.0 for d in range(3)]
            phi[q, a] = L[0] * L[1] * L[2]
            grad[q, a] = (dL[0] * L[1] * L[2], L[0] * dL[1] * L[2], L[0] * L[1] * dL[2])
    return phi, grad


PHI, GRAD = _reference_tables()


class Mesh:
    """Graph, element maps and boundary mask of the N^3-cell mesh."""

    def __init__(self, N):
        self.N = N
        self.h = 1.0 / N
        self.rm, self.col = O.graph(N)
        self.ni = O.node_index(N)                                   # (cells, 8)
        self.eg = O.elem_graph(N, self.rm, self.col).reshape(-1, 64)  # (cells, 64)
        self.bm = O.bmask(N).astype(bool)
        self.n = len(self.rm) - 1
        self.row = np.repeat(np.arange(self.n), np.diff(self.rm))   # row of each entry

    def eliminate(self, vals):
        """Dirichlet rows and columns of an operator term set to 0."""
        out = vals.copy()
        out[self.bm[self.row] | self.bm[self.col]] = 0.0
        return out

    def scatter_matrix(self, Ke):
        """values[nnz] = sum over cells of the element matrices Ke (cells or 1, 8, 8)."""
        vals = np.zeros(len(self.col))
        Ke = np.broadcast_to(Ke.reshape(-1, 64), self.eg.shape)
        np.add.at(vals, self.eg, Ke)
        return vals

    def scatter_vector(self, fe):
        out = np.zeros(self.n)
        np.add.at(out, self.ni, fe)
        return out


def advection_element(h, v):
    """Ce[a, b] = int_cell phi_a v.grad(phi_b) = (h^3 / 8) sum_q phi_a(q) v.grad_b(q) / h."""
    vg = GRAD @ np.asarray(v, float)                                # (q, b)
    return (h * h / 8.0) * np.einsum("qa,qb->ab", PHI, vg)


def advection_values(mesh, v):
    """C on the mesh graph, boundary rows and columns 0."""
    return mesh.eliminate(mesh.scatter_matrix(advection_element(mesh.h, v)[None]))


def _u_at_points(mesh, u):
    ue = u[mesh.ni]                                                 # (cells, 8)
    return ue, ue @ PHI.T                                           # (cells, q)


def mass_u_values(mesh, u):
    """M(u)_ij = int phi_i phi_j u_h, boundary rows and columns 0."""
    _, uq = _u_at_points(mesh, u)
    Me = (mesh.h ** 3 / 8.0) * np.einsum("qa,qb,cq->cab", PHI, PHI, uq)
    return mesh.eliminate(mesh.scatter_matrix(Me))


def quadratic_term(mesh, u):
    """q_i(u) = int phi_i u_h^2 on every node (no boundary rule)."""
    _, uq = _u_at_points(mesh, u)
    return mesh.scatter_vector((mesh.h ** 3 / 8.0) * (uq * uq) @ PHI)


def advection_term(mesh, u, v):
    """a_i(u) = int phi_i v.grad(u_h) on every node (no boundary rule)."""
    ue, _ = _u_at_points(mesh, u)
    vg = GRAD @ np.asarray(v, float)                                # (q, b)
    dudv = ue @ vg.T / mesh.h                                       # (cells, q): v.grad u_h
    return mesh.scatter_vector((mesh.h ** 3 / 8.0) * dudv @ PHI)


class Problem:
    """One sample: A, b of the diffusion problem plus the nonlinear terms."""

    def __init__(self, N, M, xi, alpha, beta, v=(1.0, 1.0, 1.0), sigma=0.1, kappa0=1.0, L=1.0):
        self.mesh = Mesh(N)
        self.N, self.M, self.xi = N, M, np.asarray(xi, float)
        self.alpha, self.beta, self.v = float(alpha), float(beta), tuple(float(t) for t in v)
        self.A, self.b = O.assemble(N, M, self.xi, self.mesh.rm, self.mesh.col, L=L, sigma=sigma,
                                    kappa0=kappa0)
        self.C = advection_values(self.mesh, self.v)
        self.interior = ~self.mesh.bm

    def residual(self, u):
        m = self.mesh
        nl = self.alpha * advection_term(m, u, self.v) + self.beta * quadratic_term(m, u)
        return O.spmv(m.rm, m.col, self.A, u) + np.where(self.interior, nl, 0.0) - self.b

    def jacobian(self, u):
        return self.A + self.alpha * self.C + 2.0 * self.beta * mass_u_values(self.mesh, u)


def givens(a, b):
    """(c, s) with c a + s b = sqrt(a^2 + b^2), -s a + c b = 0."""
    t = np.hypot(a, b)
    if t == 0.0:
        return 1.0, 0.0
    return a / t, b / t


def gmres(rm, col, vals, b, precond=None, restart=30, tol=1e-10, max_iter=1000):
    """Right-preconditioned restarted GMRES from x = 0.

    Returns (x, iterations, true relative residual, status)."""
    Ax = lambda x: O.spmv(rm, col, vals, x)
    Mi = precond if precond is not None else (lambda r: r.copy())
    x = np.zeros_like(b)
    beta0 = np.linalg.norm(b)
    if beta0 == 0.0:
        return x, 0, 0.0, STATUS_OK
    target = tol * beta0
    r = b.copy()
    its = 0
    done = False
    while not done and its < max_iter:
        beta = np.linalg.norm(r)
        m = restart
        V = [r / beta]
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        k = 0
        for j in range(m):
            w = Ax(Mi(V[j]))
            for i in range(j + 1):                       # modified Gram-Schmidt
                H[i, j] = np.dot(V[i], w)
                w = w - H[i, j] * V[i]
            hn = np.linalg.norm(w)
            H[j + 1, j] = hn
            for i in range(j):                           # earlier rotations
                a0, a1 = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * a0 + sn[i] * a1
                H[i + 1, j] = -sn[i] * a0 + cs[i] * a1
            cs[j], sn[j] = givens(H[j, j], H[j + 1, j])
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            k = j + 1
            if abs(g[j + 1]) <= target or hn == 0.0:
                done = True
                break
            if its >= max_iter:
                break
            V.append(w / hn)
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):                   # back substitution H y = g
            y[i] = (g[i] - np.dot(H[i, i + 1:k], y[i + 1:k])) / H[i, i]
        t = np.zeros_like(b)
        for i in range(k):
            t += y[i] * V[i]
        x = x + Mi(t)
        r = b - Ax(x)
    rel = np.linalg.norm(b - Ax(x)) / beta0
    return x, its, rel, STATUS_OK if done else STATUS_NOT_CONVERGED


def newton(prob, tol=1e-8, max_newton=20, lin_tol=1e-10, restart=30, max_lin=1000, precond=None):
    """Newton's method from u = 0.  Returns (u, newton iterations, GMRES
    iterations per step, ||F|| history, status)."""
    m = prob.mesh
    u = np.zeros(m.n)
    F = prob.residual(u)
    f0 = np.linalg.norm(F)
    hist = [f0]
    lin = []
    for k in range(max_newton + 1):
        if hist[-1] <= tol * f0:
            return u, k, lin, hist, STATUS_OK
        if k == max_newton:
            break
        du, it, _, st = gmres(m.rm, m.col, prob.jacobian(u), -F, precond, restart, lin_tol, max_lin)
        lin.append(it)
        u = u + du
        F = prob.residual(u)
        hist.append(np.linalg.norm(F))
    return u, max_newton, lin, hist, STATUS_NOT_CONVERGED
