"""CPU oracle of the multigrid-preconditioned CG, FP64, per sample.

TEST INFRASTRUCTURE ONLY: only `tests/`, `__graft_entry__.smoke()` and the
benchmark's CPU-baseline leg may import this module.  It shares no code with
the CUDA library.

The paper's solver (Sect. 3.5, Algorithm 1) is CG preconditioned by a
multigrid V-cycle with order-2 Chebyshev smoothers and a direct coarse solve.
This oracle states the geometric version on the nested hex meshes:

  levels    N_0 = N, N_{l+1} = N_l / 2 while N_l is even and N_l > 4; each level
            is assembled from the same KL coefficient on its own mesh
            (rediscretisation, Dirichlet rows by symmetric elimination).
  P_l       trilinear interpolation from the interior nodes of level l+1 to
            the interior nodes of level l: along each axis a fine index 2i
            takes coarse i with weight 1, a fine index 2i+1 takes coarse i and
            i+1 with weight 1/2 each; coarse boundary nodes (value 0) and fine
            boundary nodes are left out.  R_l = P_l^T.
  smoother  S(b, x) = x + p(D^-1 A) D^-1 (b - A x), p the Chebyshev polynomial
            of `degree` steps on [lam/ratio, lam], lam = boost x the power
            estimate of the largest eigenvalue of D^-1 A (oracle.precond), or
            with lanczos=True its Lanczos estimate from as many steps;
            ratio 5 by default: a smoother only has to damp the upper part
            of the spectrum, which factor-2 coarsening cannot represent.
  V-cycle   V_L(b) = A_L^-1 b (dense solve);
            V_l(b): x = S(b, 0); r = b - A x; x += P V_{l+1}(R r); x = S(b, x).
  PCG       oracle.precond.pcg with z = V_0(r).

Pins: tests/test_oracle_multigrid.py.
"""
import functools

import numpy as np
import scipy.sparse as sp

import oracle as O
from oracle import precond as P


def level_sizes(N):
    out = [N]
    while out[-1] % 2 == 0 and out[-1] > 4:
        out.append(out[-1] // 2)
    return out


@functools.lru_cache(maxsize=16)
def prolongation(Nc):
    """Sparse P: interior nodes of the (2 Nc)^3-cell mesh <- interior nodes of the
    Nc^3 mesh.  A pure function of Nc, built once per size (the cache only saves
    the Python loops; callers do not modify the matrix)."""
    Nf = 2 * Nc
    nf1, nc1 = Nf + 1, Nc + 1
    rows, cols, vals = [], [], []
    for k in range(1, Nf):
        for j in range(1, Nf):
            for i in range(1, Nf):
                I = i + nf1 * (j + nf1 * k)
                for ci, wi in _parents(i, Nc):
                    for cj, wj in _parents(j, Nc):
                        for ck, wk in _parents(k, Nc):
                            rows.append(I)
                            cols.append(ci + nc1 * (cj + nc1 * ck))
                            vals.append(wi * wj * wk)
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf1 ** 3, nc1 ** 3))


def _parents(i, Nc):
    """Interior coarse indices (and weights) that a fine index i interpolates from."""
    if i % 2 == 0:
        cand = [(i // 2, 1.0)]
    else:
        cand = [((i - 1) // 2, 0.5), ((i + 1) // 2, 0.5)]
    return [(c, w) for c, w in cand if 0 < c < Nc]


class Level:
    def __init__(self, N, M, xi, v0, power_iters, boost, ratio, sigma=0.1, kappa0=1.0, L=1.0, lanczos=False):
        self.N = N
        self.rm, self.col = O.graph(N)
        self.vals, self.load = O.assemble(N, M, xi, self.rm, self.col, L=L, sigma=sigma, kappa0=kappa0)
        self.d = P.diagonal(self.rm, self.col, self.vals)
        if lanczos:   # power_iters Lanczos steps instead of power steps
            self.lam = P.lam_max_lanczos(self.rm, self.col, self.vals, v0, power_iters)
        else:
            self.lam = P.lam_max(self.rm, self.col, self.vals, v0, power_iters)
        self.lmax = boost * self.lam
        self.ratio = ratio

    def A(self, x):
        return O.spmv(self.rm, self.col, self.vals, x)

    def dense(self):
        return sp.csr_matrix((self.vals, self.col, self.rm)).toarray()


def hierarchy(N, M, xi, starts, power_iters=10, boost=1.1, ratio=5.0, **kw):
    """Levels for one sample; starts[l] = start vector of level l's eigenvalue
    estimate (power iteration, or Lanczos with lanczos=True)."""
    return [Level(n, M, xi, starts[l], power_iters, boost, ratio, **kw) for l, n in enumerate(level_sizes(N))]


def smooth(lev, b, x, degree):
    r = b - lev.A(x)
    return x + P.chebyshev(lev.rm, lev.col, lev.vals, r, lev.lmax, lev.ratio, degree)


def vcycle(levels, b, degree=2, l=0):
    lev = levels[l]
    if l == len(levels) - 1:
        return np.linalg.solve(lev.dense(), b)
    Pm = prolongation(levels[l + 1].N)
    x = smooth(lev, b, np.zeros_like(b), degree)
    r = b - lev.A(x)
    xc = vcycle(levels, Pm.T @ r, degree, l + 1)
    x = x + Pm @ xc
    return smooth(lev, b, x, degree)


def mg_pcg(levels, b, tol=1e-10, max_iter=1000, degree=2):
    lev = levels[0]
    return P.pcg(lev.rm, lev.col, lev.vals, b, lambda r: vcycle(levels, r, degree), tol=tol, max_iter=max_iter)
