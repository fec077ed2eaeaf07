"""Pins for the multigrid oracle (hierarchy, transfers, V-cycle, MG-PCG).

The prolongation against an independent cell-by-cell trilinear interpolant;
R A_f P against the rediscretised coarse matrix, which the Galerkin property
of nested Q1 spaces makes exact for a constant coefficient (2x2x2 Gauss
integrates the Q1 stiffness exactly); the V-cycle operator symmetric and
positive definite; MG-PCG against a direct solve, with a small iteration
count independent of the mesh size.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle as O
from oracle import multigrid as G
from paper_1511_03703_gb300 import inputs


def test_level_sizes():
    assert G.level_sizes(64) == [64, 32, 16, 8, 4]
    assert G.level_sizes(12) == [12, 6, 3]
    assert G.level_sizes(8) == [8, 4]
    assert G.level_sizes(5) == [5]


def interior_mask(N):
    n1 = N + 1
    idx = np.arange(n1)
    i, j, k = np.meshgrid(idx, idx, idx, indexing="ij")
    inside = (i > 0) & (i < N) & (j > 0) & (j < N) & (k > 0) & (k < N)
    return inside.transpose(2, 1, 0).reshape(-1)  # node i + n1 (j + n1 k)


def test_prolongation_is_the_trilinear_interpolant():
    Nc = 4
    Nf = 2 * Nc
    nc1, nf1 = Nc + 1, Nf + 1
    fc = inputs.random_vector(21, nc1 ** 3) * interior_mask(Nc)   # boundary values 0
    Fc = fc.reshape(nc1, nc1, nc1)                                   # [k][j][i]
    got = G.prolongation(Nc) @ fc
    ref = np.zeros(nf1 ** 3)
    for k in range(nf1):
        for j in range(nf1):
            for i in range(nf1):
                if not (0 < i < Nf and 0 < j < Nf and 0 < k < Nf):
                    continue
                # coarse cell and local coordinates of the fine node
                x, y, z = i / 2.0, j / 2.0, k / 2.0
                ci, cj, ck = min(int(x), Nc - 1), min(int(y), Nc - 1), min(int(z), Nc - 1)
                u, v, w = x - ci, y - cj, z - ck
                val = 0.0
                for dk in (0, 1):
                    for dj in (0, 1):
                        for di in (0, 1):
                            wt = (u if di else 1 - u) * (v if dj else 1 - v) * (w if dk else 1 - w)
                            val += wt * Fc[ck + dk, cj + dj, ci + di]
                ref[i + nf1 * (j + nf1 * k)] = val
    assert np.max(np.abs(got - ref)) <= 1e-15


def test_galerkin_product_equals_rediscretisation_for_constant_coefficient():
    Nc = 4
    xi = np.zeros(10)
    rmf, colf = O.graph(2 * Nc)
    vf, _ = O.assemble(2 * Nc, 10, xi, rmf, colf, sigma=0.0)
    rmc, colc = O.graph(Nc)
    vc, _ = O.assemble(Nc, 10, xi, rmc, colc, sigma=0.0)
    Af = sp.csr_matrix((vf, colf, rmf))
    Ac = sp.csr_matrix((vc, colc, rmc)).toarray()
    Pm = G.prolongation(Nc)
    RAP = (Pm.T @ Af @ Pm).toarray()
    m = interior_mask(Nc)
    blk = np.ix_(m, m)
    assert np.max(np.abs(RAP[blk] - Ac[blk])) <= 1e-15 * np.max(np.abs(Ac))


def small_hierarchy(N, seed=31, **kw):
    xi = inputs.kl_samples(seed, 0, 1, 10)[0]
    starts = [inputs.random_vector(600 + l, (n + 1) ** 3) for l, n in enumerate(G.level_sizes(N))]
    return G.hierarchy(N, 10, xi, starts, **kw)


def test_vcycle_is_symmetric_positive_definite():
    levels = small_hierarchy(8)
    n = (8 + 1) ** 3
    m = interior_mask(8)
    V = np.stack([G.vcycle(levels, e) for e in np.eye(n)[m]], axis=1)[m]
    assert np.max(np.abs(V - V.T)) <= 1e-12 * np.max(np.abs(V))
    assert np.linalg.eigvalsh(0.5 * (V + V.T)).min() > 0


def test_mg_pcg_matches_direct_solve_in_few_iterations():
    its = []
    for N in (8, 16):
        levels = small_hierarchy(N, seed=40 + N)
        lev = levels[0]
        x, it, rr, st = G.mg_pcg(levels, lev.load, tol=1e-10)
        xd = spla.spsolve(sp.csr_matrix((lev.vals, lev.col, lev.rm)).tocsc(), lev.load)
        assert st == 0 and rr <= 1e-9
        assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
        its.append(it)
    # plain CG needs ~37 iterations at 16^3 (1e-8); the V-cycle keeps the count small and flat
    assert max(its) <= 8 and its[1] <= its[0] + 1, its
