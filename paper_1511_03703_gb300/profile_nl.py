"""Profiling driver: Newton-GMRES for the nonlinear advection-diffusion
problem on an N^3 mesh.

    python -m paper_1511_03703_gb300.profile_nl N s reps

Builds the level hierarchy and the advection matrix (v = (1, 1, 1)), then
`reps` times assembles every level of one ensemble of s samples (double-float
assembly with every level's pre-split copy, M = 10, seed of the 64^3 workload)
and runs Newton from u = 0 (alpha = 1, beta = 10, tol 1e-8, GMRES(30) to
1e-6 per step, V-cycle right preconditioner), printing the wall time of each
part.  Used for the launch-list summaries under profiles/.
"""
import sys
import time

import numpy as np
import torch

import paper_1511_03703_gb300 as E
from paper_1511_03703_gb300 import inputs


def main(argv):
    N, s, reps = int(argv[1]), int(argv[2]), int(argv[3])
    dev = torch.device("cuda:0")
    nl = E.Nonlinear(N, 10, v=(1.0, 1.0, 1.0), precond=E.NL_PRECOND_MG, device=dev)
    xs = inputs.kl_samples(inputs.SEED_SCALE, 0, s, 10)
    xi = torch.from_numpy(inputs.ensemble_layout(xs)).to(dev)
    starts = [torch.from_numpy(np.stack([inputs.random_vector(600 + 100 * l + e, m.n) for e in range(s)],
                                        axis=1).reshape(-1)).to(dev) for l, m in enumerate(nl.meshes)]
    p = nl.params(1.0, 10.0, tol=1e-8, lin_tol=1e-6, restart=30, max_lin=300, max_newton=20)
    u = torch.zeros(nl.mesh.n * s, dtype=torch.float64, device=dev)
    vdf = [torch.empty(2 * m.nnz * s, dtype=torch.float32, device=dev) for m in nl.meshes]
    vals, b = nl.assemble(s, xi, values_df=vdf)
    work = torch.empty(nl.workspace_size(s, vals, starts, p, vdf), dtype=torch.uint8, device=dev)
    for rep in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        u.zero_()
        vals, b = nl.assemble(s, xi, values_df=vdf)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        ni, li, rr, st, stats = nl.solve(s, vals, b, u, work, starts, p, values_df=vdf)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        print(f"rep {rep}: assemble {1e3 * (t1 - t0):.2f} ms, solve {1e3 * (t2 - t1):.2f} ms, "
              f"newton {max(ni)}, gmres {max(li)}, status {sorted(set(st))}")


if __name__ == "__main__":
    main(sys.argv)
