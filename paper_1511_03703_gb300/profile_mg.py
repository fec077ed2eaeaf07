"""Profiling driver: multigrid-preconditioned ensemble CG on an N^3 mesh.

    python -m paper_1511_03703_gb300.profile_mg N s reps [presplit|f32]

Builds the level hierarchy (N, N/2, ... > 4), then `reps` times assembles
every level of one ensemble of s samples (double-float assembly, M = 10, seed
of the 64^3 workload) and solves to 1e-8 with the V-cycle preconditioner
(graph replay of 4 iterations), printing the wall time of each part.
presplit: every level also writes its pre-split values, so that the V-cycle's
SpMVs run in double-float (as in the benchmark).  f32: the finest level writes
its pre-split values (the CG's SpMV) and every level an FP32 copy of its values
for the FP32 V-cycle (the benchmark's FP32 form; the copy is made after each
assembly).  Used for the launch-list summaries under profiles/.
"""
import sys
import time

import numpy as np
import torch

import paper_1511_03703_gb300 as E
from paper_1511_03703_gb300 import inputs


def main(argv):
    N, s, reps = int(argv[1]), int(argv[2]), int(argv[3])
    mode = argv[4] if len(argv) > 4 else ""
    presplit, f32 = mode == "presplit", mode == "f32"
    dev = torch.device("cuda:0")
    mg = E.Multigrid(N, 10, device=dev)
    xs = inputs.kl_samples(inputs.SEED_SCALE, 0, s, 10)
    xi = torch.from_numpy(inputs.ensemble_layout(xs)).to(dev)
    starts = [torch.from_numpy(np.stack([inputs.random_vector(600 + 100 * l + e, m.n) for e in range(s)],
                                        axis=1).reshape(-1)).to(dev) for l, m in enumerate(mg.meshes)]
    x = torch.zeros(mg.meshes[0].n * s, dtype=torch.float64, device=dev)
    split_levels = mg.meshes if presplit else (mg.meshes[:1] if f32 else [])
    pre = [torch.empty(2 * m.nnz * s, dtype=torch.float32, device=dev) for m in split_levels] or None
    vals, b = mg.assemble(s, xi, df=True, values_df=pre)
    v32 = mg.to_f32(s, vals) if f32 else None
    work = torch.empty(mg.workspace_size(s, vals, starts, pre, v32), dtype=torch.uint8, device=dev)
    for rep in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x.zero_()
        vals, b = mg.assemble(s, xi, df=True, values_df=pre)
        if f32:
            mg.to_f32(s, vals, out=v32)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        it, rr, st, stats = mg.solve(s, vals, b, x, 1e-8, 500, work, starts, flags=E.CG_GRAPH | E.CG_X0_ZERO,
                                     check_every=4, values_df=pre, values_f32=v32)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        print(f"rep {rep}: assemble {1e3 * (t1 - t0):.2f} ms, solve {1e3 * (t2 - t1):.2f} ms, "
              f"iterations {max(it)}, status {sorted(set(st))}")


if __name__ == "__main__":
    main(sys.argv)
