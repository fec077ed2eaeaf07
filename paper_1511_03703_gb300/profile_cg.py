"""Profiling driver: one ensemble CG with a fixed iteration count on an N^3 mesh.

    python -m paper_1511_03703_gb300.profile_cg N s iters [form]

form: f64 (default), df, split, or dfv (double-float assembly with its
pre-split copy, then ens_cg_df).

Builds the mesh set-up, assembles one ensemble of s samples (M = 10, seed of
the 64^3 workload) and runs `iters` CG iterations (tolerance 0, so exactly
that many), so that an `ncu -k regex:cg_spmv_kernel -s 1 -c 1` capture sees a
steady-state SpMV launch.  Used for the summaries under profiles/.
"""
import sys

import torch

import paper_1511_03703_gb300 as E
from paper_1511_03703_gb300 import inputs


def main(argv):
    N, s, iters = int(argv[1]), int(argv[2]), int(argv[3])
    form = argv[4] if len(argv) > 4 else "f64"
    flags = {"f64": 0, "df": E.CG_DF64, "split": E.CG_SPLIT64, "dfv": 0}[form]
    mesh = E.Mesh(N, 10)
    xs = inputs.kl_samples(inputs.SEED_SCALE, 0, s, 10)
    xi = torch.from_numpy(inputs.ensemble_layout(xs)).cuda()
    vdf = None
    if form == "dfv":  # double-float assembly writing the pre-split copy, as in the benchmark
        vdf = torch.empty(2 * mesh.nnz * s, dtype=torch.float32, device="cuda")
    vals, b = mesh.assemble(s, xi, values_df=vdf)
    x = torch.zeros(mesh.n * s, dtype=torch.float64, device="cuda")
    work = torch.empty(E.cg_workspace_size(mesh.n, s), dtype=torch.uint8, device="cuda")
    it, rr, st, stats = E.cg(mesh.graph, s, vals, b, x, 0.0, iters, work, flags=flags,
                             check_every=iters, values_df=vdf)
    torch.cuda.synchronize()
    print("N", N, "s", s, "iters", it[:2], "status", st[:2], "nnz", mesh.nnz, "rows", mesh.n)


if __name__ == "__main__":
    main(sys.argv)
