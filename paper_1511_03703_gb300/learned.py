"""Learned initial guess for ensemble CG (not in the paper; its CG starts from 0).

Pipeline, every arithmetic step in the library's kernels (this module only
allocates device memory and sequences the C-ABI calls):

  1. collect:  solve training samples with ens_cg (ensembles of s members)
               and copy each solution into a column of the snapshot matrix X;
  2. fit_basis: POD of X (ens_pod: centred, randomized range finder, Jacobi
               Rayleigh-Ritz), standardised coefficients (ens_pod_targets),
               and an FP32 copy of the basis (ens_to_f32);
  3. train:    MLP xi -> standardised coefficients with the library's own
               forward, backward and Adam kernels (ens_mlp_train), one epoch
               per CUDA graph replay;
  4. predict:  x0 = mean + Phi (coef_mean + coef_scale * MLP(xi)) per member
               (ens_guess), then ens_cg with ENS_CG_GUESS_FALLBACK, which
               restarts from x = 0 any member whose ||b - A x0|| >= ||b||.

State can be saved and restored (save / load): raw little-endian arrays plus
a JSON header, including the Adam moments and step so training can resume.
"""
import json
import os

import numpy as np

import paper_1511_03703_gb300 as E
from paper_1511_03703_gb300 import inputs

# training recipe (fixed): Adam, cosine decay, batch 256
LR0, BETA1, BETA2, EPS, BATCH = 1e-3, 0.9, 0.999, 1e-8, 256


def collect(mesh, xi_rows, s=32, tol=1e-8, max_iter=10000, flags=0, presplit=True, X=None, col0=0):
    """Solve the samples xi_rows[m, M] in ensembles of s and return the
    snapshot matrix X (n x m, FP64, device) and the iteration counts.
    presplit: double-float assembly with its pre-split copy and ens_cg_df
    (else FP64 assembly and ens_cg with `flags`)."""
    import torch
    m = xi_rows.shape[0]
    assert m % s == 0, "number of samples must be a multiple of s"
    dev = mesh.row_map.device
    if X is None:
        X = torch.empty((mesh.n, m), dtype=torch.float64, device=dev)
    work = torch.empty(E.cg_workspace_size(mesh.n, s), dtype=torch.uint8, device=dev)
    x = torch.empty(mesh.n * s, dtype=torch.float64, device=dev)
    vdf = torch.empty(2 * mesh.nnz * s, dtype=torch.float32, device=dev) if presplit else None
    vals = b = None
    iters = []
    for j in range(0, m, s):
        xi = torch.from_numpy(inputs.ensemble_layout(xi_rows[j:j + s])).to(dev)
        vals, b = mesh.assemble(s, xi, values=vals, b=b, values_df=vdf)  # df assembly when presplit
        x.zero_()
        it, rr, st, _ = E.cg(mesh.graph, s, vals, b, x, tol, max_iter, work,
                             flags=flags | E.CG_GRAPH | E.CG_X0_ZERO, check_every=8, values_df=vdf)
        if any(st):
            raise E.EnsError(max(st), f"training solve {j // s}: member statuses {st}")
        E.snapshots_put(x, X, col0 + j, s)
        iters += it
    return X, iters


class LearnedGuess:
    """POD basis + MLP for one mesh (n nodes), on the GPU."""

    def __init__(self, n, k=64, dims=E.MLP_DIMS, device="cuda"):
        import torch
        assert dims[3] == k
        self.n, self.k, self.dims = n, k, tuple(dims)
        self.device = torch.device(device)
        f64 = dict(dtype=torch.float64, device=self.device)
        f32 = dict(dtype=torch.float32, device=self.device)
        self.mean = torch.zeros(n, **f64)
        self.Phi = torch.zeros((n, k), **f64)
        self.Phi32 = torch.zeros((n, k), **f32)
        self.sigma = torch.zeros(k, **f64)
        self.coef_mean = torch.zeros(k, **f64)
        self.coef_scale = torch.ones(k, **f64)
        P = E.mlp_param_count(self.dims)
        self.params = torch.zeros(P, **f32)
        self.adam_m = torch.zeros(P, **f32)
        self.adam_v = torch.zeros(P, **f32)
        self.step = torch.zeros(2, dtype=torch.int64, device=self.device)
        self.total_steps = 1
        self._gwork = {}

    # ------------------------------------------------------------ basis
    def fit_basis(self, X, l=80, power_iters=1, seed=inputs.SEED_GUESS_TRAIN):
        """POD of the snapshot columns of X (centred in place); returns the
        standardised training targets T (float32, m x k, device)."""
        import torch
        n, m = X.shape
        assert n == self.n
        Omega = torch.from_numpy(inputs.pod_test_matrix(seed, m, l)).to(self.device)
        work = torch.empty(E.pod_workspace_size(n, m, l), dtype=torch.uint8, device=self.device)
        E.pod(X, self.k, l, Omega, self.mean, self.Phi, self.sigma, work, power_iters=power_iters)
        del work
        T = torch.empty((m, self.k), dtype=torch.float32, device=self.device)
        E.pod_targets(X, self.Phi, self.coef_mean, self.coef_scale, T)
        E.to_f32(self.Phi, self.Phi32)
        return T

    # ------------------------------------------------------------ network
    def init_params(self, seed=inputs.SEED_GUESS_TRAIN):
        import torch
        u = torch.from_numpy(inputs.mlp_init_draws(seed, self.params.numel())).to(self.device)
        E.mlp_init(u, self.params, self.dims)
        self.adam_m.zero_()
        self.adam_v.zero_()
        self.step.zero_()

    def train(self, xi_rows, T, epochs, batch=BATCH, total_steps=None, epoch_loss=True, use_graph=True):
        """Adam epochs over (xi_rows[m, d0] FP64 host or device, T[m, k]);
        returns the per-epoch mean losses (numpy) or None."""
        import torch
        xi = torch.as_tensor(xi_rows, dtype=torch.float64).to(self.device).contiguous()
        xin = torch.empty(xi.shape, dtype=torch.float32, device=self.device)
        E.to_f32(xi, xin)
        m = xin.shape[0]
        self.total_steps = total_steps or epochs * (m // batch)
        work = torch.empty(E.mlp_workspace_size(batch, self.dims), dtype=torch.uint8, device=self.device)
        el = torch.zeros(max(epochs, 1), dtype=torch.float32, device=self.device) if epoch_loss else None
        E.mlp_train(self.params, self.adam_m, self.adam_v, self.step, xin, T, batch, epochs, self.total_steps,
                    work, LR0, BETA1, BETA2, EPS, epoch_loss=el, use_graph=use_graph, dims=self.dims)
        return None if el is None else el.cpu().numpy()

    # ------------------------------------------------------------ inference
    def predict(self, xi_ens, s, x0, stream=None):
        """x0 (n*s, commuted layout) for the ensemble whose KL variables are
        xi_ens (device FP64, xi[k*s + e], the ens_assemble input)."""
        import torch
        if s not in self._gwork:
            self._gwork[s] = torch.empty(E.guess_workspace_size(s, self.dims), dtype=torch.uint8,
                                         device=self.device)
        E.guess(self.params, s, xi_ens, self.mean, self.Phi32, self.coef_mean, self.coef_scale, x0,
                self._gwork[s], dims=self.dims, stream=stream)

    # ------------------------------------------------------------ checkpoint
    _ARRAYS = ("mean", "Phi", "Phi32", "sigma", "coef_mean", "coef_scale", "params", "adam_m", "adam_v",
               "step")

    def save(self, path):
        """Directory with header.json and one raw little-endian file per array."""
        os.makedirs(path, exist_ok=True)
        files = {}
        for name in self._ARRAYS:
            a = getattr(self, name).detach().cpu().numpy()
            a = a.astype(a.dtype.newbyteorder("<"), copy=False)
            a.tofile(os.path.join(path, name + ".bin"))
            files[name] = {"dtype": a.dtype.str, "shape": list(a.shape)}
        hdr = {"format": "ens-learned-guess-1", "n": self.n, "k": self.k, "dims": list(self.dims),
               "total_steps": self.total_steps, "files": files}
        with open(os.path.join(path, "header.json"), "w") as f:
            json.dump(hdr, f, indent=1)

    @classmethod
    def load(cls, path, device="cuda"):
        import torch
        with open(os.path.join(path, "header.json")) as f:
            hdr = json.load(f)
        if hdr.get("format") != "ens-learned-guess-1":
            raise ValueError(f"{path}: not a learned-guess checkpoint")
        g = cls(hdr["n"], hdr["k"], tuple(hdr["dims"]), device)
        g.total_steps = hdr["total_steps"]
        for name, meta in hdr["files"].items():
            a = np.fromfile(os.path.join(path, name + ".bin"), dtype=np.dtype(meta["dtype"]))
            a = a.reshape(meta["shape"]).astype(a.dtype.newbyteorder("="))
            getattr(g, name).copy_(torch.from_numpy(a))
        return g
