"""CPU oracle of the learned initial guess: POD basis, MLP, Adam, FP64 numpy.

TEST INFRASTRUCTURE ONLY: only `tests/`, `__graft_entry__.smoke()` and the
benchmark's CPU-baseline leg may import this module.  It shares no code with
the CUDA library.

The learned guess is not in the paper (its CG of Sect. 3.4 starts from
x = 0); every step here is the plain textbook definition, in FP64:

  POD     centred snapshots Xc = X - mean 1^T; Phi = the k leading left
          singular vectors of Xc (LAPACK SVD through numpy), each column
          signed so that its largest-magnitude entry (first on ties) is
          positive; sigma = all singular values, descending.
  targets C = Xc^T Phi; per-column mean and population standard deviation
          (1 where it is 0); T = (C - mean) / std.
  MLP     z1 = W1 x + b1, a1 = g(z1), z2 = W2 a1 + b2, a2 = g(z2),
          y = W3 a2 + b3, with the exact GELU g(z) = z Phi_N(z) =
          z (1 + erf(z / sqrt 2)) / 2; loss = mean over batch and outputs of
          (y - t)^2; gradients by the chain rule (reverse mode).
  Adam    Kingma and Ba (ICLR 2015), Algorithm 1, with the step size
          lr0 (1 + cos(pi t / T)) / 2 at step t (cosine decay, 0-based t).
  guess   x0 = mean + Phi (coef_mean + coef_scale * chat), per member.

Parameter vector layout (shared only as an interface with the CUDA side):
W1 [d1 x d0], b1 [d1], W2 [d2 x d1], b2 [d2], W3 [d3 x d2], b3 [d3],
row-major.  Pins: tests/test_oracle_learned.py.
"""
import math

import numpy as np
from scipy.special import erf


# ------------------------------------------------------------------ POD
def pod(X, k):
    """(mean[n], Phi[n, k], sigma[min(n, m)]) of snapshots X[n, m] (columns = samples)."""
    X = np.asarray(X, dtype=np.float64)
    mean = X.mean(axis=1)
    Xc = X - mean[:, None]
    U, sigma, _ = np.linalg.svd(Xc, full_matrices=False)
    Phi = U[:, :k].copy()
    for j in range(k):
        i = int(np.argmax(np.abs(Phi[:, j])))
        if Phi[i, j] < 0.0:
            Phi[:, j] = -Phi[:, j]
    return mean, Phi, sigma


def pod_targets(Xc, Phi):
    """Standardised POD coefficients of centred snapshots Xc[n, m]:
    (coef_mean[k], coef_scale[k], T[m, k])."""
    C = np.asarray(Xc, dtype=np.float64).T @ Phi
    cm = C.mean(axis=0)
    sd = np.sqrt(((C - cm) ** 2).mean(axis=0))
    sd = np.where(sd > 0.0, sd, 1.0)
    return cm, sd, (C - cm) / sd


def guess(mean, Phi, coef_mean, coef_scale, chat):
    """x0 in ensemble layout x0[i*s + e] for s members with predictions chat[s, k]."""
    c = coef_mean[None, :] + coef_scale[None, :] * np.asarray(chat, dtype=np.float64)
    x0 = mean[:, None] + Phi @ c.T
    return np.ascontiguousarray(x0).reshape(-1)


# ------------------------------------------------------------------ MLP
SQRT2 = math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / SQRT2))


def gelu_grad(z):
    """d/dz [z Phi_N(z)] = Phi_N(z) + z phi_N(z)."""
    return 0.5 * (1.0 + erf(z / SQRT2)) + z * INV_SQRT_2PI * np.exp(-0.5 * z * z)


def param_count(dims):
    d0, d1, d2, d3 = dims
    return d1 * d0 + d1 + d2 * d1 + d2 + d3 * d2 + d3


def unpack(dims, w):
    """Views (W1, b1, W2, b2, W3, b3) into the flat parameter vector w."""
    d0, d1, d2, d3 = dims
    out, o = [], 0
    for shape in ((d1, d0), (d1,), (d2, d1), (d2,), (d3, d2), (d3,)):
        size = int(np.prod(shape))
        out.append(w[o:o + size].reshape(shape))
        o += size
    return out


def init(dims, u):
    """He-uniform start from draws u in [-1, 1]: W_l = u sqrt(6 / fan_in), biases 0."""
    u = np.asarray(u, dtype=np.float64)
    w = np.zeros(param_count(dims))
    W1, b1, W2, b2, W3, b3 = unpack(dims, w)
    U = unpack(dims, u)
    W1[:] = U[0] * math.sqrt(6.0 / dims[0])
    W2[:] = U[2] * math.sqrt(6.0 / dims[1])
    W3[:] = U[4] * math.sqrt(6.0 / dims[2])
    return w


def forward(dims, w, X, cache=False):
    """Outputs Y[B, d3] for inputs X[B, d0] (rows = samples)."""
    W1, b1, W2, b2, W3, b3 = unpack(dims, np.asarray(w, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + b1
    a1 = gelu(z1)
    z2 = a1 @ W2.T + b2
    a2 = gelu(z2)
    y = a2 @ W3.T + b3
    if cache:
        return y, (X, z1, a1, z2, a2)
    return y


def loss_grad(dims, w, X, T):
    """(loss, grad) of the mean squared error mean((Y - T)^2) over B x d3."""
    w = np.asarray(w, dtype=np.float64)
    W1, b1, W2, b2, W3, b3 = unpack(dims, w)
    y, (X, z1, a1, z2, a2) = forward(dims, w, X, cache=True)
    T = np.asarray(T, dtype=np.float64)
    diff = y - T
    loss = float(np.mean(diff * diff))
    dy = 2.0 * diff / diff.size
    g = np.zeros_like(w)
    gW1, gb1, gW2, gb2, gW3, gb3 = unpack(dims, g)
    gW3[:] = dy.T @ a2
    gb3[:] = dy.sum(axis=0)
    dz2 = (dy @ W3) * gelu_grad(z2)
    gW2[:] = dz2.T @ a1
    gb2[:] = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * gelu_grad(z1)
    gW1[:] = dz1.T @ X
    gb1[:] = dz1.sum(axis=0)
    return loss, g


def adam_step(w, g, m, v, t, total, lr0, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at 0-based step t; returns new (w, m, v)."""
    lr = 0.5 * lr0 * (1.0 + math.cos(math.pi * t / total))
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** (t + 1))
    vhat = v / (1.0 - beta2 ** (t + 1))
    return w - lr * mhat / (np.sqrt(vhat) + eps), m, v


def train(dims, w, X, T, batch, epochs, total, lr0, beta1=0.9, beta2=0.999, eps=1e-8,
          m=None, v=None, step=0):
    """Epochs over X[n, d0] / T[n, d3] in fixed consecutive mini-batches.
    Returns (w, m, v, step, epoch_losses) with each epoch's mean batch loss."""
    n = X.shape[0]
    assert n % batch == 0
    w = np.asarray(w, dtype=np.float64).copy()
    m = np.zeros_like(w) if m is None else m.copy()
    v = np.zeros_like(w) if v is None else v.copy()
    losses = []
    for _ in range(epochs):
        acc = 0.0
        for b in range(n // batch):
            sl = slice(b * batch, (b + 1) * batch)
            loss, g = loss_grad(dims, w, X[sl], T[sl])
            acc += loss
            w, m, v = adam_step(w, g, m, v, step, total, lr0, beta1, beta2, eps)
            step += 1
        losses.append(acc / (n // batch))
    return w, m, v, step, losses
