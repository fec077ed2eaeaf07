"""Pins for the learned-guess oracle (POD, MLP, Adam), independent of it.

POD against a matrix built with a known SVD (mean, singular values, singular
vectors, the sign rule, Eckart-Young); GELU against the standard normal CDF
table value and the identity g(x) - g(-x) = x; the forward pass against its
affine limits (all GELUs in the linear regime, or all switched off); the
backward pass against central finite differences; Adam against the closed
form of a step taken with a constant gradient; training against a teacher
network it can represent.
"""
import math

import numpy as np
import pytest

from oracle import learned as L
from paper_1511_03703_gb300 import inputs

DIMS_SMALL = (3, 5, 4, 2)


def known_svd(n, m, r, seed, decay=0.5):
    """X = mean 1^T + U diag(sigma) V^T with V^T 1 = 0 (the centring leaves
    the factors unchanged), sigma_i = decay^i."""
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((n, r)))
    B = rng.standard_normal((m, r))
    B -= B.mean(axis=0)
    V, _ = np.linalg.qr(B)
    sigma = decay ** np.arange(r)
    mean = rng.standard_normal(n)
    return mean[:, None] + (U * sigma) @ V.T, mean, U, sigma, V


def test_pod_recovers_constructed_svd_and_sign_rule():
    n, m, r, k = 60, 25, 12, 6
    X, mean, U, sigma, V = known_svd(n, m, r, 7)
    mu, Phi, s = L.pod(X, k)
    assert np.max(np.abs(mu - mean)) <= 1e-14 * np.max(np.abs(mean)) * 10
    assert np.allclose(s[:r], sigma, rtol=1e-12, atol=0)
    assert np.all(s[r:] <= 1e-13)
    for j in range(k):
        i = int(np.argmax(np.abs(Phi[:, j])))
        assert Phi[i, j] > 0
        u = U[:, j] * np.sign(U[np.argmax(np.abs(U[:, j])), j])
        assert np.max(np.abs(Phi[:, j] - u)) <= 1e-11
    assert np.max(np.abs(Phi.T @ Phi - np.eye(k))) <= 1e-14
    # Eckart-Young: the rank-k projection error is the discarded energy
    Xc = X - mu[:, None]
    err = np.linalg.norm(Xc - Phi @ (Phi.T @ Xc)) ** 2
    assert abs(err - np.sum(sigma[k:] ** 2)) <= 1e-12 * np.sum(sigma ** 2)


def test_pod_targets_are_scaled_right_singular_vectors():
    n, m, r, k = 50, 30, 8, 5
    X, mean, U, sigma, V = known_svd(n, m, r, 8)
    mu, Phi, s = L.pod(X, k)
    cm, sd, T = L.pod_targets(X - mu[:, None], Phi)
    signs = np.sign(np.sum(Phi * U[:, :k], axis=0))
    C_exact = V[:, :k] * sigma[:k] * signs
    assert np.max(np.abs(cm)) <= 1e-14
    assert np.allclose(sd, sigma[:k] / math.sqrt(m), rtol=1e-12)
    assert np.allclose(T, C_exact / (sigma[:k] / math.sqrt(m)), atol=1e-11)
    # every standardised column has mean 0 and population variance 1
    assert np.allclose(T.mean(axis=0), 0.0, atol=1e-13)
    assert np.allclose((T ** 2).mean(axis=0), 1.0, rtol=1e-12)


def test_guess_reconstructs_training_columns():
    n, m, r = 40, 20, 6
    X, *_ = known_svd(n, m, r, 9)
    mu, Phi, s = L.pod(X, r)  # k = rank: the basis spans every centred column
    cm, sd, T = L.pod_targets(X - mu[:, None], Phi)
    cols = [3, 11, 19]
    x0 = L.guess(mu, Phi, cm, sd, T[cols]).reshape(n, len(cols))
    assert np.max(np.abs(x0 - X[:, cols])) <= 1e-13 * np.max(np.abs(X))


def test_gelu_table_value_symmetry_and_limits():
    # g(1) = Phi_N(1), the standard normal CDF at 1
    assert abs(L.gelu(np.float64(1.0)) - 0.8413447460685429) <= 1e-16
    assert L.gelu(np.float64(0.0)) == 0.0
    x = np.linspace(-6, 6, 97)
    assert np.max(np.abs(L.gelu(x) - L.gelu(-x) - x)) <= 1e-15 * 8
    big = np.array([12.0, 50.0, 300.0])
    assert np.array_equal(L.gelu(big), big)
    assert np.all(L.gelu(-big) == 0.0)
    h = 1e-6
    z = np.linspace(-5, 5, 41)
    fd = (L.gelu(z + h) - L.gelu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - L.gelu_grad(z))) <= 1e-9


def random_params(dims, seed, scale=1.0):
    return scale * inputs.random_vector(seed, L.param_count(dims), -1.0, 1.0)


def test_forward_linear_regime_is_affine_composition():
    dims = DIMS_SMALL
    w = np.abs(random_params(dims, 41)) + 0.1
    W1, b1, W2, b2, W3, b3 = L.unpack(dims, w)
    b1 += 20.0
    b2 += 20.0
    X = np.abs(inputs.random_vector(42, 7 * dims[0])).reshape(7, dims[0])
    Y = L.forward(dims, w, X)
    # every pre-activation exceeds 10, where g(z) = z in FP64
    A = W3 @ W2 @ W1
    c = W3 @ (W2 @ b1 + b2) + b3
    assert np.allclose(Y, X @ A.T + c, rtol=1e-14, atol=0)


def test_forward_switched_off_gives_output_bias():
    dims = DIMS_SMALL
    w = 0.01 * random_params(dims, 43)
    W1, b1, W2, b2, W3, b3 = L.unpack(dims, w)
    b1[:] = -50.0
    b2[:] = -50.0
    X = inputs.random_vector(44, 5 * dims[0]).reshape(5, dims[0])
    assert np.array_equal(L.forward(dims, w, X), np.broadcast_to(b3, (5, dims[3])))


def test_gradient_matches_central_differences():
    dims = DIMS_SMALL
    w = random_params(dims, 51)
    X = inputs.random_vector(52, 7 * dims[0]).reshape(7, dims[0])
    T = inputs.random_vector(53, 7 * dims[3]).reshape(7, dims[3])
    loss, g = L.loss_grad(dims, w, X, T)
    h = 1e-6
    fd = np.empty_like(w)
    for i in range(len(w)):
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd[i] = (L.loss_grad(dims, wp, X, T)[0] - L.loss_grad(dims, wm, X, T)[0]) / (2 * h)
    assert np.max(np.abs(fd - g)) <= 1e-6 * np.max(np.abs(g))
    assert abs(loss - np.mean((L.forward(dims, w, X) - T) ** 2)) == 0.0


def test_adam_constant_gradient_closed_form():
    g = np.array([0.3, -2.0, 1e-3, 5.0])
    w0 = np.array([1.0, 2.0, 3.0, 4.0])
    lr0, total, eps = 1e-2, 100, 1e-8
    # step 0: m_hat = g, v_hat = g^2, lr = lr0
    w1, m, v = L.adam_step(w0, g, np.zeros(4), np.zeros(4), 0, total, lr0, eps=eps)
    assert np.allclose(w1 - w0, -lr0 * g / (np.abs(g) + eps), rtol=1e-12)
    # with a constant gradient m_hat = g and v_hat = g^2 at every step;
    # the cosine schedule halves the step at t = total/2 and ends at 0
    w, m, v = w0.copy(), np.zeros(4), np.zeros(4)
    steps = []
    for t in range(total + 1):
        wn, m, v = L.adam_step(w, g, m, v, t, total, lr0, eps=eps)
        steps.append(wn - w)
        w = wn
    assert np.allclose(steps[50], -0.5 * lr0 * g / (np.abs(g) + eps), rtol=1e-9)
    assert np.allclose(steps[total], 0.0, atol=1e-18)


def test_init_he_uniform_bounds():
    dims = (10, 256, 256, 64)
    u = inputs.mlp_init_draws(2005, L.param_count(dims))
    w = L.init(dims, u)
    W1, b1, W2, b2, W3, b3 = L.unpack(dims, w)
    for W, fan in ((W1, 10), (W2, 256), (W3, 256)):
        lim = math.sqrt(6.0 / fan)
        assert np.max(np.abs(W)) <= lim and np.max(np.abs(W)) > 0.99 * lim
        # uniform on [-lim, lim]: variance lim^2 / 3 = 2 / fan_in (He)
        assert abs(np.var(W) - 2.0 / fan) < 0.1 * 2.0 / fan
    assert not np.any(b1) and not np.any(b2) and not np.any(b3)


def test_training_fits_a_teacher_network():
    dims = (3, 16, 16, 2)
    teacher = random_params(dims, 61)
    X = inputs.random_vector(62, 64 * 3).reshape(64, 3)
    T = L.forward(dims, teacher, X)
    w0 = L.init(dims, inputs.mlp_init_draws(63, L.param_count(dims)))
    w, m, v, step, losses = L.train(dims, w0, X, T, batch=16, epochs=150, total=600, lr0=1e-2)
    assert step == 600
    assert losses[-1] < 0.02 * losses[0]
    assert all(np.isfinite(losses))
