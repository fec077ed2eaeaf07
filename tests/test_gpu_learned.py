"""Learned initial guess on the GPU against the FP64 oracle (oracle/learned.py).

Bars: POD singular values and vectors to 1e-10 where the range finder is
exact (l spans the whole centred range) and to 1e-6 for a randomized basis,
with orthonormality to 1e-12 and the Eckart-Young optimum; FP32 MLP outputs to
2e-5 and gradients to 1e-4 relative of the FP64 oracle; Adam to FP32
rounding; the zero-guess fallback bitwise equal to a zero-guess solve; a
trained guess that saves CG iterations at the same tolerance.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import learned as L
import paper_1511_03703_gb300 as E
from paper_1511_03703_gb300 import inputs
from paper_1511_03703_gb300.learned import LearnedGuess, collect
from helpers import gpu, oracle_members, to_dev, to_np
from test_oracle_learned import known_svd

pytestmark = pytest.mark.gpu

DIMS = E.MLP_DIMS


@pytest.fixture(scope="module")
def torch():
    import torch as T
    assert T.cuda.is_available()
    E.lib()
    return T


def run_pod(torch, X_np, k, l, q, seed=5):
    n, m = X_np.shape
    X = to_dev(X_np)
    Om = to_dev(inputs.pod_test_matrix(seed, m, l))
    mean = torch.empty(n, dtype=torch.float64, device=gpu())
    Phi = torch.empty((n, k), dtype=torch.float64, device=gpu())
    sig = torch.empty(k, dtype=torch.float64, device=gpu())
    work = torch.empty(E.pod_workspace_size(n, m, l), dtype=torch.uint8, device=gpu())
    E.pod(X, k, l, Om, mean, Phi, sig, work, power_iters=q)
    return X, to_np(mean), to_np(Phi), to_np(sig)


def test_snapshots_put_is_a_copy(torch):
    n, s, m = 37, 8, 24
    x = to_dev(inputs.random_vector(3, n * s))
    X = torch.zeros((n, m), dtype=torch.float64, device=gpu())
    E.snapshots_put(x, X, 8, s)
    Xh = to_np(X)
    assert np.array_equal(Xh[:, 8:16], to_np(x).reshape(n, s))
    assert not Xh[:, :8].any() and not Xh[:, 16:].any()
    with pytest.raises(E.EnsError):
        E.snapshots_put(x, X, 20, s)


@pytest.mark.parametrize("q", [0, 1, 2])
def test_pod_exact_range_matches_oracle(torch, q):
    n, m, k = 300, 40, 16
    X_np, *_ = known_svd(n, m, m - 1, 11, decay=0.7)
    Xd, mean, Phi, sig = run_pod(torch, X_np, k, m - 1, q)
    mo, Po, so = L.pod(X_np, k)
    assert np.max(np.abs(mean - mo)) <= 1e-14 * np.max(np.abs(mo)) * 10
    assert np.allclose(sig, so[:k], rtol=1e-10, atol=0)
    assert np.max(np.abs(Phi - Po)) <= 1e-8
    assert np.max(np.abs(Phi.T @ Phi - np.eye(k))) <= 1e-12
    # X was centred in place
    assert np.max(np.abs(to_np(Xd) - (X_np - mo[:, None]))) <= 1e-13 * np.max(np.abs(X_np))


def test_pod_randomized_subspace(torch):
    rng = np.random.default_rng(21)
    n, m, k, l = 4000, 600, 16, 32
    U, _ = np.linalg.qr(rng.standard_normal((n, m)))
    V, _ = np.linalg.qr(rng.standard_normal((m, m)))
    sigma = np.exp(-np.arange(m) / 3.0)
    X_np = (U * sigma) @ V.T + 0.5
    Xd, mean, Phi, sig = run_pod(torch, X_np, k, l, 1)
    mo, Po, so = L.pod(X_np, k)
    assert np.allclose(sig, so[:k], rtol=1e-6, atol=0)
    assert np.max(np.abs(Phi.T @ Phi - np.eye(k))) <= 1e-12
    assert np.max(np.abs(Phi - Po)) <= 1e-5
    Xc = X_np - mo[:, None]
    err = np.linalg.norm(Xc - Phi @ (Phi.T @ Xc)) ** 2
    opt = np.sum(so[k:] ** 2)
    assert opt <= err <= opt * (1 + 1e-6)


def test_pod_identical_snapshots_report_breakdown(torch):
    X_np = np.tile(inputs.random_vector(7, 200)[:, None], (1, 30))
    with pytest.raises(E.EnsError) as ei:
        run_pod(torch, X_np, 4, 8, 1)
    assert ei.value.code == 6


def test_pod_argument_errors(torch):
    X = torch.zeros((50, 20), dtype=torch.float64, device=gpu())
    Om = torch.zeros((20, 20), dtype=torch.float64, device=gpu())
    v = torch.zeros(50 * 20, dtype=torch.float64, device=gpu())
    work = torch.empty(E.pod_workspace_size(50, 20, 20), dtype=torch.uint8, device=gpu())
    for k, l in ((4, 20), (0, 8), (9, 8), (4, 81)):  # l <= m - 1, 1 <= k <= l <= 80
        with pytest.raises(E.EnsError) as ei:
            E.pod(X, k, l, Om, v, v, v, work)
        assert ei.value.code == 1
    small = torch.empty(16, dtype=torch.uint8, device=gpu())
    with pytest.raises(E.EnsError) as ei:
        E.pod(X, 4, 8, Om, v, v, v, small)
    assert ei.value.code == 9


def test_pod_targets_and_guess_match_oracle(torch):
    n, m, k = 500, 64, 12
    X_np, *_ = known_svd(n, m, 40, 31, decay=0.8)
    Xd, mean, Phi, sig = run_pod(torch, X_np, k, 40, 1)
    cmean = torch.empty(k, dtype=torch.float64, device=gpu())
    cscale = torch.empty(k, dtype=torch.float64, device=gpu())
    T = torch.empty((m, k), dtype=torch.float32, device=gpu())
    Phid = to_dev(Phi)
    E.pod_targets(Xd, Phid, cmean, cscale, T)
    cmo, cso, To = L.pod_targets(X_np - mean[:, None], Phi)
    assert np.max(np.abs(to_np(cmean) - cmo)) <= 1e-13 * np.max(cso)
    assert np.allclose(to_np(cscale), cso, rtol=1e-12)
    assert np.max(np.abs(to_np(T) - To)) <= 1e-6 * np.max(np.abs(To))
    # the FP32 copy of the basis is the round-to-nearest of the FP64 basis
    Phi32 = torch.empty((n, k), dtype=torch.float32, device=gpu())
    E.to_f32(Phid, Phi32)
    assert np.array_equal(to_np(Phi32), Phi.astype(np.float32))


@pytest.mark.parametrize("s", [1, 4, 32])
def test_guess_matches_oracle(torch, s):
    n, k = 729, 64
    rng = np.random.default_rng(s)
    Phi = np.linalg.qr(rng.standard_normal((n, k)))[0]
    mean = inputs.random_vector(41, n, 0.0, 0.1)
    cm = inputs.random_vector(42, k, -1e-3, 1e-3)
    cs = inputs.random_vector(43, k, 0.01, 1.0)
    w = L.init(DIMS, inputs.mlp_init_draws(44, L.param_count(DIMS))) + 0.05 * inputs.random_vector(
        45, L.param_count(DIMS))
    w32 = w.astype(np.float32)
    xs = inputs.kl_samples(46, 0, s, 10)
    x0 = torch.empty(n * s, dtype=torch.float64, device=gpu())
    work = torch.empty(E.guess_workspace_size(s), dtype=torch.uint8, device=gpu())
    Phi32 = torch.empty((n, k), dtype=torch.float32, device=gpu())
    E.to_f32(to_dev(Phi), Phi32)
    E.guess(to_dev(w32), s, to_dev(inputs.ensemble_layout(xs)), to_dev(mean), Phi32, to_dev(cm), to_dev(cs),
            x0, work)
    chat = L.forward(DIMS, w32.astype(np.float64), xs.astype(np.float32).astype(np.float64))
    ref = L.guess(mean, Phi, cm, cs, chat)
    scale = np.abs(mean)[:, None] + np.abs(Phi) @ np.abs(cm[:, None] + cs[:, None] * chat.T)
    assert np.all(np.abs(to_np(x0) - ref) <= 2e-5 * scale.reshape(-1) + 1e-300)


def mlp_case(batch, seed, dims=DIMS):
    w = L.init(dims, inputs.mlp_init_draws(seed, L.param_count(dims)))
    w = (w + 0.05 * inputs.random_vector(seed + 1, len(w))).astype(np.float32)
    X = inputs.kl_samples(seed + 2, 0, batch, dims[0]).astype(np.float32)
    T = inputs.random_vector(seed + 3, batch * dims[3]).reshape(batch, dims[3]).astype(np.float32)
    return w, X, T


@pytest.mark.parametrize("batch", [1, 37, 256])
def test_mlp_forward_matches_oracle(torch, batch):
    w, X, _ = mlp_case(batch, 100)
    y = torch.empty((batch, DIMS[3]), dtype=torch.float32, device=gpu())
    work = torch.empty(E.mlp_workspace_size(batch), dtype=torch.uint8, device=gpu())
    E.mlp_forward(to_dev(w), to_dev(X), y, work)
    ref = L.forward(DIMS, w.astype(np.float64), X.astype(np.float64))
    assert np.max(np.abs(to_np(y) - ref)) <= 2e-5 * np.max(np.abs(ref))


@pytest.mark.parametrize("batch", [7, 256])
def test_mlp_gradient_matches_oracle(torch, batch):
    w, X, T = mlp_case(batch, 200)
    grad = torch.empty(len(w), dtype=torch.float32, device=gpu())
    loss = torch.empty(1, dtype=torch.float32, device=gpu())
    work = torch.empty(E.mlp_workspace_size(batch), dtype=torch.uint8, device=gpu())
    E.mlp_grad(to_dev(w), to_dev(X), to_dev(T), grad, work, loss=loss)
    lo, go = L.loss_grad(DIMS, w.astype(np.float64), X.astype(np.float64), T.astype(np.float64))
    assert abs(float(to_np(loss)[0]) - lo) <= 1e-5 * lo
    g = to_np(grad).astype(np.float64)
    for a, b in zip(L.unpack(DIMS, g), L.unpack(DIMS, go)):
        assert np.max(np.abs(a - b)) <= 1e-4 * np.max(np.abs(b))


def test_mlp_init_matches_oracle(torch):
    P = L.param_count(DIMS)
    u = inputs.mlp_init_draws(2005, P)
    w = torch.empty(P, dtype=torch.float32, device=gpu())
    E.mlp_init(to_dev(u), w)
    ref = L.init(DIMS, u.astype(np.float64))
    assert np.max(np.abs(to_np(w) - ref)) <= 1e-7 * np.max(np.abs(ref))


def test_adam_matches_oracle(torch):
    P = 5000
    w0 = inputs.random_vector(301, P).astype(np.float32)
    gs = [(inputs.random_vector(302 + i, P) * 10.0 ** inputs.random_vector(310 + i, P, -6, 0))
          .astype(np.float32) for i in range(4)]
    w, m, v = to_dev(w0), torch.zeros(P, dtype=torch.float32, device=gpu()), \
        torch.zeros(P, dtype=torch.float32, device=gpu())
    step = torch.zeros(2, dtype=torch.int64, device=gpu())
    wo, mo, vo = w0.astype(np.float64), np.zeros(P), np.zeros(P)
    for t, g in enumerate(gs):
        E.mlp_adam(w, to_dev(g), m, v, step, total_steps=10, lr0=1e-2)
        wo, mo, vo = L.adam_step(wo, g.astype(np.float64), mo, vo, t, 10, 1e-2)
    assert to_np(step).tolist() == [4, 0]
    assert np.max(np.abs(to_np(w) - wo)) <= 4e-7
    # FP32 rounding of each moment update, relative to the gradients summed
    gabs = sum(np.abs(g.astype(np.float64)) for g in gs)
    assert np.all(np.abs(to_np(m) - mo) <= 1e-6 * gabs)
    assert np.all(np.abs(to_np(v) - vo) <= 1e-6 * gabs ** 2)


def test_mlp_train_matches_oracle_and_graph_is_bitwise(torch):
    dims = (10, 32, 32, 8)
    n, batch, epochs = 64, 16, 3
    w, X, T = mlp_case(n, 400, dims)
    out = {}
    for graph in (False, True):
        wd = to_dev(w)
        m = torch.zeros_like(wd)
        v = torch.zeros_like(wd)
        step = torch.zeros(2, dtype=torch.int64, device=gpu())
        el = torch.zeros(epochs, dtype=torch.float32, device=gpu())
        work = torch.empty(E.mlp_workspace_size(batch, dims), dtype=torch.uint8, device=gpu())
        E.mlp_train(wd, m, v, step, to_dev(X), to_dev(T), batch, epochs, epochs * n // batch, work,
                    lr0=1e-3, epoch_loss=el, use_graph=graph, dims=dims)
        out[graph] = (to_np(wd), to_np(el), to_np(step))
    assert np.array_equal(out[False][0], out[True][0]) and np.array_equal(out[False][1], out[True][1])
    assert out[True][2].tolist() == [epochs * n // batch, 0]
    wo, mo, vo, st, losses = L.train(dims, w.astype(np.float64), X.astype(np.float64), T.astype(np.float64),
                                     batch, epochs, epochs * n // batch, 1e-3)
    assert np.allclose(out[True][1], losses, rtol=1e-4)
    d = np.abs(out[True][0] - wo)
    assert np.max(d) <= 2 * st * 1e-3
    assert np.mean(d > 1e-5) < 0.01


def test_train_resume_equals_one_run(torch):
    dims = (10, 16, 16, 4)
    n, batch = 32, 8
    w, X, T = mlp_case(n, 500, dims)
    res = []
    for split in ((4,), (1, 3)):
        wd = to_dev(w)
        m, v = torch.zeros_like(wd), torch.zeros_like(wd)
        step = torch.zeros(2, dtype=torch.int64, device=gpu())
        work = torch.empty(E.mlp_workspace_size(batch, dims), dtype=torch.uint8, device=gpu())
        for ep in split:
            E.mlp_train(wd, m, v, step, to_dev(X), to_dev(T), batch, ep, 16, work, dims=dims)
        res.append(to_np(wd))
    assert np.array_equal(res[0], res[1])


# ------------------------------------------------------- zero-guess fallback
def ensemble(torch, N, s, seed, M=10):
    mesh = E.Mesh(N, M)
    xs = inputs.kl_samples(seed, 0, s, M)
    vals, b = mesh.assemble(s, to_dev(inputs.ensemble_layout(xs)))
    return mesh, xs, vals, b


def solve(torch, mesh, s, vals, b, x0, flags, tol=1e-10):
    x = x0.clone()
    work = torch.empty(E.cg_workspace_size(mesh.n, s), dtype=torch.uint8, device=gpu())
    it, rr, st, stats = E.cg(mesh.graph, s, vals, b, x, tol, 5000, work, flags=flags, check_every=4)
    return to_np(x).reshape(-1, s), it, rr, st, stats


@pytest.mark.parametrize("flags", [0, E.CG_SPLIT64, E.CG_DF64 | E.CG_GRAPH])
def test_fallback_is_bitwise_zero_guess(torch, flags):
    s = 4
    mesh, xs, vals, b = ensemble(torch, 8, s, 601)
    zero = torch.zeros(mesh.n * s, dtype=torch.float64, device=gpu())
    bad = to_dev(1e3 * inputs.random_vector(602, mesh.n * s))
    X0, it0, rr0, st0, s0 = solve(torch, mesh, s, vals, b, zero, flags)
    X1, it1, rr1, st1, s1 = solve(torch, mesh, s, vals, b, bad, flags | E.CG_GUESS_FALLBACK)
    assert s0.guess_fallbacks == 0 and s1.guess_fallbacks == s
    assert it0 == it1 and st0 == st1 == [0] * s and np.array_equal(X0, X1)


def test_fallback_per_member(torch):
    s = 8
    mesh, xs, vals, b = ensemble(torch, 9, s, 611)
    rm, col, ov, ob = oracle_members(9, 10, xs)
    good = []
    for e in range(s):
        xo, _, _, _ = O.cg(rm, col, ov[e], ob[e], tol=1e-13)
        good.append(xo * (1 + 1e-9 * inputs.random_vector(620 + e, mesh.n)))
    x0 = np.stack(good, axis=1)
    x0[:, 4:7] = 1e3 * inputs.random_vector(630, mesh.n * 3).reshape(-1, 3)
    x0[5, 7] = np.nan
    zero = torch.zeros(mesh.n * s, dtype=torch.float64, device=gpu())
    Xz, itz, _, _, _ = solve(torch, mesh, s, vals, b, zero, 0)
    Xg, itg, rrg, stg, stats = solve(torch, mesh, s, vals, b, to_dev(x0.reshape(-1)), E.CG_GUESS_FALLBACK)
    assert stats.guess_fallbacks == 4 and stg == [0] * s and max(rrg) <= 1e-10
    for e in range(4):
        assert itg[e] < itz[e] // 2, (e, itg[e], itz[e])
        xo = O.cg(rm, col, ov[e], ob[e], tol=1e-13)[0]
        assert np.linalg.norm(Xg[:, e] - xo) <= 1e-8 * np.linalg.norm(xo)
    for e in range(4, 8):
        assert itg[e] == itz[e] and np.array_equal(Xg[:, e], Xz[:, e])
    # without the fallback a non-finite start breaks down (status 6) in its
    # own member only
    Xn, itn, rrn, stn, _ = solve(torch, mesh, s, vals, b, to_dev(x0.reshape(-1)), 0)
    assert stn[7] == 6 and stn[:4] == [0] * 4


def test_fallback_in_batched_launch(torch):
    items, refs = [], []
    for N, s, seed in ((6, 4, 641), (8, 8, 642)):
        mesh, xs, vals, b = ensemble(torch, N, s, seed)
        zero = torch.zeros(mesh.n * s, dtype=torch.float64, device=gpu())
        refs.append(solve(torch, mesh, s, vals, b, zero, 0))
        x = to_dev(1e3 * inputs.random_vector(seed + 1, mesh.n * s))
        items.append((mesh.graph, s, vals, b, x))
    batch = E.Batch(items)
    work = torch.empty(batch.workspace_size(), dtype=torch.uint8, device=gpu())
    its, rrs, sts, stats = batch.solve(1e-10, 5000, work, flags=E.CG_GUESS_FALLBACK, check_every=4)
    assert stats.guess_fallbacks == 12
    for (g, s, vals, b, x), ref, it in zip(items, refs, its):
        assert it == ref[1] and np.array_equal(to_np(x).reshape(-1, s), ref[0])


# ------------------------------------------------------- end to end
def test_learned_guess_saves_iterations(torch, tmp_path):
    """16^3 mesh, M = 10: 512 training solves, POD 64 modes, the 10-256-256-64
    network; 64 fresh samples solved from zero and from the learned guess to
    the same tolerance."""
    N, M, s, tol = 16, 10, 32, 1e-8
    mesh = E.Mesh(N, M)
    xtr = inputs.kl_samples(inputs.SEED_GUESS_TRAIN, 0, 512, M)
    X, _ = collect(mesh, xtr, s=s, tol=tol)
    g = LearnedGuess(mesh.n)
    T = g.fit_basis(X)
    assert np.max(np.abs(to_np(g.Phi).T @ to_np(g.Phi) - np.eye(64))) <= 1e-12
    g.init_params()
    losses = g.train(xtr, T, epochs=1000)
    assert losses[-1] < 0.5 * losses[0], (losses[0], losses[-1])
    # checkpoint round trip
    g.save(str(tmp_path / "ck"))
    g2 = LearnedGuess.load(str(tmp_path / "ck"))
    assert torch.equal(g2.params, g.params) and torch.equal(g2.Phi32, g.Phi32) and \
        torch.equal(g2.step, g.step)
    xte = inputs.kl_samples(inputs.SEED_GUESS_TEST, 0, 64, M)
    work = torch.empty(E.cg_workspace_size(mesh.n, s), dtype=torch.uint8, device=gpu())
    it_zero, it_guess, fb = [], [], 0
    rm, col = O.graph(N)
    for j in range(0, 64, s):
        xi = to_dev(inputs.ensemble_layout(xte[j:j + s]))
        vals, b = mesh.assemble(s, xi)
        x = torch.zeros(mesh.n * s, dtype=torch.float64, device=gpu())
        it, rr, st, _ = E.cg(mesh.graph, s, vals, b, x, tol, 5000, work)
        assert st == [0] * s
        it_zero += it
        g2.predict(xi, s, x)
        it, rr, st, stats = E.cg(mesh.graph, s, vals, b, x, tol, 5000, work, flags=E.CG_GUESS_FALLBACK)
        assert st == [0] * s and max(rr) <= tol * 1.01
        it_guess += it
        fb += stats.guess_fallbacks
        X1 = to_np(x).reshape(-1, s)
        for e in (0, s - 1):
            v, bb = O.assemble(N, M, xte[j + e], rm, col)
            xo = O.cg(rm, col, v, bb, tol=1e-13)[0]
            assert np.linalg.norm(X1[:, e] - xo) <= 1e-7 * np.linalg.norm(xo)
    assert fb <= 6
    print("mean iterations zero %.2f learned %.2f fallbacks %d" % (np.mean(it_zero), np.mean(it_guess), fb))
    assert np.mean(it_guess) <= 0.85 * np.mean(it_zero), (np.mean(it_guess), np.mean(it_zero))
