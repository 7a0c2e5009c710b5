"""Pins of the warm-start oracle (network, loss, gradient, Adam, randomized basis).

The paper has no learned component; these pin the oracle's definitions against things other
than themselves: hand-computed network values, central finite differences of the loss, the closed
form of Adam's steps under a constant gradient, orthonormality, exact reproduction of rank-K
snapshot sets and the SVD's dominant subspace.
"""
import math

import numpy as np

from oracle import warmstart as W


def test_forward_hand_values():
    # 1 -> 1 -> 1: y = 2 tanh(0.5 x) + 1
    theta = np.array([0.5, 0.0, 2.0, 1.0])
    y, _ = W.forward(theta, [1, 1, 1], np.array([[1.0], [-2.0]]))
    assert abs(y[0, 0] - (2 * math.tanh(0.5) + 1)) < 1e-15
    assert abs(y[1, 0] - (2 * math.tanh(-1.0) + 1)) < 1e-15
    # one linear layer 2 -> 3: y = W x + b with W row-major
    theta = np.array([1, 2, 3, 4, 5, 6, 0.5, -0.5, 1.5], dtype=float)
    y, _ = W.forward(theta, [2, 3], np.array([[1.0, -1.0]]))
    assert np.allclose(y[0], [1 - 2 + 0.5, 3 - 4 - 0.5, 5 - 6 + 1.5], atol=0, rtol=0)


def test_loss_definition():
    theta = np.array([1, 0, 0, 1, 0, 0], dtype=float)  # identity 2 -> 2
    X = np.array([[1.0, 2.0], [3.0, -1.0]])
    T = np.array([[0.0, 2.0], [1.0, 1.0]])
    w = np.array([2.0, 0.5])
    # (2 (1^2 + 0^2) + 0.5 (2^2 + 2^2)) / 2
    assert abs(W.loss(theta, [2, 2], X, T, w) - (2 * 1 + 0.5 * 8) / 2) < 1e-15


def _fd_grad(theta, sizes, X, T, w, h=1e-6):
    g = np.zeros_like(theta)
    for i in range(len(theta)):
        tp = theta.copy()
        tm = theta.copy()
        tp[i] += h
        tm[i] -= h
        g[i] = (W.loss(tp, sizes, X, T, w) - W.loss(tm, sizes, X, T, w)) / (2 * h)
    return g


def _case(seed=0, sizes=(3, 5, 4, 2), B=7):
    rng = np.random.default_rng(seed)
    sizes = list(sizes)
    theta = rng.standard_normal(W.n_params(sizes)) * 0.7
    X = rng.standard_normal((B, sizes[0]))
    T = rng.standard_normal((B, sizes[-1]))
    w = rng.uniform(0.2, 2.0, size=B)
    return theta, sizes, X, T, w


def test_gradient_matches_central_differences():
    for seed, sizes in [(0, (3, 5, 4, 2)), (1, (2, 3)), (2, (4, 6, 6, 6, 3))]:
        theta, sizes, X, T, w = _case(seed, sizes)
        L, g = W.loss_grad(theta, sizes, X, T, w)
        assert abs(L - W.loss(theta, sizes, X, T, w)) < 1e-14
        gfd = _fd_grad(theta, sizes, X, T, w)
        assert np.abs(g - gfd).max() <= 1e-7 * np.abs(gfd).max()


def test_adam_constant_gradient_closed_form():
    # with a constant gradient the bias corrections make every step lr g / (|g| + eps)
    rng = np.random.default_rng(3)
    theta = rng.standard_normal(10)
    g = rng.standard_normal(10)
    m = np.zeros(10)
    v = np.zeros(10)
    th = theta.copy()
    for t in range(1, 6):
        th, m, v = W.adam(th, g, m, v, t, lr=1e-2)
        expect = theta - t * 1e-2 * g / (np.abs(g) + 1e-8)
        assert np.abs(th - expect).max() < 1e-12


def test_orth_rows_is_the_positive_qr_factor():
    rng = np.random.default_rng(4)
    Z = rng.standard_normal((6, 40))
    Q = W.orth_rows(Z)
    assert np.abs(Q @ Q.T - np.eye(6)).max() < 1e-14
    Rt = Z @ Q.T  # Z = R^T Q  =>  Z Q^T = R^T, lower triangular with a positive diagonal
    assert np.abs(np.triu(Rt, 1)).max() < 1e-13
    assert (np.diag(Rt) > 0).all()


def test_range_basis_reproduces_rank_K_snapshots():
    rng = np.random.default_rng(5)
    n, m, K = 40, 300, 8
    Y = rng.standard_normal((n, K)) @ rng.standard_normal((K, m))
    Om = rng.standard_normal((n, K))
    for q in (0, 1):
        Q = W.range_basis(Y, Om, q)
        assert np.abs(Q @ Q.T - np.eye(K)).max() < 1e-13
        assert np.linalg.norm(Y - Y @ Q.T @ Q) <= 1e-12 * np.linalg.norm(Y)


def test_range_basis_finds_the_dominant_singular_subspace():
    rng = np.random.default_rng(6)
    n, m, K = 60, 200, 6
    U, _ = np.linalg.qr(rng.standard_normal((n, n)))
    V, _ = np.linalg.qr(rng.standard_normal((m, n)))
    s = np.concatenate([np.linspace(10, 5, K), 1e-3 * np.ones(n - K)])
    Y = (U * s) @ V.T
    Q = W.range_basis(Y, rng.standard_normal((n, K)), 2)
    Vk = np.linalg.svd(Y, full_matrices=False)[2][:K]
    cosines = np.linalg.svd(Q @ Vk.T, compute_uv=False)
    assert 1 - cosines.min() < 1e-12


# ---- training-data preparation ----------------------------------------------------------------------
def _correlated(n, K, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((K, K)) * np.logspace(0, -3, K)  # strongly correlated, badly scaled columns
    return rng.standard_normal((n, K)) @ A.T


def test_whitened_features_have_identity_covariance():
    F = _correlated(500, 12, 1)
    Wm, Fw = W.whiten(F, rel_shift=0.0)
    assert np.allclose(np.triu(Wm), Wm, atol=0, rtol=0)          # W = R^{-1} is upper triangular
    assert np.all(np.diag(Wm) > 0)
    cov = Fw.T @ Fw / len(Fw)
    assert np.abs(cov - np.eye(12)).max() < 1e-8   # rounding times kappa(F^T F) ~ 1e6
    # the shift (1e-10 of the largest variance) perturbs the covariance by about shift / smallest variance:
    # 1e-8 for features whose variances span two decades
    rng = np.random.default_rng(3)
    F2 = rng.standard_normal((500, 12)) @ (rng.standard_normal((12, 12)) * np.logspace(0, -1, 12)).T
    _, Fs = W.whiten(F2)
    assert np.abs(Fs.T @ Fs / len(Fs) - np.eye(12)).max() < 1e-6
    # planted mistake: W^T instead of W whitens nothing
    assert np.abs((F @ Wm.T).T @ (F @ Wm.T) / len(F) - np.eye(12)).max() > 1e-1


def test_target_scaling_closed_forms():
    T = np.array([[3.0, 0.0], [4.0, 2.0]])
    so, Ts, w = W.target_scaling(T)
    assert np.allclose(so, [np.sqrt(12.5), np.sqrt(2.0)], rtol=1e-15)
    assert np.allclose(np.sqrt(np.mean(Ts * Ts, axis=0)), 1.0, rtol=1e-15)
    # ||t_1||^2 = 9, ||t_2||^2 = 20, mean 14.5: w = (14.5 / 9, 14.5 / 20), every weighted norm equals the mean
    assert np.allclose(w, [14.5 / 9, 14.5 / 20], rtol=1e-15)
    assert np.allclose(w * np.sum(T * T, axis=1), 14.5, rtol=1e-15)


def test_cascade_stage_removes_the_explained_part():
    rng = np.random.default_rng(2)
    T0 = rng.standard_normal((200, 6))
    r0, s0, t0 = W.cascade_stage(None, T0=T0)
    assert np.array_equal(r0, T0) and np.array_equal(s0, np.ones(6)) and np.array_equal(t0, T0)
    # a stage that predicted T0 - E exactly (with scale 1) leaves E, rescaled to unit RMS per column
    E = 1e-3 * rng.standard_normal((200, 6)) * np.arange(1, 7)
    r1, s1, t1 = W.cascade_stage(r0, Y=T0 - E, scale_prev=s0)
    assert np.allclose(r1, E, rtol=1e-12, atol=1e-15)
    assert np.allclose(s1, np.sqrt(np.mean(E * E, axis=0)), rtol=1e-12)
    assert np.allclose(np.sqrt(np.mean(t1 * t1, axis=0)), 1.0, rtol=1e-12)
