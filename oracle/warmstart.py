"""Learned warm start: network, loss, gradient, Adam and the snapshot basis, in plain FP64.

Test infrastructure: part of the CPU oracle, see `oracle/__init__.py`.

The paper has no learned component (its PCG starts from x_0 = 0, Sec. 6); this module is the
definition the GPU warm-start kernels are checked against:
  * network: y = W_{L-1} h_{L-1} + b_{L-1}, h_{l+1} = tanh(W_l h_l + b_l), h_0 = x; parameters packed
    layer by layer as W_l (row-major, sizes[l+1] x sizes[l]) then b_l;
  * loss: L = (1/B) sum_n w_n ||y(x_n) - t_n||^2 over a batch of B rows;
  * gradient: reverse-mode chain rule of that loss, written out layer by layer;
  * Adam (Kingma and Ba 2015, Algorithm 1): m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
    theta <- theta - lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps);
  * basis: randomized subspace iteration (Halko, Martinsson and Tropp 2011, Alg. 4.4) on the rows of
    a snapshot matrix Y (n x m): Q = orth(Omega^T Y), then per power iteration P = orth(Q Y^T),
    Q = orth(P Y), where orth(Z) returns the rows of Q~ from Z^T = Q~ R with diag(R) > 0 (the
    unique thin QR factor), computed here by Householder QR (numpy) and a sign fix.
  * training-data preparation: Cholesky whitening of the features (G = F^T F / n + 1e-10 max diag(G),
    G = R^T R, W = R^{-1}, whitened features F W), the RMS of every target coordinate and the targets
    scaled by it, per-sample weights mean ||t||^2 / ||t_n||^2, and one stage of the cascade (the error
    the earlier stages left, rescaled to unit RMS per coordinate).
Pins: the gradient against central finite differences of the loss, the forward map against hand
values, Adam's first steps against their closed form, the basis against orthonormality, exact
reproduction of rank-K snapshot sets, and the SVD's dominant subspace; the whitened features' training
covariance is the identity and W is upper triangular; the scaled targets have unit RMS per coordinate;
the weights make every weighted sample norm equal; a cascade stage that removes a known part leaves
exactly the rest.
"""
import numpy as np


def layer_slices(sizes):
    """[(slice of W_l, shape), (slice of b_l)] for every layer of the packed parameter vector."""
    out = []
    off = 0
    for l in range(len(sizes) - 1):
        nw = sizes[l + 1] * sizes[l]
        out.append(((slice(off, off + nw), (sizes[l + 1], sizes[l])), slice(off + nw, off + nw + sizes[l + 1])))
        off += nw + sizes[l + 1]
    return out


def n_params(sizes):
    return sum(sizes[l + 1] * sizes[l] + sizes[l + 1] for l in range(len(sizes) - 1))


def unpack(theta, sizes):
    theta = np.asarray(theta, dtype=np.float64)
    return [(theta[ws].reshape(shape), theta[bs]) for (ws, shape), bs in layer_slices(sizes)]


def forward(theta, sizes, X):
    """Network outputs for the rows of X (B x sizes[0]) and the activations h_0 .. h_{L-1}."""
    layers = unpack(theta, sizes)
    h = np.asarray(X, dtype=np.float64)
    hs = [h]
    for l, (W, b) in enumerate(layers):
        z = h @ W.T + b
        h = np.tanh(z) if l + 1 < len(layers) else z
        hs.append(h)
    return h, hs


def loss(theta, sizes, X, T, w=None):
    Y, _ = forward(theta, sizes, X)
    R = Y - np.asarray(T, dtype=np.float64)
    w = np.ones(len(R)) if w is None else np.asarray(w, dtype=np.float64)
    return float(np.sum(w[:, None] * R * R) / len(R))


def loss_grad(theta, sizes, X, T, w=None):
    """(L, dL/dtheta) by the chain rule, one layer at a time from the output back."""
    layers = unpack(theta, sizes)
    Y, hs = forward(theta, sizes, X)
    B = len(Y)
    w = np.ones(B) if w is None else np.asarray(w, dtype=np.float64)
    R = Y - np.asarray(T, dtype=np.float64)
    L = float(np.sum(w[:, None] * R * R) / B)
    grad = np.zeros(n_params(sizes))
    dz = 2.0 * w[:, None] * R / B               # dL/dz of the last layer (no activation)
    for l in range(len(layers) - 1, -1, -1):
        (ws, shape), bs = layer_slices(sizes)[l]
        W, _ = layers[l]
        grad[ws] = (dz.T @ hs[l]).ravel()        # dL/dW_l = dz^T h_l
        grad[bs] = dz.sum(axis=0)                # dL/db_l
        if l > 0:
            dh = dz @ W                          # dL/dh_l
            dz = dh * (1.0 - hs[l] ** 2)         # tanh'(z) = 1 - tanh(z)^2
    return L, grad


def adam(theta, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t = 1 for the first); returns (theta, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def orth_rows(Z):
    """Rows of Q with Z = R^T Q, R upper triangular with a positive diagonal."""
    Qt, R = np.linalg.qr(np.asarray(Z, dtype=np.float64).T)
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return (Qt * s).T


def range_basis(Y, Omega, power_its=0):
    """Randomized subspace iteration on the rows of Y (n x m) with test matrix Omega (n x K)."""
    Y = np.asarray(Y, dtype=np.float64)
    Q = orth_rows(np.asarray(Omega, dtype=np.float64).T @ Y)
    for _ in range(power_its):
        P = orth_rows(Q @ Y.T)
        Q = orth_rows(P @ Y)
    return Q


def whiten(F, rel_shift=1e-10):
    """Cholesky whitening of the rows of F (n x K): returns (W, F W) with W = R^{-1}, where
    F^T F / n + rel_shift * max diag = R^T R, R upper triangular with a positive diagonal."""
    F = np.asarray(F, dtype=np.float64)
    n, K = F.shape
    G = F.T @ F / n
    G = G + rel_shift * np.max(np.diag(G)) * np.eye(K)
    R = np.linalg.cholesky(G).T          # G = L L^T, R = L^T
    W = np.linalg.inv(R)
    return W, F @ W


def target_scaling(T):
    """(so, T / so, w): the RMS of every column of T (n x K), the columns scaled to unit RMS, and the
    weights w_n = mean_r ||t_r||^2 / ||t_n||^2."""
    T = np.asarray(T, dtype=np.float64)
    so = np.maximum(np.sqrt(np.mean(T * T, axis=0)), 1e-300)
    sq = np.sum(T * T, axis=1)
    w = np.mean(sq) / np.maximum(sq, 1e-300)
    return so, T / so, w


def cascade_stage(resid, Y=None, scale_prev=None, T0=None):
    """One stage of the cascade: with T0 the first stage (resid = T0, scale = 1); otherwise
    resid - Y * scale_prev (the part the previous stage explains removed), scale = the RMS of every column
    of that residual. Returns (resid, scale, targets = resid / scale)."""
    if T0 is not None:
        r = np.array(T0, dtype=np.float64)
        scale = np.ones(r.shape[1])
    else:
        r = np.asarray(resid, dtype=np.float64) - np.asarray(Y, dtype=np.float64) * np.asarray(scale_prev)
        scale = np.maximum(np.sqrt(np.mean(r * r, axis=0)), 1e-30)
    return r, scale, r / scale
