"""Planted mistakes in the oracle (on the CPU) must be caught by its pins.

Each test copies the oracle's state, plants one plausible error (a sign,
a dropped term, a transposed operand, a wrong power) and checks that the
corresponding pin fails by a wide margin. This shows the pins are sharp.
"""
import numpy as np

from oracle import direct, fd
from oracle.system import Discretization


def _mismatch(disc):
    A = disc.dense()
    Ad = direct.dense_A(disc)
    return np.abs(A - Ad).max() / np.abs(Ad).max()


def test_wrong_sign_of_W_is_caught():
    disc = Discretization([2, 3, 2], [2, 2], T=0.7, nu=1.3)
    assert _mismatch(disc) < 1e-12
    disc.Wsym = -disc.Wsym
    assert _mismatch(disc) > 1e-3


def test_dropped_cross_term_of_Bs_is_caught():
    disc = Discretization([2, 3, 2], [2, 2], T=0.7, nu=1.3)
    K2 = disc.sp[1]["K2"]
    all_terms = disc.terms()
    kept = [t for t in all_terms if not (np.allclose(t[1][1], K2) or np.allclose(t[1][1], K2.T))]
    assert len(kept) == len(all_terms) - 2
    disc.terms = lambda *a, **k: kept
    assert _mismatch(disc) > 1e-3


def test_transposed_eigenvectors_are_caught():
    disc = Discretization([4, 5, 6], [2, 3])
    P = fd.dense_P(disc)
    F = fd.FastDiagonalization(disc)
    r = np.random.default_rng(0).standard_normal(disc.N_dof) + 0j
    good = np.abs(F.apply(r) - np.linalg.solve(P, r)).max()
    F.U = [None] + [U.T for U in F.U[1:]]
    bad = np.abs(F.apply(r) - np.linalg.solve(P, r)).max()
    assert good < 1e-12 * np.abs(r).max() * 1e3 and bad > 1e3 * good


def test_lambda_instead_of_lambda_squared_is_caught():
    disc = Discretization([4, 5, 6], [2, 3])
    P = fd.dense_P(disc)
    F = fd.FastDiagonalization(disc)
    r = np.random.default_rng(1).standard_normal(disc.N_dof) + 0j
    ref = np.linalg.solve(P, r)
    F.H = lambda li, F=F: disc.Lt + disc.nu ** 2 * li * disc.Mt + disc.nu * li * disc.Wsym
    assert np.abs(F.apply(r) - ref).max() > 1e-3 * np.abs(ref).max()


def _mutated_loss_grad(old, new):
    """A copy of the oracle's gradient with one planted textual change."""
    import inspect
    from oracle import warmstart
    src = inspect.getsource(warmstart.loss_grad)
    assert old in src
    ns = dict(vars(warmstart))
    exec(src.replace(old, new), ns)
    return ns["loss_grad"]


def _fd_mismatch(grad_fn):
    from oracle import warmstart as W
    rng = np.random.default_rng(0)
    sizes = [3, 5, 4, 2]
    theta = rng.standard_normal(W.n_params(sizes)) * 0.7
    X = rng.standard_normal((7, 3))
    T = rng.standard_normal((7, 2))
    w = rng.uniform(0.2, 2.0, size=7)
    _, g = grad_fn(theta, sizes, X, T, w)
    gfd = np.zeros_like(theta)
    for i in range(len(theta)):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += 1e-6
        tm[i] -= 1e-6
        gfd[i] = (W.loss(tp, sizes, X, T, w) - W.loss(tm, sizes, X, T, w)) / 2e-6
    return np.abs(g - gfd).max() / np.abs(gfd).max()


def test_dropped_tanh_derivative_is_caught():
    assert _fd_mismatch(_mutated_loss_grad("dh * (1.0 - hs[l] ** 2)", "dh")) > 1e-2


def test_bias_gradient_taken_as_a_mean_is_caught():
    assert _fd_mismatch(_mutated_loss_grad("dz.sum(axis=0)", "dz.mean(axis=0)")) > 1e-2


def test_flipped_residual_sign_is_caught():
    assert _fd_mismatch(_mutated_loss_grad("dz = 2.0 * w[:, None] * R / B", "dz = -2.0 * w[:, None] * R / B")) > 1e-2


def test_missing_sample_weights_are_caught():
    assert _fd_mismatch(_mutated_loss_grad("dz = 2.0 * w[:, None] * R / B", "dz = 2.0 * R / B")) > 1e-2


def test_ultraweak_initial_term_with_flipped_sign_is_caught():
    from oracle import rhs as orhs
    from oracle import direct as odirect
    nu = 1.3
    u = lambda t, x: (1 + t ** 2) * x ** 2 * (1 - x) + 0j
    f = lambda t, x: 2j * t * x ** 2 * (1 - x) - nu * (1 + t ** 2) * (2 - 6 * x)
    u0 = lambda x: x ** 2 * (1 - x) + 0j
    disc = Discretization([3, 4], [2, 3], T=0.7, nu=nu, formulation="uw")
    G, w, pts = odirect.sb_matrix(disc)
    ref = (G.conj().T * w) @ np.array([u(*q) for q in pts])
    good = orhs.rhs_ultraweak(disc, f, u0)
    planted = orhs.rhs_ultraweak(disc, f, None) - (orhs.rhs_ultraweak(disc, None, u0))
    assert np.abs(good - ref).max() <= 1e-11 * np.abs(ref).max()
    assert np.abs(planted - ref).max() > 1e-2 * np.abs(ref).max()


def _grouped_mismatch(cross=2.0, g_sign=1.0):
    """The grouped additive-potential form (the mat-vec's Kronecker terms) against brute-force quadrature,
    with an optional planted mistake: the cross-term factor or the sign of M_v inside G_l."""
    from tests.test_oracle_pins import _pot_fn
    d, nu = 2, 1.3
    V = [[(lambda x: 1.5 * (x - .45) ** 2), (lambda x: 1 + 0 * x)],
         [(lambda x: 1 + 0 * x), (lambda x: 2.5 * (x - .45) ** 2)]]
    disc = Discretization([3, 4, 3], [2, 3], T=0.7, nu=nu, potential=V)
    M = [None] + [disc.sp[l]["M"] for l in (1, 2)]
    G, Al = [None], [None]
    for l in (1, 2):
        v = V[l - 1][l - 1]
        W = disc.weighted_space(l, v)
        W2 = disc.weighted_space(l, lambda x, v=v: v(x) * v(x))
        G.append(nu * disc.sp[l]["L"] + g_sign * W["M"])
        Al.append(nu ** 2 * disc.sp[l]["J"] + W2["M"] - nu * (W["K2"] + W["K2"].T))
    k = lambda a, b, c: np.kron(c, np.kron(b, a))
    A = k(disc.Lt, M[1], M[2]) + k(disc.Wsym, G[1], M[2]) + k(disc.Wsym, M[1], G[2])
    A = A + k(disc.Mt, Al[1], M[2]) + k(disc.Mt, M[1], Al[2]) + cross * k(disc.Mt, G[1], G[2])
    Ad = direct.dense_A(disc, _pot_fn(V))
    return np.abs(A - Ad).max() / np.abs(Ad).max()


def test_grouped_potential_form_mistakes_are_caught():
    assert _grouped_mismatch() < 1e-12
    assert _grouped_mismatch(cross=1.0) > 1e-3
    assert _grouped_mismatch(g_sign=-1.0) > 1e-3
