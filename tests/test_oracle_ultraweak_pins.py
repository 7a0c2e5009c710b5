"""Pins of the ultraweak formulation in the oracle (Sec. 4.4, Eq. uw-discrete-system).

The ultraweak method seeks u_h = S z_h with z_h in the space with final conditions W_h:
(S z_h, S w_h) = F(w_h) + i (u0, w_h(., 0)) for all w_h in W_h, F(w) = (f, w). Pinned against:
brute-force (d+1)-dimensional quadrature of the matrix on the final-condition basis; the identity
(u, S w) = (S u, w) + i (u(0), w(0)) for w(T) = 0, evaluated for exact solutions by brute-force
quadrature of (u, S B_i); Hermitian positive definiteness; and convergence of u_h = S z_h, which is
the L2(Q)-orthogonal projection of u onto S(W_h).
"""
import numpy as np

from oracle import direct, rhs
from oracle.system import Discretization


def test_kronecker_matrix_matches_brute_force_on_the_final_condition_space():
    for n_el, p, pot in [([3, 4], [2, 3], None), ([2, 3, 2], [2, 2], None),
                         ([3, 3], [3, 2], [[lambda x: 2.0 + np.cos(3 * x)]])]:
        disc = Discretization(n_el, p, T=0.7, nu=1.3, potential=pot, formulation="uw")
        A = disc.dense()
        V = None
        if pot:
            V = lambda x: 2.0 + np.cos(3 * x[0])
        Ad = direct.dense_A(disc, V)
        assert np.abs(A - Ad).max() <= 1e-12 * np.abs(Ad).max()
        assert np.abs(A - A.conj().T).max() <= 1e-12 * np.abs(A).max()
        assert np.linalg.eigvalsh(A).min() > 0


def test_time_restriction_keeps_the_initial_and_drops_the_final_function():
    ls = Discretization([4, 3], [2, 2], formulation="ls")
    uw = Discretization([4, 3], [2, 2], formulation="uw")
    assert ls.n == uw.n
    # the initial function is the only one with b(0) != 0; the final one the only one with b(T) != 0
    t_ls = rhs.tables(ls, 0, pts=[0.0, 1.0])[0]
    t_uw = rhs.tables(uw, 0, pts=[0.0, 1.0])[0]
    assert np.allclose(t_ls[0], 0) and abs(t_ls[1, -1] - 1) < 1e-14
    assert abs(t_uw[0, 0] - 1) < 1e-14 and np.allclose(t_uw[1], 0)


def test_rhs_equals_u_against_S_of_the_test_functions():
    # exact solutions with polynomial space factors, so the Gauss rule integrates both sides exactly
    nu = 1.3
    cases = [
        # u = (1 + t^2) x^2 (1 - x): S u = 2 i t x^2 (1 - x) - nu (1 + t^2)(2 - 6 x)
        (lambda t, x: (1 + t ** 2) * x ** 2 * (1 - x) + 0j,
         lambda t, x: 2j * t * x ** 2 * (1 - x) - nu * (1 + t ** 2) * (2 - 6 * x),
         lambda x: x ** 2 * (1 - x) + 0j),
        # u = (1 - i t + t^3) x (1 - x): S u = (1 + 3 i t^2) x (1 - x) + 2 nu (1 - i t + t^3)
        (lambda t, x: (1 - 1j * t + t ** 3) * x * (1 - x),
         lambda t, x: (1 + 3j * t ** 2) * x * (1 - x) + 2 * nu * (1 - 1j * t + t ** 3),
         lambda x: x * (1 - x) + 0j),
    ]
    for u, f, u0 in cases:
        disc = Discretization([3, 4], [2, 3], T=0.7, nu=nu, formulation="uw")
        b = rhs.rhs_ultraweak(disc, f, u0)
        G, w, pts = direct.sb_matrix(disc)
        ref = (G.conj().T * w) @ np.array([u(*q) for q in pts])
        assert np.abs(b - ref).max() <= 1e-11 * np.abs(ref).max()


def test_ultraweak_solution_converges():
    u = lambda t, x: np.exp(1j * np.pi ** 2 * t) * np.sin(np.pi * x)
    u0 = lambda x: np.sin(np.pi * x) + 0j
    errs = []
    for n in (8, 16):
        disc = Discretization([n, n], [3, 3], formulation="uw")
        z = np.linalg.solve(disc.dense(), rhs.rhs_ultraweak(disc, None, u0))
        S, pts, wts = rhs.apply_S_on_grid(disc, z, extra=3)
        U = u(pts[0][None, :], pts[1][:, None])
        W = np.outer(wts[1], wts[0])
        errs.append(np.sqrt(np.sum(W * np.abs(S - U) ** 2) / np.sum(W * np.abs(U) ** 2)))
    assert errs[1] < 2e-2
    assert np.log2(errs[0] / errs[1]) > 2.5


def test_fast_diagonalization_inverts_p_hat_on_the_final_condition_space():
    from oracle import fd
    disc = Discretization([4, 5, 6], [2, 3], formulation="uw")
    P = fd.dense_P(disc)
    F = fd.FastDiagonalization(disc)
    rng = np.random.default_rng(0)
    r = rng.standard_normal(disc.N_dof) + 1j * rng.standard_normal(disc.N_dof)
    ref = np.linalg.solve(P, r)
    assert np.abs(F.apply(r) - ref).max() <= 1e-12 * np.abs(ref).max()
