"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU needed).

Each test checks the oracle against something other than itself: closed forms
of cardinal B-splines, integration-by-parts identities, brute-force
quadrature of the sesquilinear form, the assembled dense preconditioner, a
dense direct solve, the paper's printed tables, and convergence rates.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import bspline, matrices, direct, fd, pcg, rhs, norms
from oracle.system import Discretization

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([float(v) for v in line.split()])
    return rows


# --------------------------------------------------------------------------------------------- basis
@pytest.mark.parametrize("p", [1, 2, 3, 4, 6])
def test_partition_of_unity_and_derivatives(p):
    knots = bspline.open_uniform_knots(p, 7)
    x = np.linspace(0, 1, 301)
    D = bspline.basis_all(knots, p, x, nder=2)
    assert D.shape[2] == 7 + p
    np.testing.assert_allclose(D[0].sum(axis=1), 1.0, atol=1e-14)
    np.testing.assert_allclose(D[1].sum(axis=1), 0.0, atol=1e-11)
    np.testing.assert_allclose(D[2].sum(axis=1), 0.0, atol=1e-9)
    assert (D[0] >= -1e-15).all()
    # open knot vector: interpolation at the end points
    assert D[0][0, 0] == pytest.approx(1.0) and D[0][-1, -1] == pytest.approx(1.0)


def _cardinal(n, s, x):
    """s-th derivative of the cardinal B-spline of degree n (support [0, n+1]) by its truncated-power form."""
    tot = 0.0
    for k in range(n + 2):
        if x - k > 0:
            tot += (-1) ** k * math.comb(n + 1, k) * (x - k) ** (n - s)
    return tot / math.factorial(n - s)


@pytest.mark.parametrize("p", [2, 3, 4])
def test_interior_entries_match_cardinal_autocorrelation(p):
    """Interior rows: M = h N_{2p+1}, L = -N''_{2p+1}/h, J = N''''_{2p+1}/h^3, K = -N'_{2p+1} at p+1+k."""
    n_el = 16
    h = 1.0 / n_el
    F = matrices.assemble_1d(p, n_el, 1.0)
    i = 8
    for k in range(-p, p + 1):
        c = p + 1 + k
        assert F["M"][i, i + k] == pytest.approx(h * _cardinal(2 * p + 1, 0, c), rel=1e-12, abs=1e-15)
        assert F["L"][i, i + k] == pytest.approx(-_cardinal(2 * p + 1, 2, c) / h, rel=1e-11, abs=1e-11)
        assert F["J"][i, i + k] == pytest.approx(_cardinal(2 * p + 1, 4, c) / h ** 3, rel=1e-10, abs=1e-8)
        assert F["K"][i, i + k] == pytest.approx(-_cardinal(2 * p + 1, 1, c), rel=1e-12, abs=1e-13)


@pytest.mark.parametrize("p,n_el,length", [(2, 5, 1.0), (3, 9, 2.0), (4, 6, 0.7)])
def test_global_identities(p, n_el, length):
    F = matrices.assemble_1d(p, n_el, length)
    m = n_el + p
    knots = bspline.open_uniform_knots(p, n_el)
    # row sums of M: int b_i = length (xi_{i+p+1} - xi_i) / (p + 1)
    np.testing.assert_allclose(F["M"].sum(axis=1), length * (knots[p + 1:p + 1 + m] - knots[:m]) / (p + 1), rtol=1e-13)
    # derivatives of the partition of unity vanish
    np.testing.assert_allclose(F["L"].sum(axis=1), 0, atol=1e-10)
    np.testing.assert_allclose(F["K"].sum(axis=1), 0, atol=1e-12)
    np.testing.assert_allclose(F["J"].sum(axis=1), 0, atol=1e-7 * np.abs(F["J"]).max())
    # int (b_i b_j)' = b_i b_j |_0^length: K + K^T = e_m e_m^T - e_1 e_1^T
    E = np.zeros((m, m))
    E[-1, -1], E[0, 0] = 1.0, -1.0
    np.testing.assert_allclose(F["K"] + F["K"].T, E, atol=1e-13)
    # time restriction (drop the first function): K_t + K_t^T = e_{n_t} e_{n_t}^T
    Kt = matrices.restrict_time(F["K"])
    E2 = np.zeros_like(Kt)
    E2[-1, -1] = 1.0
    np.testing.assert_allclose(Kt + Kt.T, E2, atol=1e-13)
    # space restriction (zero boundary values): int b_j'' b_i = - int b_j' b_i'
    np.testing.assert_allclose(matrices.restrict_space(F["K2"]), -matrices.restrict_space(F["L"]), atol=1e-10 * np.abs(F["L"]).max())
    # symmetric positive definiteness of the restricted mass and stiffness
    assert np.linalg.eigvalsh(matrices.restrict_space(F["M"])).min() > 0
    assert np.linalg.eigvalsh(matrices.restrict_space(F["L"])).min() > 0
    assert np.linalg.eigvalsh(matrices.restrict_time(F["L"])).min() > 0


# ------------------------------------------------------------------------------------------- system
def _pot_fn(terms):
    return lambda x: sum(np.prod([t[l](x[l]) for l in range(len(x))]) for t in terms)


CASES = [
    ([3, 3], [2, 2], None),
    ([3, 4], [1, 3], None),
    ([2, 3, 2], [2, 2], None),
    ([2, 2, 3], [2, 3], "rank2"),
    ([3, 3], [2, 3], "rank1"),
    ([1, 2, 2, 2], [1, 2], None),
]


def _potential(kind, d):
    if kind is None:
        return None
    if kind == "rank1":
        return [[(lambda x: 3 * (x - .5) ** 2 + 0.2) for _ in range(d)]]
    return [[(lambda x: 2 * (x - .5) ** 2), (lambda x: 1 + 0 * x)],
            [(lambda x: 1 + 0 * x), (lambda x: np.exp(-(x - 0.4) ** 2 / 0.1))]]


def _additive_A(disc, V):
    """A for V = sum_l v_l(x_l) in the grouped form the mat-vec planner uses:
    L_t (x) M..M + sum_l W (x) G_l + sum_l M_t (x) A_l + 2 sum_{l<k} M_t (x) G_l (x) G_k, with
    G_l = nu L + M_{v_l} and A_l = nu^2 J + M_{v_l^2} - nu (K2_{v_l} + K2_{v_l}^T)."""
    d, nu = disc.d, disc.nu
    M = [None] + [disc.sp[l]["M"] for l in range(1, d + 1)]
    G, Al = [None], [None]
    for l in range(1, d + 1):
        (v,) = [t[l - 1] for t in V if np.any(t[l - 1](np.linspace(0, 1, 7)) != 1.0)]
        W = disc.weighted_space(l, v)
        W2 = disc.weighted_space(l, lambda x, v=v: v(x) * v(x))
        G.append(nu * disc.sp[l]["L"] + W["M"])
        Al.append(nu ** 2 * disc.sp[l]["J"] + W2["M"] - nu * (W["K2"] + W["K2"].T))

    def kron(f):
        K = f[0]
        for l in range(1, d + 1):
            K = np.kron(f[l], K)
        return K
    A = kron([disc.Lt] + M[1:])
    for l in range(1, d + 1):
        f = [disc.Wsym] + M[1:]
        f[l] = G[l]
        A = A + kron(f)
        f = [disc.Mt] + M[1:]
        f[l] = Al[l]
        A = A + kron(f)
        for k in range(l + 1, d + 1):
            f = [disc.Mt] + M[1:]
            f[l], f[k] = G[l], G[k]
            A = A + 2 * kron(f)
    return A


@pytest.mark.parametrize("n_el,p", [([3, 4, 3], [2, 3]), ([2, 3, 2, 3], [2, 2]), ([4, 5], [3, 2])])
def test_additive_potential_grouping_equals_bruteforce_quadrature(n_el, p):
    """For an additive potential the cross terms of the expansion collapse to 2 G_l (x) G_k, because
    K2 + K2^T = -2 L for spatial functions vanishing on the boundary: the grouped form is A itself."""
    d = len(n_el) - 1
    V = [[(lambda x, s=1.5 + r: s * (x - .45) ** 2) if l == r else (lambda x: 1 + 0 * x) for l in range(d)]
         for r in range(d)]
    disc = Discretization(n_el, p, T=0.7, nu=1.3, potential=V)
    Ad = direct.dense_A(disc, _pot_fn(V))
    assert np.abs(_additive_A(disc, V) - Ad).max() <= 1e-12 * np.abs(Ad).max()
    for l in range(1, d + 1):
        K2, L = disc.sp[l]["K2"], disc.sp[l]["L"]
        assert np.abs(K2 + K2.T + 2 * L).max() <= 1e-13 * np.abs(L).max()


@pytest.mark.parametrize("n_el,p,pot", CASES)
def test_kronecker_A_equals_bruteforce_quadrature(n_el, p, pot):
    d = len(n_el) - 1
    P = _potential(pot, d)
    disc = Discretization(n_el, p, T=0.7, nu=1.3, potential=P)
    A = disc.dense()
    Ad = direct.dense_A(disc, _pot_fn(P) if P else None)
    assert np.abs(A - Ad).max() <= 1e-12 * np.abs(Ad).max()
    # Hermitian positive definite (the paper's "symmetric positive definite")
    assert np.abs(A - A.conj().T).max() <= 1e-13 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0
    # matrix-free application by mode products equals the dense matrix
    x = np.random.default_rng(0).standard_normal(disc.N_dof) * (1 + 0.5j)
    np.testing.assert_allclose(disc.apply(x), A @ x, rtol=0, atol=1e-12 * np.abs(A).max() * np.abs(x).max())


def test_load_vector_equals_bruteforce():
    P = _potential("rank1", 2)
    disc = Discretization([2, 3, 2], [2, 2], T=0.9, nu=0.8, potential=P)
    f = lambda t, x1, x2: np.exp(1j * (t + 2 * x1)) * (1 + x2 ** 2)
    b1 = rhs.load_vector(disc, f)
    b2 = direct.load_vector(disc, lambda q: f(q[0], q[1], q[2]), _pot_fn(P))
    np.testing.assert_allclose(b1, b2, rtol=0, atol=1e-13 * np.abs(b2).max())


# --------------------------------------------------------------------------------------------- FD
@pytest.mark.parametrize("n_el,p,nu,T", [([5, 7], [2, 3], 1.0, 1.0), ([4, 5, 6], [2, 3], 1.0, 1.0),
                                         ([3, 4, 3, 5], [3, 2], 0.6, 1.7), ([6, 4, 4], [1, 4], 2.0, 0.5)])
def test_fd_equals_dense_inverse_of_P(n_el, p, nu, T):
    disc = Discretization(n_el, p, T=T, nu=nu)
    P = fd.dense_P(disc)
    assert np.abs(P - P.conj().T).max() <= 1e-12 * np.abs(P).max()
    F = fd.FastDiagonalization(disc)
    for l in range(1, disc.d + 1):
        U = F.U[l]
        np.testing.assert_allclose(U.T @ disc.sp[l]["M"] @ U, np.eye(disc.n[l]), atol=1e-12)
        np.testing.assert_allclose(U.T @ disc.sp[l]["L"] @ U, np.diag(F.lam[l]), atol=1e-10 * F.lam[l].max())
    r = np.random.default_rng(3).standard_normal(disc.N_dof) + 1j * np.random.default_rng(4).standard_normal(disc.N_dof)
    s_dense = np.linalg.solve(P, r)
    s_fd = F.apply(r)
    assert np.abs(s_fd - s_dense).max() <= 1e-12 * np.abs(s_dense).max()


def test_kappa_U_table():
    """Table cond_number_space: kappa_2(U_l) depends on p only (checked at n_el = 32 and 64)."""
    for p, kappa in _golden("kappa_U_table.txt"):
        for n_el in (32, 64):
            disc = Discretization([2, n_el], [2, int(p)])
            k = fd.FastDiagonalization(disc).kappa_U(1)
            assert float(f"{k:.2g}") == pytest.approx(kappa), (p, n_el, k)
            # the factorization's defining property: kappa_2(U) = sqrt(kappa_2(M))
            assert k == pytest.approx(math.sqrt(np.linalg.cond(disc.sp[1]["M"])), rel=1e-8)


def test_spectral_equivalence_of_Bs_and_LML():
    """Fig. spectral_equivalence: eig((L M^{-1} L)^{-1} B_s) clustered near 1, stable under refinement."""
    for p in (2, 3, 4):
        spans = []
        for n_el in (8, 16, 32):
            disc = Discretization([2, n_el, n_el], [2, p])
            M1, L1, J1, K2 = (disc.sp[1][k] for k in ("M", "L", "J", "K2"))
            Ms, Ls = np.kron(M1, M1), np.kron(L1, M1) + np.kron(M1, L1)
            Bs = np.kron(J1, M1) + np.kron(M1, J1) + np.kron(K2.T, K2) + np.kron(K2, K2.T)
            ev = scipy.linalg.eigh(Bs, Ls.T @ np.linalg.solve(Ms, Ls), eigvals_only=True)
            spans.append((ev.min(), ev.max()))
        lo, hi = np.array(spans).T
        assert lo.min() > 0.99 and hi.max() < 2.0
        assert hi.max() - hi.min() < 0.05


# --------------------------------------------------------------------------------------------- PCG
def test_pcg_matches_dense_direct_solve():
    P = _potential("rank1", 2)
    disc = Discretization([4, 5, 4], [2, 3], potential=P)
    A = disc.dense()
    F = fd.FastDiagonalization(disc)
    b = np.random.default_rng(7).standard_normal(disc.N_dof) + 0.3j
    x, it, rr, _ = pcg.pcg(disc.apply, F.apply, b, tol=1e-13, maxit=200)
    xd = np.linalg.solve(A, b)
    assert np.abs(x - xd).max() <= 1e-10 * np.abs(xd).max()
    xf, itf, _, _ = pcg.pcg(disc.apply, F.apply, b, tol=1e-13, maxit=200, flexible=True)
    assert np.abs(xf - xd).max() <= 1e-10 * np.abs(xd).max()
    # V = 0: P-hat differs from A only through B_s vs L M^{-1} L, so PCG converges in few steps
    disc0 = Discretization([4, 5, 4], [2, 3])
    _, it0, _, _ = pcg.pcg(disc0.apply, fd.FastDiagonalization(disc0).apply, b, tol=1e-8)
    assert it0 <= 12


OM = 0.2
AMP = (2 / OM ** 2) ** 0.25


def _u_tw(t, x1, x2):
    return AMP * np.exp(-1j * (x1 ** 2 + x2 ** 2 + t ** 2) / OM ** 2)


def _f_tw(t, x1, x2):
    return AMP * (4j / OM ** 2 + 4 * (x1 ** 2 + x2 ** 2) / OM ** 4 + 2 * t / OM ** 2) * np.exp(-1j * (x1 ** 2 + x2 ** 2 + t ** 2) / OM ** 2)


def test_travelling_wave_forcing_is_S_of_u():
    """The printed forcing of Sec. 6.2 equals i u_t - Delta u (nu = 1), checked by finite differences."""
    t, x1, x2, e = 0.37, 0.21, 0.66, 1e-4
    ut = (_u_tw(t + e, x1, x2) - _u_tw(t - e, x1, x2)) / (2 * e)
    lap = sum((_u_tw(t, *(np.array([x1, x2]) + e * np.eye(2)[k])) - 2 * _u_tw(t, x1, x2)
               + _u_tw(t, *(np.array([x1, x2]) - e * np.eye(2)[k]))) / e ** 2 for k in range(2))
    assert abs(1j * ut - lap - _f_tw(t, x1, x2)) < 1e-4 * abs(_f_tw(t, x1, x2))


@pytest.mark.parametrize("p,n_el,iters", [(int(a), int(b), int(c)) for a, b, c in _golden("table1_iterations.txt") if b <= 16])
def test_table1_iteration_counts(p, n_el, iters):
    """Table 1: P-hat-CG iterations on the travelling wave (tolerance 1e-8, zero initial guess)."""
    disc = Discretization([n_el, n_el, n_el], [p, p])
    b, _ = rhs.full_lifting(disc, _u_tw, _f_tw)
    F = fd.FastDiagonalization(disc)
    _, it, rr, _ = pcg.pcg(disc.apply, F.apply, b, tol=1e-8, maxit=200)
    assert rr <= 1e-8
    assert abs(it - iters) <= 1


# ------------------------------------------------------------------------------ discretisation error
def _rates(u, f, u0, p, meshes=(8, 16, 32)):
    errs = []
    for n_el in meshes:
        disc = Discretization([n_el, n_el], [p, p])
        b, c = rhs.rhs_initial(disc, f, u0)
        x, _, _, _ = pcg.pcg(disc.apply, fd.FastDiagonalization(disc).apply, b, tol=1e-12)
        errs.append(norms.errors(disc, rhs.embed_solution(disc, x, c=c), u, f if f else (lambda t, x: 0 * t * x))[1])
    e = np.array(errs)
    return np.log2(e[:-1] / e[1:])


@pytest.mark.parametrize("p", [2, 3])
def test_convergence_rate_initial_datum(p):
    """Remark 1: V-norm error O(h^{p-1}); u = exp(i pi^2 t) sin(pi x) solves S u = 0 with u0 = sin(pi x)."""
    u = lambda t, x: np.exp(1j * np.pi ** 2 * t) * np.sin(np.pi * x)
    rates = _rates(u, None, lambda x: np.sin(np.pi * x), p)
    assert rates[-1] >= p - 1 - 0.15


@pytest.mark.parametrize("p", [2, 3])
def test_convergence_rate_modal_forcing(p):
    """Sec. 6.1 modal example with M = 1: f = e^{i pi^2 t} e_1, u = -i t e^{i pi^2 t} e_1, e_1 = sqrt(2) sin(pi x)."""
    e1 = lambda x: np.sqrt(2) * np.sin(np.pi * x)
    u = lambda t, x: -1j * t * np.exp(1j * np.pi ** 2 * t) * e1(x)
    f = lambda t, x: np.exp(1j * np.pi ** 2 * t) * e1(x)
    rates = _rates(u, f, None, p)
    assert rates[-1] >= p - 1 - 0.15
