"""Pins of the oracle's potential-aware preconditioner P_V (an extension of Eq. prec_definition to
S_V = i d_t + sum_l H_l, H_l = -nu d_ll + v_l, for potentials that are sums of one-direction factors):

* G_l = nu L_l + M_{v_l} against the Galerkin matrix of H_l by brute force (SciPy B-splines, numpy's
  Gauss-Legendre rule, Dirichlet-reduced basis: (H_l b_j, b_i) = nu (b_j', b_i') + (v_l b_j, b_i));
* Algorithm 1 with the eigenpairs of (G_l, M_l) against the dense inverse of P_V assembled from its
  definition (1D+t, 2D+t, 3D+t);
* V = 0 gives the paper's P-hat; P_V is Hermitian positive definite; a product potential is rejected.
"""
import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle import fd
from oracle.system import Discretization


def _basis(p, n_el, x, der):
    t = np.concatenate([np.zeros(p), np.linspace(0.0, 1.0, n_el + 1), np.ones(p)])
    m = n_el + p
    out = np.zeros((len(x), m))
    for j in range(m):
        c = np.zeros(m)
        c[j] = 1.0
        b = BSpline(t, c, p, extrapolate=False)
        out[:, j] = (b.derivative(der) if der else b)(x)
    return np.nan_to_num(out)


def _galerkin_H(p, n_el, nu, v):
    """(H b_j, b_i) on (0,1) for the basis without its two end functions, by Gauss-Legendre quadrature
    with p + 3 points per element (exact for the polynomial parts; v is a quadratic below)."""
    g, w = np.polynomial.legendre.leggauss(p + 3)
    h = 1.0 / n_el
    x = np.concatenate([(e + 0.5 * (g + 1.0)) * h for e in range(n_el)])
    wt = np.tile(0.5 * h * w, n_el)
    B0, B1 = _basis(p, n_el, x, 0)[:, 1:-1], _basis(p, n_el, x, 1)[:, 1:-1]
    vv = v(x) if v is not None else np.zeros_like(x)
    return nu * (B1.T * wt) @ B1 + (B0.T * (wt * vv)) @ B0


def _additive(d, shift=0.0):
    return [[(lambda x, s=1.5 + r + shift: s * (x - .45) ** 2) if l == r else (lambda x: 1 + 0 * x)
             for l in range(d)] for r in range(d)]


@pytest.mark.parametrize("n_el,p,nu", [([3, 5], [2, 3], 1.0), ([2, 4, 3], [2, 2], 1.3), ([2, 3, 2, 4], [1, 3], 0.8)])
def test_spatial_operators_are_the_galerkin_matrices_of_H_l(n_el, p, nu):
    d = len(n_el) - 1
    V = _additive(d)
    disc = Discretization(n_el, p, T=0.9, nu=nu, potential=V)
    G = fd.spatial_operators(disc)
    for l in range(1, d + 1):
        ref = _galerkin_H(disc.p[l], n_el[l], nu, V[l - 1][l - 1])
        assert np.abs(G[l] - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("n_el,p,nu,T", [([4, 5], [2, 3], 1.0, 1.0), ([3, 4, 3], [2, 2], 1.3, 0.7),
                                         ([2, 2, 3, 2], [2, 3], 0.8, 1.2)])
def test_potential_fd_equals_dense_inverse_of_P_V(n_el, p, nu, T):
    d = len(n_el) - 1
    disc = Discretization(n_el, p, T=T, nu=nu, potential=_additive(d))
    P = fd.dense_P_potential(disc)
    assert np.abs(P - P.conj().T).max() <= 1e-13 * np.abs(P).max()
    assert np.linalg.eigvalsh(P).min() > 0
    F = fd.PotentialFastDiagonalization(disc)
    r = np.random.default_rng(3).standard_normal(disc.N_dof) * (1 - 0.4j)
    ref = np.linalg.solve(P, r)
    assert np.abs(F.apply(r) - ref).max() <= 1e-11 * np.abs(ref).max()


def test_without_potential_it_is_p_hat():
    disc = Discretization([3, 4, 5], [2, 3], T=0.8, nu=1.1)
    P = fd.dense_P(disc)
    assert np.abs(fd.dense_P_potential(disc) - P).max() <= 1e-13 * np.abs(P).max()
    r = np.random.default_rng(4).standard_normal(disc.N_dof) + 0.5j
    a = fd.PotentialFastDiagonalization(disc).apply(r)
    b = fd.FastDiagonalization(disc).apply(r)
    assert np.abs(a - b).max() <= 1e-11 * np.abs(b).max()


def test_product_potential_is_rejected():
    bump = [[(lambda x: np.exp(-(x - .5) ** 2 / .05)) for _ in range(2)]]
    disc = Discretization([3, 4, 4], [2, 2], potential=bump)
    with pytest.raises(ValueError):
        fd.spatial_operators(disc)
    two_in_one = [[(lambda x: x ** 2), (lambda x: 1 + 0 * x)], [(lambda x: 1 + x), (lambda x: 1 + 0 * x)]]
    disc = Discretization([3, 4, 4], [2, 2], potential=two_in_one)
    with pytest.raises(ValueError):
        fd.spatial_operators(disc)


def test_fewer_iterations_than_p_hat_on_the_harmonic_workload_family():
    """2D+t p=3, harmonic V, wavepacket datum (the 64^2 x 64 benchmark workload at n_el = 16): PCG to 1e-8
    with P_V takes 8 iterations where P-hat takes 11, and both give the same solution."""
    from inputs import CONFIGS, potential, initial_factors, product_fn
    from oracle import pcg, rhs
    cfg = dict(CONFIGS["c2"])
    cfg["n_el"] = [16, 16, 16]
    disc = Discretization(cfg["n_el"], [cfg["p"]] * 3, T=cfg["T"], nu=cfg["nu"], potential=potential(cfg))
    b, _ = rhs.rhs_initial(disc, None, product_fn(initial_factors(cfg)))
    x0, it0, _, _ = pcg.pcg(disc.apply, fd.FastDiagonalization(disc).apply, b, tol=1e-8, maxit=200)
    x1, it1, _, _ = pcg.pcg(disc.apply, fd.PotentialFastDiagonalization(disc).apply, b, tol=1e-8, maxit=200)
    assert (it0, it1) == (11, 8)
    assert np.linalg.norm(x1 - x0) <= 1e-6 * np.linalg.norm(x0)


# ---- the ANOVA approximation for products of factors (approximate=True) ------------------------------

def test_anova_form_equals_the_exact_one_for_an_additive_potential():
    """The ANOVA terms of V = sum_l v_l are v_l plus constants summing to zero: the Kronecker sum H_s, hence P_V,
    is unchanged."""
    disc = Discretization([3, 4, 3, 2], [2, 2], T=0.8, nu=1.2, potential=_additive(3))
    P = fd.dense_P_potential(disc)
    assert np.abs(fd.dense_P_potential(disc, approximate=True) - P).max() <= 1e-12 * np.abs(P).max()


def test_anova_terms_of_a_polynomial_product_match_closed_form_means():
    """V = (1 + x1)(2 - x2^2): means 3/2 and 5/3, E[V] = 5/2, g_1 = (5/3)(1 + x) - 5/4, g_2 = (3/2)(2 - x^2) - 5/4."""
    V = [[(lambda x: 1.0 + x), (lambda x: 2.0 - x ** 2)]]
    disc = Discretization([3, 4, 5], [2, 3], nu=0.9, potential=V)
    G = fd.spatial_operators(disc, approximate=True)
    g = [None, lambda x: 5.0 / 3.0 * (1.0 + x) - 1.25, lambda x: 1.5 * (2.0 - x ** 2) - 1.25]
    for l in (1, 2):
        ref = 0.9 * disc.sp[l]["L"] + disc.weighted_space(l, g[l])["M"]
        assert np.abs(G[l] - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("n_el,p", [([4, 5, 4], [2, 3]), ([2, 3, 2, 3], [2, 2])])
def test_anova_fd_equals_dense_inverse_for_a_product_potential(n_el, p):
    d = len(n_el) - 1
    bump = [[(lambda x: 2.0 * np.exp(-(x - .5) ** 2 / .05)) for _ in range(d)]]
    disc = Discretization(n_el, p, T=0.9, nu=1.1, potential=bump)
    P = fd.dense_P_potential(disc, approximate=True)
    assert np.linalg.eigvalsh(P).min() > 0
    r = np.random.default_rng(5).standard_normal(disc.N_dof) * (1 + 0.3j)
    ref = np.linalg.solve(P, r)
    got = fd.PotentialFastDiagonalization(disc, approximate=True).apply(r)
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


def test_anova_preconditioner_on_the_bump_workload_family():
    """3D+t p = 2, Gaussian bump, wavepacket datum at 16 x 8^3 elements: PCG to 1e-8 with the ANOVA P_V takes
    8 iterations where P-hat takes 9 (16 x 16^3: 11 against 14; 48 x 24^3: 11 against 16)."""
    from inputs import CONFIGS, potential, initial_factors, product_fn
    from oracle import pcg, rhs
    cfg = dict(CONFIGS["c3p2_bump"])
    cfg["n_el"] = [16, 8, 8, 8]
    disc = Discretization(cfg["n_el"], [cfg["p"]] * 4, T=cfg["T"], nu=cfg["nu"], potential=potential(cfg))
    b, _ = rhs.rhs_initial(disc, None, product_fn(initial_factors(cfg)))
    _, it0, _, _ = pcg.pcg(disc.apply, fd.FastDiagonalization(disc).apply, b, tol=1e-8, maxit=200)
    _, it1, _, _ = pcg.pcg(disc.apply, fd.PotentialFastDiagonalization(disc, approximate=True).apply, b, tol=1e-8,
                           maxit=200)
    assert (it0, it1) == (9, 8)
