"""Pins of the oracle's system on a mapped domain (`oracle.geometry`, Sec. 3.2 and Eq. syst_mat, Eq. space_mat).

  * F = id gives the parametric system of `oracle.system` (Kronecker factors), d = 1, 2, 3.
  * An affine map (a box with sides a, b) gives the closed forms of M_s, L_s, B_s built from the
    one-direction matrices with the scale factors written out by hand.
  * On the quarter annulus the three spatial forms of a function u-hat = eta_1 (1 - eta_1) eta_2 (1 - eta_2)
    (which lies in the spline space with its boundary conditions for p >= 2) equal the integrals
    int u^2, int |grad u|^2 and int (Delta u)^2 over the annulus computed by adaptive quadrature in polar
    coordinates with the textbook polar gradient and Laplacian (u_r, u_theta / r; u_rr + u_r / r +
    u_thetatheta / r^2): independent of the chain-rule form the oracle uses. A dropped first-order term of
    the physical Laplacian, a missing |det J| or a transposed metric fails them.
  * The mapped system is Hermitian positive definite, and PCG preconditioned by the parametric P-hat
    (the paper's solver, Sec. 5: F = id only) reaches the sparse direct solution.
"""
import math

import numpy as np
import pytest
import scipy.integrate as si
import scipy.sparse.linalg as spla

from inputs.geometry import Affine, Identity, Perturbed, QuarterAnnulus
from oracle import fd, geometry, pcg
from oracle.matrices import space_matrices
from oracle.system import Discretization


@pytest.mark.parametrize("n_el,p", [([4, 5], [2, 3]), ([3, 4, 5], [2, 2, 3]), ([2, 3, 3, 4], [1, 2, 2, 2])])
def test_identity_map_gives_the_parametric_system(n_el, p):
    d = len(n_el) - 1
    A = geometry.GeoDiscretization(n_el, p, Identity(d)).dense()
    A0 = Discretization(n_el, p).dense()
    assert np.abs(A - A0).max() <= 1e-12 * np.abs(A0).max()


def test_affine_map_closed_forms():
    n_el, p, a, b = [3, 5, 4], 3, 0.7, 1.9
    g = geometry.GeoDiscretization(n_el, p, Affine([a, b]))
    s1, s2 = space_matrices(p, n_el[1]), space_matrices(p, n_el[2])
    kr = np.kron
    Ms = a * b * kr(s2["M"], s1["M"])
    Ls = a * b * (kr(s2["M"], s1["L"]) / a ** 2 + kr(s2["L"], s1["M"]) / b ** 2)
    # Delta u = u_11 / a^2 + u_22 / b^2; K2[i, j] = int b_i b''_j
    Bs = a * b * (kr(s2["M"], s1["J"]) / a ** 4 + kr(s2["J"], s1["M"]) / b ** 4 +
                  (kr(s2["K2"], s1["K2"].T) + kr(s2["K2"].T, s1["K2"])) / (a * b) ** 2)
    for got, want in [(g.Ms, Ms), (g.Ls, Ls), (g.Bs, Bs)]:
        assert np.abs(got.toarray() - want).max() <= 1e-12 * np.abs(want).max()


def _coeffs_of_bubble(p, n_el):
    """Spline coefficients (restricted basis) of eta (1 - eta): its L2 projection, exact in the space."""
    s = space_matrices(p, n_el)
    from oracle.bspline import open_uniform_knots, basis_all, element_quadrature
    x, w = element_quadrature(n_el, p + 2)
    B = basis_all(open_uniform_knots(p, n_el), p, x, nder=0)[0][:, 1:-1]
    rhs = B.T @ (w * x * (1 - x))
    return np.linalg.solve(s["M"], rhs)


def _polar_integrals(r0, r1):
    """int u^2, int |grad u|^2, int (Delta u)^2 over the quarter annulus for u = P(eta_1) Q(eta_2),
    eta_1 = (r - r0) / (r1 - r0), eta_2 = 2 theta / pi, P = Q = eta (1 - eta), in polar coordinates."""
    dr, dth = r1 - r0, 0.5 * math.pi

    def parts(r, th):
        e1, e2 = (r - r0) / dr, th / dth
        P, P1, P2 = e1 * (1 - e1), (1 - 2 * e1) / dr, -2.0 / dr ** 2
        Q, Q1, Q2 = e2 * (1 - e2), (1 - 2 * e2) / dth, -2.0 / dth ** 2
        u, ur, ut = P * Q, P1 * Q, P * Q1
        urr, utt = P2 * Q, P * Q2
        return u, ur, ut, urr, utt

    def integrand(k):
        def f(th, r):
            u, ur, ut, urr, utt = parts(r, th)
            if k == 0:
                v = u * u
            elif k == 1:
                v = ur * ur + (ut / r) ** 2
            else:
                v = (urr + ur / r + utt / r ** 2) ** 2
            return v * r
        return f

    return [si.dblquad(integrand(k), r0, r1, 0.0, dth, epsabs=0, epsrel=1e-13)[0] for k in range(3)]


def test_quarter_annulus_forms_match_polar_integrals():
    r0, r1, p, ne = 1.0, 2.0, 3, 8
    g = geometry.GeoDiscretization([2, ne, ne], p, QuarterAnnulus(r0, r1))
    c1 = _coeffs_of_bubble(p, ne)
    c = np.kron(c1, c1)
    got = [c @ (S @ c) for S in (g.Ms, g.Ls, g.Bs)]
    want = _polar_integrals(r0, r1)
    for gv, wv in zip(got, want):
        assert abs(gv - wv) <= 1e-7 * abs(wv), (gv, wv)


@pytest.mark.parametrize("mutation", ["no_first_order", "no_det", "metric_transposed_inverse"])
def test_planted_mistakes_fail_the_polar_pin(monkeypatch, mutation):
    orig = geometry.metric_terms

    def bad(J, H):
        adet, G, h = orig(J, H)
        if mutation == "no_first_order":
            return adet, G, 0.0 * h
        if mutation == "no_det":
            return np.ones_like(adet), G, h
        Ji = np.linalg.inv(J)
        return adet, np.transpose(Ji, (0, 2, 1)) @ Ji, h  # J^{-T} J^{-1} instead of J^{-1} J^{-T}

    monkeypatch.setattr(geometry, "metric_terms", bad)
    r0, r1, p, ne = 1.0, 2.0, 3, 8
    g = geometry.GeoDiscretization([2, ne, ne], p, QuarterAnnulus(r0, r1))
    c1 = _coeffs_of_bubble(p, ne)
    c = np.kron(c1, c1)
    got = [c @ (S @ c) for S in (g.Ms, g.Ls, g.Bs)]
    want = _polar_integrals(r0, r1)
    assert max(abs(gv - wv) / abs(wv) for gv, wv in zip(got, want)) > 1e-3


@pytest.mark.parametrize("gmap,n_el,p", [(QuarterAnnulus(1.0, 2.0), [4, 5, 4], [2, 3, 2]),
                                         (Perturbed(0.08, 2), [3, 4, 5], 2),
                                         (Perturbed(0.05, 3), [2, 3, 3, 3], 2),
                                         (Perturbed(0.1, 1), [5, 7], 3)])
def test_mapped_system_is_hermitian_positive_definite(gmap, n_el, p):
    A = geometry.GeoDiscretization(n_el, p, gmap).dense()
    assert np.abs(A - A.conj().T).max() <= 1e-12 * np.abs(A).max()
    np.linalg.cholesky(A)


@pytest.mark.parametrize("gmap,n_el,p", [(QuarterAnnulus(1.0, 2.0), [6, 7, 6], [2, 3, 2]),
                                         (Perturbed(0.05, 3), [3, 4, 3, 4], [2, 2, 2, 2])])
def test_parametric_phat_preconditions_the_mapped_system(gmap, n_el, p):
    g = geometry.GeoDiscretization(n_el, p, gmap)
    F = fd.FastDiagonalization(Discretization(n_el, p))
    rng = np.random.default_rng(3)
    f = rng.standard_normal(g.N_dof) + 1j * rng.standard_normal(g.N_dof)
    x, it, rr, _ = pcg.pcg(g.apply, F.apply, f, tol=1e-12, maxit=500)
    xd = spla.spsolve(g.sparse(), f)
    assert rr <= 1e-12
    assert np.abs(x - xd).max() <= 1e-9 * np.abs(xd).max()
    assert it < 120


def test_prec_scales_of_an_affine_map_are_the_inverse_squared_sides():
    a, b = 0.7, 1.9
    disc = Discretization([3, 5, 4], [2, 3, 3])
    s = geometry.prec_scales(Affine([a, b]), disc)
    assert abs(s[0] - 1 / a ** 2) <= 1e-14 / a ** 2 and abs(s[1] - 1 / b ** 2) <= 1e-14 / b ** 2


def test_scaled_phat_is_the_box_preconditioner():
    """P-hat with eigenvalue scales 1 / a_l^2 is (prod a_l) times the inverse of P-hat assembled straight
    from Eq. prec_definition with the box's own one-direction matrices (mass a_l M_l, stiffness L_l / a_l)."""
    n_el, p, sides = [4, 5, 6], [2, 3, 2], [0.6, 1.7]
    disc = Discretization(n_el, p)
    F = fd.FastDiagonalization(disc, scales=[1 / a ** 2 for a in sides])
    Ms, Ls = np.ones((1, 1)), np.zeros((1, 1))
    for l, a in zip((1, 2), sides):
        M, L = a * disc.sp[l]["M"], disc.sp[l]["L"] / a
        Ls = np.kron(M, Ls) + np.kron(L, Ms)
        Ms = np.kron(M, Ms)
    P = np.kron(Ms, disc.Lt) + np.kron(Ls.T @ np.linalg.solve(Ms, Ls), disc.Mt) + np.kron(Ls, disc.Wsym)
    r = np.random.default_rng(4).standard_normal(disc.N_dof) + 0j
    want = np.prod(sides) * np.linalg.solve(P, r)
    assert np.abs(F.apply(r) - want).max() <= 1e-10 * np.abs(want).max()


def test_scaled_phat_restores_the_parametric_iteration_count_on_a_box():
    n_el, p, sides = [8, 12, 12], [3, 3, 3], [1.0, 0.5 * math.pi]
    disc = Discretization(n_el, p)
    g = geometry.GeoDiscretization(n_el, p, Affine(sides))
    f = np.random.default_rng(5).standard_normal(disc.N_dof) + 0j
    _, it_unit, _, _ = pcg.pcg(disc.apply, fd.FastDiagonalization(disc).apply, f, tol=1e-8, maxit=2000)
    sc = geometry.prec_scales(Affine(sides), disc)
    _, it_scaled, _, _ = pcg.pcg(g.apply, fd.FastDiagonalization(disc, scales=sc).apply, f, tol=1e-8, maxit=2000)
    _, it_plain, _, _ = pcg.pcg(g.apply, fd.FastDiagonalization(disc).apply, f, tol=1e-8, maxit=2000)
    assert abs(it_scaled - it_unit) <= 2, (it_scaled, it_unit)
    assert it_plain > 2 * it_scaled
