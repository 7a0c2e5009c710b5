"""Pins of the oracle's lifting of general Dirichlet and initial data (Sec. 2.2: u = u_bar + u_lift,
f_bar = f - S u_lift), independent of the oracle's own B-spline and matrix code:

* the right-hand side rhs_i = (f - S_V g_h, S_V B_i) by brute force: the basis and its derivatives
  from scipy.interpolate.BSpline, the tensor Gauss rule from numpy's Gauss-Legendre nodes (the rule
  the method integrates f with, p + 2 points per element), S_V applied to g_h and to every interior
  test function pointwise;
* the projection that defines g_h: for u in the spline space the kept coefficients are u's own
  (obtained by interpolation at the Greville abscissae with the scipy basis).
"""
import numpy as np
import pytest

from scipy.interpolate import BSpline

from oracle import rhs as orhs
from tests._common import oracle_disc, rel_err


def _knots(p, n_el, length):
    return np.concatenate([np.zeros(p), np.linspace(0.0, 1.0, n_el + 1), np.ones(p)]) * length


def _basis(p, n_el, length, x, der):
    """(len(x), n_el + p): derivative `der` of every basis function of the open uniform knot vector."""
    t = _knots(p, n_el, length)
    m = n_el + p
    out = np.zeros((len(x), m))
    for j in range(m):
        c = np.zeros(m)
        c[j] = 1.0
        b = BSpline(t, c, p, extrapolate=False)
        out[:, j] = (b.derivative(der) if der else b)(x)
    return out


def _gauss(n_el, nq, length):
    g, w = np.polynomial.legendre.leggauss(nq)
    h = length / n_el
    x = np.concatenate([(e + 0.5 * (g + 1.0)) * h for e in range(n_el)])
    return x, np.tile(0.5 * h * w, n_el)


def _brute_rhs(n_el, p, T, nu, u_fn, f_fn, V, XD):
    """rhs of the lifted problem by pointwise S_V on the tensor grid (time axis last, x_1 before it)."""
    d = len(n_el) - 1
    L = [T] + [1.0] * d
    pts, wts, B = [], [], []
    for l in range(d + 1):
        x, w = _gauss(n_el[l], p[l] + 2, L[l])
        pts.append(x)
        wts.append(w)
        B.append([_basis(p[l], n_el[l], L[l], x, k) for k in range(3)])
    # axes of the coefficient / grid tensors: (x_d, ..., x_1, t)
    def ev(C, ders):
        """sum_j C[j] prod_l d^{ders[l]} b_{j_l}(x_l) on the grid."""
        G = C
        for l in range(d + 1):
            ax = d if l == 0 else d - l
            G = np.moveaxis(np.tensordot(B[l][ders[l]], G, axes=([1], [ax])), 0, ax)
        return G
    co = np.meshgrid(*[pts[l] for l in range(d, 0, -1)], pts[0], indexing="ij")
    grid = [co[d]] + [co[d - l] for l in range(1, d + 1)]  # t, x_1, ..., x_d
    Vq = np.zeros_like(grid[0]) if V is None else sum(np.prod([term[l - 1](grid[l]) for l in range(1, d + 1)], axis=0)
                                                      for term in V)
    zero = [0] * (d + 1)
    def S_of(C):
        out = 1j * ev(C, [1] + [0] * d) + Vq * ev(C, zero)
        for l in range(1, d + 1):
            ders = list(zero)
            ders[l] = 2
            out = out - nu * ev(C, ders)
        return out
    R = f_fn(*grid) - S_of(XD)
    W = np.ones_like(R)
    for l in range(d + 1):
        shp = [1] * (d + 1)
        shp[d if l == 0 else d - l] = len(wts[l])
        W = W * wts[l].reshape(shp)
    m = [n_el[l] + p[l] for l in range(d + 1)]
    ranges = [range(1, m[0])] + [range(1, m[l] - 1) for l in range(1, d + 1)]
    out = np.zeros(tuple(len(ranges[l]) for l in range(d, 0, -1)) + (len(ranges[0]),), dtype=complex)
    for idx in np.ndindex(out.shape):
        C = np.zeros(tuple(m[l] for l in range(d, 0, -1)) + (m[0],))
        full = tuple(ranges[d - a][idx[a]] if a < d else ranges[0][idx[d]] for a in range(d + 1))
        C[full] = 1.0
        out[idx] = np.sum(W * R * np.conj(S_of(C)))
    return out.ravel()


def _u1(t, x):
    return np.exp(1j * (2.0 * t + x)) * (1.0 + x ** 2) + 0.3 * t


def _f1(t, x):
    return np.cos(3.0 * x) * (1.0 + 1j * t)


def _u2(t, x1, x2):
    return np.exp(1j * (t + 2.0 * x1 - x2)) * (1.0 + x1 * x2) + 0.2j * t * x2


def _f2(t, x1, x2):
    return (x1 - 0.3) * np.exp(-1j * t) + 0.5 * x2 ** 2


def _u3(t, x1, x2, x3):
    return np.exp(1j * (t + x1 - 2.0 * x3)) * (1.0 + x2 * x3) + 0.1 * t * x1


def _f3(t, x1, x2, x3):
    return (x1 + 1j * x2) * np.exp(-1j * t) + x3 ** 2


@pytest.mark.parametrize("n_el,p,T,nu,pot", [([3, 4], [2, 3], 1.0, 1.0, False), ([2, 3], [3, 2], 0.7, 1.3, True),
                                             ([2, 2, 3], [2, 2, 3], 1.2, 0.9, False),
                                             ([2, 3, 2], [2, 3, 2], 1.0, 1.0, True),
                                             ([2, 1, 2, 1], [2, 2, 2, 2], 0.9, 1.2, True)])
def test_full_lifting_rhs_is_load_of_f_minus_S_of_lifting(n_el, p, T, nu, pot):
    d = len(n_el) - 1
    V = None
    if pot:
        V = [[(lambda x: 1.0 + x ** 2)] * d, [(lambda x: np.cos(x))] * d]
    u_fn, f_fn = {1: (_u1, _f1), 2: (_u2, _f2), 3: (_u3, _f3)}[d]
    disc = oracle_disc(n_el, p, T=T, nu=nu, potential=V)
    b, XD = orhs.full_lifting(disc, u_fn, f_fn)
    ref = _brute_rhs(n_el, p, T, nu, u_fn, f_fn, V, np.asarray(XD))
    assert rel_err(b, ref) < 1e-10


def test_full_lifting_keeps_the_coefficients_of_a_spline():
    """u in the spline space: the lifting's coefficients are u's own on the boundary and initial functions."""
    n_el, p, T = [3, 4, 3], [2, 3, 2], 1.3
    L = [T, 1.0, 1.0]
    m = [n_el[l] + p[l] for l in range(3)]
    rng = np.random.default_rng(5)
    C = rng.standard_normal((m[2], m[1], m[0])) + 1j * rng.standard_normal((m[2], m[1], m[0]))
    # interpolation at the Greville abscissae with the scipy basis gives each direction's evaluation
    def u_fn(t, x1, x2):
        shape = np.broadcast(t, x1, x2).shape
        tt, a, b = (np.broadcast_to(v, shape).ravel() for v in (t, x1, x2))
        Bt = _basis(p[0], n_el[0], L[0], tt, 0)
        B1 = _basis(p[1], n_el[1], L[1], a, 0)
        B2 = _basis(p[2], n_el[2], L[2], b, 0)
        return np.einsum("kji,qk,qj,qi->q", C, B2, B1, Bt).reshape(shape)
    f_fn = lambda t, x1, x2: 0.0 * t * x1 * x2
    disc = oracle_disc(n_el, p, T=T)
    _, XD = orhs.full_lifting(disc, u_fn, f_fn)
    XD = np.asarray(XD)
    mask = np.zeros(C.shape, dtype=bool)
    mask[..., 0] = True
    mask[0], mask[-1], mask[:, 0], mask[:, -1] = True, True, True, True
    assert rel_err(XD[mask], C[mask]) < 1e-11
    assert np.all(XD[~mask] == 0)
