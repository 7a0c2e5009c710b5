"""Univariate B-splines on open knot vectors (Sec. 3.1 of the paper).

Test infrastructure: part of the CPU oracle, see `oracle/__init__.py`.

The basis b_{i,p}, i = 1..m, is defined by the Cox-de Boor recursion on an
open knot vector xi_1 = ... = xi_{p+1} = 0 < interior knots <
xi_{m} = ... = xi_{m+p+1} = 1; with uniform elements and maximal regularity
m = n_el + p. Derivatives follow from differentiating the recursion. Code is
0-based: basis index i runs 0..m-1.
"""
import numpy as np


def open_uniform_knots(p, n_el):
    """Open knot vector on [0,1] with n_el uniform elements and single interior knots (max regularity)."""
    interior = [k / n_el for k in range(1, n_el)]
    return np.array([0.0] * (p + 1) + interior + [1.0] * (p + 1))


def _ratio(a, b):
    # Cox-de Boor convention: a term whose knot span has zero length is dropped (0/0 := 0).
    return a / b if b != 0.0 else 0.0


def basis_all(knots, p, x, nder=2):
    """Values and derivatives (orders 0..nder) of all m = len(knots)-p-1 B-splines at points x.

    Returns an array D of shape (nder+1, len(x), m) with D[s, q, i] = d^s b_{i,p}(x_q).
    Degree 0: indicator of [xi_i, xi_{i+1}) (the last non-empty span also takes x = 1).
    Degree k: b_{i,k} = (x-xi_i)/(xi_{i+k}-xi_i) b_{i,k-1} + (xi_{i+k+1}-x)/(xi_{i+k+1}-xi_{i+1}) b_{i+1,k-1}.
    Derivative: d^s b_{i,k} = k [ d^{s-1} b_{i,k-1}/(xi_{i+k}-xi_i) - d^{s-1} b_{i+1,k-1}/(xi_{i+k+1}-xi_{i+1}) ].
    """
    x = np.atleast_1d(np.asarray(x, dtype=float))
    t = np.asarray(knots, dtype=float)
    nk = len(t)
    m = nk - p - 1
    last_span = max(j for j in range(nk - 1) if t[j + 1] > t[j])
    # N[k][s] : array (len(x), nk-1-k) of s-th derivatives of degree-k B-splines
    N = [[None] * (nder + 1) for _ in range(p + 1)]
    B0 = np.zeros((len(x), nk - 1))
    for j in range(nk - 1):
        if t[j + 1] > t[j]:
            inside = (x >= t[j]) & (x < t[j + 1])
            if j == last_span:
                inside = inside | (x == t[j + 1])
            B0[:, j] = inside.astype(float)
    N[0][0] = B0
    for s in range(1, nder + 1):
        N[0][s] = np.zeros_like(B0)
    for k in range(1, p + 1):
        cnt = nk - 1 - k
        for s in range(0, nder + 1):
            out = np.zeros((len(x), cnt))
            for i in range(cnt):
                if s == 0:
                    a = _ratio(1.0, t[i + k] - t[i])
                    b = _ratio(1.0, t[i + k + 1] - t[i + 1])
                    out[:, i] = a * (x - t[i]) * N[k - 1][0][:, i] + b * (t[i + k + 1] - x) * N[k - 1][0][:, i + 1]
                else:
                    a = _ratio(k, t[i + k] - t[i])
                    b = _ratio(k, t[i + k + 1] - t[i + 1])
                    out[:, i] = a * N[k - 1][s - 1][:, i] - b * N[k - 1][s - 1][:, i + 1]
            N[k][s] = out
    D = np.stack([N[p][s][:, :m] for s in range(nder + 1)])
    return D


def gauss_legendre(nq):
    """Gauss-Legendre nodes and weights on [-1, 1] (library routine)."""
    return np.polynomial.legendre.leggauss(nq)


def element_quadrature(n_el, nq, length=1.0):
    """Tensor of quadrature points/weights: nq Gauss points in each of n_el uniform elements of [0, length].

    Points are ordered element by element, left to right (the same order the
    library's quadrature-point query uses).
    """
    g, w = gauss_legendre(nq)
    h = length / n_el
    pts = np.concatenate([(e + 0.5 * (g + 1.0)) * h for e in range(n_el)])
    wts = np.concatenate([0.5 * h * w for _ in range(n_el)])
    return pts, wts


def default_nq(p):
    """Quadrature points per element used for every integral of the method: p + 2.

    The paper does not state its quadrature. With p + 2 points the unweighted
    Galerkin matrices are exact and polynomial weights up to degree 3 are too.
    """
    return p + 2
