"""Errors in the L2(Q) norm and in the graph norm of V (Sec. 2.1, Theorem 2, Remark 1).

Test infrastructure: part of the CPU oracle, see `oracle/__init__.py`.

||v||_V^2 = ||v||_{L2(Q)}^2 + ||S v||_{L2(Q)}^2 with S = i d_t - nu Delta (+ V).
For the exact solution S u = f, so S(u - u_h) = f - S u_h. Integrals use a
tensor Gauss rule with nq_extra more points per element than the assembly.
"""
import numpy as np

from .bspline import element_quadrature
from .rhs import tables, grid_coords, potential_fn
from .system import mode_product


def errors(disc, U_full, u_fn, f_fn, nq_extra=3):
    """Returns (||u - u_h||_L2, ||u - u_h||_V) for the full coefficient tensor U_full of u_h."""
    d, nu = disc.d, disc.nu
    pts, wts = [], []
    for l in range(d + 1):
        x, w = element_quadrature(disc.n_el[l], disc.nq[l] + nq_extra, disc.T if l == 0 else 1.0)
        pts.append(x)
        wts.append(w)
    T = [tables(disc, l, pts=pts[l], full=True) for l in range(d + 1)]

    def evaluate(tders, sders):
        Z = mode_product(U_full, T[0][tders], d)
        for l in range(1, d + 1):
            Z = mode_product(Z, T[l][sders[l - 1]], d - l)
        return Z

    uh = evaluate(0, [0] * d)
    duh = evaluate(1, [0] * d)
    lap = sum(evaluate(0, [2 if k == l else 0 for k in range(d)]) for l in range(d))
    Suh = 1j * duh - nu * lap
    co = grid_coords(disc, pts=pts)
    V = potential_fn(disc)
    if V is not None:
        Suh = Suh + V(*co[1:]) * uh
    W = np.ones([1] * (d + 1))
    for l in range(d + 1):
        shp = [1] * (d + 1)
        shp[d if l == 0 else d - l] = len(wts[l])
        W = W * wts[l].reshape(shp)
    e = u_fn(*co) - uh
    se = f_fn(*co) - Suh
    l2 = np.sqrt(np.sum(W * np.abs(e) ** 2))
    sn = np.sqrt(np.sum(W * np.abs(se) ** 2))
    return l2, np.sqrt(l2 ** 2 + sn ** 2)
