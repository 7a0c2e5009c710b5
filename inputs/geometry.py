"""Analytic geometry maps F: (0,1)^d -> Omega (the single-patch parametrisation of Sec. 3.2, Assumption 1).

Inputs only: each map returns its first and second derivatives at given parametric points; what the
method does with them (Jacobian determinants, metric, the physical Laplacian) is the oracle's and the
library's business. Points are arrays of shape (npts, d); J[q, m, a] = dF_m / d eta_a and
H[q, m, a, b] = d^2 F_m / (d eta_a d eta_b).

  Identity(d)            F = id (the parametric domain, where the paper's fast solver lives)
  Affine(scales)         F(eta) = diag(scales) eta (a box with other side lengths)
  QuarterAnnulus(r0, r1) d = 2, F(eta) = r (cos theta, sin theta), r = r0 + (r1 - r0) eta_1,
                         theta = (pi / 2) eta_2 (a curved, non-affine domain)
  Perturbed(eps, d)      F(eta) = eta + eps prod_l sin(pi eta_l) (1, ..., 1): the unit box with its
                         interior distorted (the boundary stays where it is); injective for small eps
"""
import math

import numpy as np


class Identity:
    def __init__(self, d):
        self.d = d

    def F(self, pts):
        return np.array(pts, dtype=float)

    def jac_hess(self, pts):
        n = len(pts)
        J = np.broadcast_to(np.eye(self.d), (n, self.d, self.d)).copy()
        return J, np.zeros((n, self.d, self.d, self.d))


class Affine:
    def __init__(self, scales):
        self.s = np.asarray(scales, dtype=float)
        self.d = len(self.s)

    def F(self, pts):
        return np.asarray(pts, dtype=float) * self.s

    def jac_hess(self, pts):
        n = len(pts)
        J = np.broadcast_to(np.diag(self.s), (n, self.d, self.d)).copy()
        return J, np.zeros((n, self.d, self.d, self.d))


class QuarterAnnulus:
    d = 2

    def __init__(self, r0=1.0, r1=2.0):
        self.r0, self.r1 = float(r0), float(r1)

    def polar(self, pts):
        pts = np.asarray(pts, dtype=float)
        return self.r0 + (self.r1 - self.r0) * pts[:, 0], 0.5 * math.pi * pts[:, 1]

    def F(self, pts):
        r, th = self.polar(pts)
        return np.stack([r * np.cos(th), r * np.sin(th)], axis=1)

    def jac_hess(self, pts):
        r, th = self.polar(pts)
        dr, dth = self.r1 - self.r0, 0.5 * math.pi
        c, s = np.cos(th), np.sin(th)
        n = len(r)
        J = np.zeros((n, 2, 2))
        J[:, 0, 0], J[:, 0, 1] = dr * c, -r * s * dth
        J[:, 1, 0], J[:, 1, 1] = dr * s, r * c * dth
        H = np.zeros((n, 2, 2, 2))
        # x = r cos th: x_11 = 0, x_12 = -dr s dth, x_22 = -r c dth^2; y = r sin th likewise
        H[:, 0, 0, 1] = H[:, 0, 1, 0] = -dr * s * dth
        H[:, 0, 1, 1] = -r * c * dth * dth
        H[:, 1, 0, 1] = H[:, 1, 1, 0] = dr * c * dth
        H[:, 1, 1, 1] = -r * s * dth * dth
        return J, H


class Perturbed:
    def __init__(self, eps, d):
        self.eps, self.d = float(eps), d

    def F(self, pts):
        pts = np.asarray(pts, dtype=float)
        phi = np.prod(np.sin(math.pi * pts), axis=1)
        return pts + self.eps * phi[:, None]

    def jac_hess(self, pts):
        pts = np.asarray(pts, dtype=float)
        n, d = pts.shape
        sn, cs = np.sin(math.pi * pts), np.cos(math.pi * pts)
        # phi = prod_l sin(pi eta_l); d phi / d eta_a and d^2 phi / (d eta_a d eta_b)
        g = np.zeros((n, d))
        h = np.zeros((n, d, d))
        for a in range(d):
            fa = math.pi * cs[:, a]
            others = np.prod(np.delete(sn, a, axis=1), axis=1) if d > 1 else np.ones(n)
            g[:, a] = fa * others
            h[:, a, a] = -math.pi ** 2 * sn[:, a] * others
            for b in range(d):
                if b != a:
                    rest = np.prod(np.delete(sn, [a, b], axis=1), axis=1) if d > 2 else np.ones(n)
                    h[:, a, b] = fa * math.pi * cs[:, b] * rest
        J = np.broadcast_to(np.eye(d), (n, d, d)).copy() + self.eps * g[:, None, :]
        H = np.broadcast_to(self.eps * h[:, None, :, :], (n, d, d, d)).copy()
        return J, H


def tensor_points(grids):
    """The tensor grid of 1D point sets grids[0] (direction 1, fastest) .. grids[d-1], shape (npts, d)."""
    mesh = np.meshgrid(*grids[::-1], indexing="ij")
    return np.stack([m.ravel() for m in mesh[::-1]], axis=1)


def geometry_at(gmap, grids):
    """(J, H) of the map on the tensor grid of the directions' quadrature points, direction 1 fastest,
    flattened to J[q, m, a], H[q, m, a, b]."""
    return gmap.jac_hess(tensor_points(grids))
