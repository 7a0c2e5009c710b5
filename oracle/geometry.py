"""The least-squares system on a mapped domain Omega = F((0,1)^d) (Sec. 3.2, Eq. syst_mat, Eq. space_mat).

Test infrastructure: part of the CPU oracle, see `oracle/__init__.py`.

With the push-forward basis B_i = B-hat_i o F^{-1} (Eq. disc_space) the system keeps the form
    A = M_s (x) L_t + nu^2 B_s (x) M_t + nu L_s (x) (W_t + W_t^*)                  (Eq. syst_mat)
with the time matrices of the parametric case, but the spatial matrices of Eq. space_mat are integrals
over the physical domain, which no longer split into one-direction factors:
    M_s[i,j] = int_Omega B_i B_j,   L_s[i,j] = int_Omega grad B_i . grad B_j,
    B_s[i,j] = int_Omega Delta B_i Delta B_j.
Pulled back to the parametric box (x = F(eta), J = dF/d eta, G = J^{-1} J^{-T}):
    dx = |det J| d eta,   grad_x u . grad_x v = grad u-hat^T G grad v-hat,
    Delta_x u = sum_ab G^{ab} d_a d_b u-hat + sum_a h^a d_a u-hat,
    h^a = - sum_m (J^{-1})_{am} sum_bc (d_b d_c F_m) G^{bc}
(the chain rule twice; the first-order term carries the curvature of the map). Every integral is the
spline quadrature of the parametric case (p + 2 Gauss points per element and direction) on the tensor grid
of the directions' points. The potential is not included (the paper's geometry statement has V = 0), and the
right-hand sides in the tests are given vectors.

The paper's fast solver (Sec. 5) is for F = id only; on a mapped domain P-hat stays the parametric one and
serves as a preconditioner (`oracle.fd.FastDiagonalization` of the parametric Discretization).
"""
import numpy as np
import scipy.sparse as sp

from .bspline import open_uniform_knots, basis_all
from .system import Discretization


def metric_terms(J, H):
    """Per point: |det J|, G = J^{-1} J^{-T}, and the first-order coefficients h of the physical Laplacian."""
    det = np.linalg.det(J)
    Jinv = np.linalg.inv(J)
    G = Jinv @ np.transpose(Jinv, (0, 2, 1))
    # h^a = - sum_m Jinv[a, m] sum_{b,c} H[m, b, c] G[b, c]
    tr = np.einsum("qmbc,qbc->qm", H, G)
    h = -np.einsum("qam,qm->qa", Jinv, tr)
    return np.abs(det), G, h


def prec_scales(gmap, disc_or_grids):
    """Per-direction scales s_l of the parametric preconditioner's eigenvalues on a mapped domain:
    s_l = int |det J| G^{ll} / int |det J| over the parametric box (the mean of the metric's diagonal). For
    an affine map with sides a_l this is 1 / a_l^2, which makes the scaled P-hat the box's own (up to a
    constant factor); for a curved map it matches the mean scale of the physical Laplacian in each
    direction. disc_or_grids: a Discretization (its quadrature) or the list of 1D (points, weights)."""
    if hasattr(disc_or_grids, "quad"):
        qw = [disc_or_grids.quad(l) for l in range(1, disc_or_grids.d + 1)]
    else:
        qw = disc_or_grids
    grids = [x for x, _ in qw]
    mesh = np.meshgrid(*grids[::-1], indexing="ij")
    pts = np.stack([m.ravel() for m in mesh[::-1]], axis=1)
    wq = qw[0][1]
    for l in range(1, len(qw)):
        wq = np.kron(qw[l][1], wq)
    J, H = gmap.jac_hess(pts)
    adet, G, _ = metric_terms(J, H)
    w = wq * adet
    return [float(np.sum(w * G[:, l, l]) / np.sum(w)) for l in range(len(qw))]


class GeoDiscretization:
    """Space-time spline discretisation of (0, T) x F((0,1)^d), potential-free.

    n_el, p, T, nu: as `oracle.system.Discretization`; gmap: an object with jac_hess(points) returning
    (J[q, m, a], H[q, m, a, b]) at parametric points (npts, d), such as the maps of `inputs.geometry`.
    """

    def __init__(self, n_el, p, gmap, T=1.0, nu=1.0):
        if isinstance(p, int):
            p = [p] * len(n_el)
        self.base = Discretization(n_el, p, T=T, nu=nu)
        b = self.base
        self.d, self.nu = b.d, b.nu
        self.n, self.N_s, self.N_dof, self.shape = b.n, b.N_s, b.N_dof, b.shape
        d = self.d
        # restricted 1D tables (value, first, second derivative) at each direction's quadrature points
        tabs, grids, wts = [], [], []
        for l in range(1, d + 1):
            x, w = b.quad(l)
            D = basis_all(open_uniform_knots(b.p[l], b.n_el[l]), b.p[l], x, nder=2)[:, :, 1:-1]
            tabs.append([sp.csr_matrix(D[s]) for s in range(3)])
            grids.append(x)
            wts.append(w)
        # tensor grid, direction 1 fastest (the same order as the library's spatial quadrature grid)
        mesh = np.meshgrid(*grids[::-1], indexing="ij")
        pts = np.stack([m.ravel() for m in mesh[::-1]], axis=1)
        wq = wts[0]
        for l in range(1, d):
            wq = np.kron(wts[l], wq)
        J, H = gmap.jac_hess(pts)
        adet, G, h = metric_terms(J, H)

        def table(orders):
            """Tensor-product table of the derivative orders[l] in direction l (sparse, npts x N_s)."""
            T_ = tabs[0][orders[0]]
            for l in range(1, d):
                T_ = sp.kron(tabs[l][orders[l]], T_, format="csr")
            return T_

        def order(*axes):
            o = [0] * d
            for a in axes:
                o[a] += 1
            return o

        Phi = table([0] * d)
        dPhi = [table(order(a)) for a in range(d)]
        ddPhi = [[table(order(a, c)) for c in range(d)] for a in range(d)]
        wdet = wq * adet
        W = sp.diags(wdet)
        self.Ms = (Phi.T @ W @ Phi).tocsr()
        Ls = None
        for a in range(d):
            for c in range(d):
                t = dPhi[a].T @ sp.diags(wdet * G[:, a, c]) @ dPhi[c]
                Ls = t if Ls is None else Ls + t
        self.Ls = Ls.tocsr()
        lap = None
        for a in range(d):
            t = sp.diags(h[:, a]) @ dPhi[a]
            for c in range(d):
                t = t + sp.diags(G[:, a, c]) @ ddPhi[a][c]
            lap = t if lap is None else lap + t
        self.Bs = (lap.T @ W @ lap).tocsr()
        self.Lt, self.Mt, self.Wsym = b.Lt, b.Mt, b.Wsym

    def terms(self):
        """(spatial matrix, time matrix, coefficient) of Eq. syst_mat."""
        return [(self.Ms, self.Lt, 1.0), (self.Bs, self.Mt, self.nu ** 2), (self.Ls, self.Wsym, self.nu)]

    def apply(self, x):
        """A x with x in the vec order (time fastest): Y = sum_k c_k S_k X T_k^T, X of shape (N_s, n_t)."""
        X = np.asarray(x, dtype=complex).reshape(self.N_s, self.n[0])
        Y = sum(c * (S @ X) @ T.T for S, T, c in self.terms())
        return Y.ravel()

    def dense(self):
        A = np.zeros((self.N_dof, self.N_dof), dtype=complex)
        for S, T, c in self.terms():
            A += c * np.kron(S.toarray(), T)
        return A

    def sparse(self):
        return sum(c * sp.kron(S, sp.csr_matrix(T), format="csr") for S, T, c in self.terms()).tocsc()
