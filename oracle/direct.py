"""Brute-force assembly of the least-squares matrix and load vector by (d+1)-dimensional quadrature.

Test infrastructure: part of the CPU oracle, see `oracle/__init__.py`.

[A]_{ij} = A(B_j, S B_i) = int_Q (S B_j) conj(S B_i)       (Sec. 4.3, discrete system)
[f]_i    = F(S B_i)      = int_Q f conj(S B_i)
with S = i d_t - nu Delta (+ V(x) when a potential is given). Every basis
function and its derivatives are evaluated at every point of the tensor
Gauss grid; nothing of the Kronecker structure is used, so this pins the
Kronecker form of `system.Discretization` (Eq. syst_mat) independently.
Tiny meshes only: cost O(N_q N_dof^2).
"""
import itertools

import numpy as np

from .bspline import open_uniform_knots, basis_all


def _restricted_basis(disc, l):
    x, w = disc.quad(l)
    length = disc.T if l == 0 else 1.0
    D = basis_all(open_uniform_knots(disc.p[l], disc.n_el[l]), disc.p[l], x / length, nder=2)
    D = D / np.array([1.0, length, length ** 2])[:, None, None]
    if l == 0:
        D = D[:, :, :-1] if disc.formulation == "uw" else D[:, :, 1:]
    else:
        D = D[:, :, 1:-1]
    return x, w, D


def sb_matrix(disc, V=None):
    """G[q, j] = (S B_j)(point q) on the tensor Gauss grid, and the grid weights and points."""
    d, nu = disc.d, disc.nu
    data = [_restricted_basis(disc, l) for l in range(d + 1)]
    grids = [np.arange(len(data[l][0])) for l in range(d + 1)]
    pts, wts, rows = [], [], []
    idx_ranges = [range(disc.n[l]) for l in range(d + 1)]
    for qs in itertools.product(*grids):
        xq = [data[l][0][qs[l]] for l in range(d + 1)]
        wq = np.prod([data[l][1][qs[l]] for l in range(d + 1)])
        vq = V(np.array(xq[1:])) if V is not None else 0.0
        row = np.zeros(disc.N_dof, dtype=complex)
        # enumerate basis multi-indices in vec order: time fastest, then x_1, ..., x_d
        for j, ii in enumerate(itertools.product(*reversed(idx_ranges))):
            ii = ii[::-1]  # ii[0] = time index, ii[l] = space index of direction l
            bt, dbt = data[0][2][0][qs[0], ii[0]], data[0][2][1][qs[0], ii[0]]
            vals = [data[l][2][0][qs[l], ii[l]] for l in range(1, d + 1)]
            sec = [data[l][2][2][qs[l], ii[l]] for l in range(1, d + 1)]
            Bs = np.prod(vals)
            lap = sum(sec[l] * np.prod([vals[k] for k in range(d) if k != l]) for l in range(d))
            row[j] = 1j * dbt * Bs - nu * bt * lap + vq * bt * Bs
        pts.append(xq)
        wts.append(wq)
        rows.append(row)
    return np.array(rows), np.array(wts), np.array(pts)


def dense_A(disc, V=None):
    """[A]_{ij} = int (S B_j) conj(S B_i) by tensor quadrature."""
    G, w, _ = sb_matrix(disc, V)
    return (G.conj().T * w) @ G


def load_vector(disc, f, V=None):
    """[f]_i = int f conj(S B_i) by tensor quadrature; f(t, x) takes a point (t, x_1, ..., x_d)."""
    G, w, pts = sb_matrix(disc, V)
    fv = np.array([f(p) for p in pts])
    return (G.conj().T * w) @ fv
