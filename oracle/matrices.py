"""Univariate Galerkin matrices and their restriction (Eq. time_mat, Eq. space_mat, Sec. 3.2, Sec. 5).

Test infrastructure: part of the CPU oracle, see `oracle/__init__.py`.

For the basis b_i(x) = b-hat_i(x / length) on [0, length] (Sec. 3.2: b_{i,p_t} = b-hat_{i,p_t}(. / T)):
  M[i,j]  = int b_i  b_j            (mass)
  L[i,j]  = int b'_j b'_i           (stiffness)
  J[i,j]  = int b''_i b''_j         (second-derivative mass, the 1D factor of B_s)
  K[i,j]  = int b'_j b_i            (advection; W_t = i K in Eq. time_mat)
  K2[i,j] = int b''_j b_i           (1D factor of the cross terms of int Delta B_i Delta B_j)
Weighted variants multiply the integrand by w(x) (separable potential factors).
All matrices are dense m x m here (the oracle favours plainness over storage).
"""
import numpy as np

from .bspline import open_uniform_knots, basis_all, element_quadrature, default_nq


def assemble_1d(p, n_el, length=1.0, nq=None, weight=None):
    """Full-basis (m = n_el + p) matrices on [0, length] by Gauss quadrature.

    weight: None or an array of the weight at the element quadrature points
    (same ordering as `bspline.element_quadrature`).
    Returns dict with keys M, L, J, K, K2.
    """
    nq = default_nq(p) if nq is None else nq
    knots = open_uniform_knots(p, n_el)
    x, w = element_quadrature(n_el, nq, length)
    D = basis_all(knots, p, x / length, nder=2)
    b = D[0]
    d1 = D[1] / length
    d2 = D[2] / length ** 2
    ww = w if weight is None else w * np.asarray(weight, dtype=float)
    M = (b * ww[:, None]).T @ b
    L = (d1 * ww[:, None]).T @ d1
    J = (d2 * ww[:, None]).T @ d2
    K = (b * ww[:, None]).T @ d1          # K[i,j] = sum_q w b_i(x_q) b'_j(x_q)
    K2 = (b * ww[:, None]).T @ d2         # K2[i,j] = sum_q w b_i(x_q) b''_j(x_q)
    return dict(M=M, L=L, J=J, K=K, K2=K2)


def restrict_time(A, formulation="ls"):
    """Least squares: drop the first basis function (the only one nonzero at t = 0), n_t = m_t - 1
    (Sec. 3.2). Ultraweak: drop the last one (the space with final conditions at T, Sec. 4.4)."""
    return A[:-1, :-1] if formulation == "uw" else A[1:, 1:]


def restrict_space(A):
    """Drop the first and last basis functions (nonzero on the boundary): n_s = m - 2 (Sec. 3.2)."""
    return A[1:-1, 1:-1]


def time_matrices(p, n_el, T):
    """Restricted time matrices L_t, M_t, W_t + W_t^* of Eq. time_mat on (0, T)."""
    F = assemble_1d(p, n_el, T)
    Lt = restrict_time(F["L"])
    Mt = restrict_time(F["M"])
    Wt = 1j * restrict_time(F["K"])
    return dict(L=Lt, M=Mt, W=Wt, Wsym=Wt + Wt.conj().T, full=F)


def space_matrices(p, n_el, length=1.0):
    """Restricted spatial matrices M_l, L_l, J_l, K2_l on (0, length) (Eq. space_mat factors, Sec. 5)."""
    F = assemble_1d(p, n_el, length)
    return dict(M=restrict_space(F["M"]), L=restrict_space(F["L"]), J=restrict_space(F["J"]),
                K2=restrict_space(F["K2"]), full=F)
