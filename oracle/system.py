"""The least-squares system matrix in Kronecker form (Eq. syst_mat, Eq. space_mat, Eq. time_mat).

Test infrastructure: part of the CPU oracle, see `oracle/__init__.py`.

Unknowns are ordered as in the vec operator of Sec. 3.3 with time as the
first (fastest) index: a coefficient tensor X has numpy shape
(n_d, ..., n_1, n_t) in C order, so `X.ravel()` is vec(X).

A = M_s (x) L_t + nu^2 B_s (x) M_t + nu L_s (x) (W_t + W_t^*)          (Eq. syst_mat)
with, on the box (0,1)^d, M_s = M_d (x) ... (x) M_1,
L_s = sum_l ( ... M (x) L_l (x) M ... ) (int grad B_i . grad B_j),
B_s = int Delta B_i Delta B_j = sum_l (J_l with M elsewhere)
      + sum_{l != k} (K2_l^T at l, K2_k at k, M elsewhere),
where K2[i,j] = int b''_j b_i. (Expanding Delta = sum_l d_ll in the definition
of B_s in Eq. space_mat; no integration by parts is used here.)

Potential extension (not in the paper): S_V = i d_t - nu Delta + V(x), with a
separable real potential V = sum_r prod_l v_{r,l}(x_l). Expanding
(S_V B_j, S_V B_i) adds
   M_{V^2,s} (x) M_t  +  M_{V,s} (x) (W_t + W_t^*)
   - nu sum_r sum_l (K2_{v_rl} + K2_{v_rl}^T at l, M_{v_rk} elsewhere) (x) M_t,
where M_{w} / K2_{w} are weighted 1D matrices.
"""
import numpy as np

from .bspline import element_quadrature, default_nq
from .matrices import assemble_1d, restrict_space, restrict_time


class Discretization:
    """Space-time tensor-product spline discretisation of the unit box times (0, T).

    n_el: [n_el_t, n_el_1, ..., n_el_d]; p: [p_t, p_s] or [p_t, p_1, ..., p_d].
    potential: None, or a list of rank-one terms, each a list of d callables v_{r,l}(x_l).
    formulation: "ls" (the least-squares method: time basis without its first function) or "uw"
    (the ultraweak method of Sec. 4.4: the same matrix on the time basis without its last function,
    i.e. the space with final conditions; the unknowns z give u_h = S z_h).
    """

    def __init__(self, n_el, p, T=1.0, nu=1.0, potential=None, formulation="ls"):
        self.d = len(n_el) - 1
        self.n_el = list(n_el)
        if len(p) == 2 and self.d != 1:
            p = [p[0]] + [p[1]] * self.d
        self.p = list(p)
        self.T = float(T)
        self.nu = float(nu)
        self.potential = potential
        self.formulation = formulation
        self.nq = [default_nq(q) for q in self.p]
        lengths = [self.T] + [1.0] * self.d
        self.full = [assemble_1d(self.p[l], self.n_el[l], lengths[l]) for l in range(self.d + 1)]
        self.n = [self.n_el[0] + self.p[0] - 1] + [self.n_el[l] + self.p[l] - 2 for l in range(1, self.d + 1)]
        self.shape = tuple(self.n[l] for l in range(self.d, 0, -1)) + (self.n[0],)
        self.N_s = int(np.prod(self.n[1:]))
        self.N_dof = self.N_s * self.n[0]
        Ft = self.full[0]
        self.Lt = restrict_time(Ft["L"], formulation)
        self.Mt = restrict_time(Ft["M"], formulation)
        self.Wt = 1j * restrict_time(Ft["K"], formulation)
        self.Wsym = self.Wt + self.Wt.conj().T
        self.sp = [None] + [{k: restrict_space(v) for k, v in self.full[l].items()} for l in range(1, self.d + 1)]

    # -- quadrature helpers -------------------------------------------------------------------
    def quad(self, l):
        """Element Gauss points / weights of direction l (0 = time on (0,T), l >= 1 on (0,1))."""
        return element_quadrature(self.n_el[l], self.nq[l], self.T if l == 0 else 1.0)

    def weighted_space(self, l, fn, full=False):
        """Weighted matrices of direction l for the weight function fn(x_l) (restricted unless full)."""
        x, _ = self.quad(l)
        F = assemble_1d(self.p[l], self.n_el[l], 1.0, weight=fn(x))
        return F if full else {k: restrict_space(v) for k, v in F.items()}

    # -- Kronecker terms --------------------------------------------------------------------
    def terms(self, with_potential=True, full_time=False, full_space=False):
        """List of (coefficient, [T, S_1, ..., S_d]) with A = sum coef * S_d (x) ... (x) S_1 (x) T.

        full_time / full_space: use the unrestricted (all basis functions) 1D
        matrices in time / space; the liftings of Sec. 2.2 need those columns.
        """
        d, nu = self.d, self.nu
        if full_time:
            Ft = self.full[0]
            Lt, Mt = Ft["L"], Ft["M"]
            Wsym = 1j * (Ft["K"] - Ft["K"].T)
        else:
            Lt, Mt, Wsym = self.Lt, self.Mt, self.Wsym
        sp = [None] + [(self.full[l] if full_space else self.sp[l]) for l in range(1, d + 1)]
        M = [None] + [sp[l]["M"] for l in range(1, d + 1)]
        out = []
        # M_s (x) L_t
        out.append((1.0, [Lt] + M[1:]))
        # nu^2 B_s (x) M_t
        for l in range(1, d + 1):
            f = [Mt] + M[1:]
            f[l] = sp[l]["J"]
            out.append((nu ** 2, f))
            for k in range(1, d + 1):
                if k == l:
                    continue
                f = [Mt] + M[1:]
                f[l] = sp[l]["K2"].T
                f[k] = sp[k]["K2"]
                out.append((nu ** 2, f))
        # nu L_s (x) (W + W^*): the cross terms (i d_t u, -nu Delta v) + (-nu Delta u, i d_t v) after
        # integrating by parts in space, which needs u and v to vanish on the boundary. With the
        # unrestricted spatial functions (the lifting of boundary data, Sec. 2.2: f - S u_lift) the
        # terms stay as they are: -i nu K_t (x) K2_l^T + i nu K_t^T (x) K2_l (K2^T[i,j] = int b_j b''_i).
        for l in range(1, d + 1):
            if full_space:
                Kt = self.full[0]["K"] if full_time else restrict_time(self.full[0]["K"], self.formulation)
                f = [Kt] + M[1:]
                f[l] = sp[l]["K2"].T
                out.append((-1j * nu, f))
                f = [Kt.T] + M[1:]
                f[l] = sp[l]["K2"]
                out.append((1j * nu, f))
            else:
                f = [Wsym] + M[1:]
                f[l] = sp[l]["L"]
                out.append((nu, f))
        if with_potential and self.potential:
            V = self.potential
            R = len(V)
            for r in range(R):
                for r2 in range(R):
                    f = [Mt] + [self.weighted_space(l, (lambda x, a=V[r][l - 1], b=V[r2][l - 1]: a(x) * b(x)),
                                                    full_space)["M"]
                                for l in range(1, d + 1)]
                    out.append((1.0, f))
                Wr = [self.weighted_space(l, V[r][l - 1], full_space) for l in range(1, d + 1)]
                out.append((1.0, [Wsym] + [Wr[l - 1]["M"] for l in range(1, d + 1)]))
                for l in range(1, d + 1):
                    f = [Mt] + [Wr[k - 1]["M"] for k in range(1, d + 1)]
                    K2 = Wr[l - 1]["K2"]
                    f[l] = K2 + K2.T
                    out.append((-nu, f))
        return out

    # -- dense assembly and matrix-free application ----------------------------------------------
    def dense(self, with_potential=True):
        """Assembled A (dense, tiny meshes only): sum coef * kron(S_d, ..., S_1, T)."""
        A = np.zeros((self.N_dof, self.N_dof), dtype=complex)
        for c, f in self.terms(with_potential):
            K = f[0]
            for l in range(1, self.d + 1):
                K = np.kron(f[l], K)
            A += c * K
        return A

    def apply(self, x, with_potential=True):
        """A x by Eq. kron_vec_multi: each Kronecker term applied as d+1 mode products."""
        X = np.asarray(x, dtype=complex).reshape(self.shape)
        return apply_terms(self.terms(with_potential), X, self.d).ravel()

    def axis(self, l):
        """numpy axis of mode l (0 = time) in the (n_d, ..., n_1, n_t) layout."""
        return self.d - l if l > 0 else self.d


def apply_terms(terms, X, d):
    """sum over terms of coef * X x_time T x_1 S_1 ... x_d S_d (Eq. kron_vec_multi); X has shape (n_d..n_1, n_t)."""
    Y = None
    for c, f in terms:
        Z = X
        for l in range(d + 1):
            Z = mode_product(Z, f[l], d - l if l > 0 else d)
        Y = c * Z if Y is None else Y + c * Z
    return Y


def mode_product(X, J, axis):
    """m-mode product X x_m J of Sec. 3.3: contracts axis `axis` of X with the columns of J."""
    Y = np.tensordot(J, X, axes=([1], [axis]))
    return np.moveaxis(Y, 0, axis)
