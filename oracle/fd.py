"""The preconditioner P-hat and its Fast Diagonalization (Eq. prec_definition, Eq. space_eig,
Eq. preconditioner_str2, Algorithm 1 of Sec. 5).

Test infrastructure: part of the CPU oracle, see `oracle/__init__.py`.

P-hat = M_s (x) L_t + nu^2 L_s^T M_s^{-1} L_s (x) M_t + nu L_s (x) (W_t + W_t^*)
with the spatial factors of the parametric box (0,1)^d (the spatial matrices
of the potential-free operator, Sec. 5). Algorithm 1:
  1. generalized eigendecompositions L_l U_l = M_l U_l Lambda_l, U_l^T M_l U_l = I;
  2. y = (U_s^T (x) I_t) r;
  3. x_i = H_i^{-1} y_i with H_i = L_t + nu^2 lambda_i^2 M_t + nu lambda_i (W_t + W_t^*),
     lambda_i = [Lambda_s]_{ii} = sum_l lambda_{l, i_l};
  4. s = (U_s (x) I_t) x.
(Step 4 prints an undefined s-tilde; it is read as the vector x of step 3.)
"""
import numpy as np
import scipy.linalg

from .system import mode_product


def dense_P(disc):
    """Assembled P-hat (dense; tiny meshes only), straight from Eq. prec_definition."""
    d, nu = disc.d, disc.nu
    Ms = np.ones((1, 1))
    Ls = np.zeros((1, 1))
    for l in range(1, d + 1):
        M, L = disc.sp[l]["M"], disc.sp[l]["L"]
        Ls = np.kron(M, Ls) + np.kron(L, Ms)
        Ms = np.kron(M, Ms)
    LML = Ls.T @ np.linalg.solve(Ms, Ls)
    return np.kron(Ms, disc.Lt) + nu ** 2 * np.kron(LML, disc.Mt) + nu * np.kron(Ls, disc.Wsym)


class FastDiagonalization:
    """Algorithm 1 (setup = step 1 and the H_i; apply = steps 2-4).

    scales: None, or per-direction factors s_l multiplying the eigenvalues of step 1 (a mapped domain:
    `oracle.geometry.prec_scales`). With s_l = 1 / a_l^2 this is the preconditioner of the box with sides
    a_l divided by prod_l a_l (its stiffness L_l / a_l and mass a_l M_l have the eigenvectors of (L_l, M_l)
    scaled by a_l^{-1/2} and the eigenvalues scaled by 1 / a_l^2); PCG does not see the constant factor.
    """

    def __init__(self, disc, scales=None):
        self.disc = disc
        self.U, self.lam = [None], [None]
        for l in range(1, disc.d + 1):
            lam, U = scipy.linalg.eigh(disc.sp[l]["L"], disc.sp[l]["M"])   # step 1, Eq. space_eig
            if scales is not None:
                lam = scales[l - 1] * lam
            self.U.append(U)
            self.lam.append(lam)
        # Lambda_s in vec order (x_1 fastest): spatial array of shape (n_d, ..., n_1)
        lam_s = np.zeros(disc.shape[:-1])
        for l in range(1, disc.d + 1):
            shp = [1] * disc.d
            shp[disc.d - l] = disc.n[l]
            lam_s = lam_s + self.lam[l].reshape(shp)
        self.lam_s = lam_s.ravel()

    def H(self, lam_i):
        """H_i = L_t + nu^2 lambda_i^2 M_t + nu lambda_i (W_t + W_t^*)."""
        disc = self.disc
        return disc.Lt + disc.nu ** 2 * lam_i ** 2 * disc.Mt + disc.nu * lam_i * disc.Wsym

    def apply(self, r, chunk=512):
        """s = P-hat^{-1} r by steps 2-4 of Algorithm 1."""
        disc = self.disc
        Y = np.asarray(r, dtype=complex).reshape(disc.shape)
        for l in range(1, disc.d + 1):                      # step 2: y = (U_s^T (x) I) r
            Y = mode_product(Y, self.U[l].T, disc.axis(l))
        Yf = Y.reshape(disc.N_s, disc.n[0])
        Xf = np.empty_like(Yf)
        for a in range(0, disc.N_s, chunk):                 # step 3: x_i = H_i^{-1} y_i (pagewise solve)
            lam = self.lam_s[a:a + chunk]
            Hs = np.stack([self.H(li) for li in lam])
            Xf[a:a + chunk] = np.linalg.solve(Hs, Yf[a:a + chunk][:, :, None])[:, :, 0]
        X = Xf.reshape(disc.shape)
        for l in range(1, disc.d + 1):                      # step 4: s = (U_s (x) I) x
            X = mode_product(X, self.U[l], disc.axis(l))
        return X.ravel()

    def kappa_U(self, l):
        """kappa_2(U_l) = ||U_l||_2 ||U_l^{-1}||_2 (Table cond_number_space)."""
        return np.linalg.cond(self.U[l], 2)


# ------------------------------------------------------------------------------------------------
# Potential-aware variant (an extension: the paper treats V = 0). For V = sum_l v_l(x_l) the
# operator is S_V = i d_t + sum_l H_l with H_l = -nu d_ll + v_l; the construction of Eq.
# prec_definition applied to it replaces the spatial stiffness nu L_s by the Kronecker sum of the
# Galerkin matrices G_l = nu L_l + M_{v_l} of the H_l:
#   P_V = M_s (x) L_t + H_s^T M_s^{-1} H_s (x) M_t + H_s (x) (W_t + W_t^*),  H_s = sum_l G_l (Kronecker sum).
# Algorithm 1 is unchanged with the generalized eigenpairs of (G_l, M_l) and
# H_i = L_t + lambda_i^2 M_t + lambda_i (W_t + W_t^*) (nu is inside G_l). With V = 0 this is P-hat.

def additive_factors(disc):
    """v_l for each spatial direction (None where V has no factor there), if the potential is a sum of
    one-direction factors with at most one per direction; raises ValueError otherwise. A factor counts as
    absent where it equals 1 at every quadrature point of its direction."""
    d = disc.d
    out = [None] * (d + 1)
    for term in (disc.potential or []):
        live = [l for l in range(1, d + 1) if not np.all(term[l - 1](disc.quad(l)[0]) == 1.0)]
        if len(live) != 1 or out[live[0]] is not None:
            raise ValueError("potential is not a sum of one-direction factors")
        out[live[0]] = term[live[0] - 1]
    return out


def anova_factors(disc):
    """First-order ANOVA terms of a separable V = sum_r prod_l f_{r,l}(x_l) on the unit cube:
    g_l(x_l) = E[V | x_l] - ((d-1)/d) E[V] = sum_r f_{r,l}(x_l) prod_{k != l} mu_{r,k} - ((d-1)/d) sum_r prod_k mu_{r,k},
    mu_{r,k} the mean of f_{r,k} over (0,1) (direction k's Gauss rule). sum_l g_l is the L2-best additive
    approximation of V; for an additive V it is V itself."""
    d = disc.d
    V = disc.potential or []
    mu = []
    for term in V:
        row = []
        for k in range(1, d + 1):
            x, w = disc.quad(k)
            row.append(float(np.sum(w * term[k - 1](x))))
        mu.append(row)
    V0 = sum(np.prod(row) for row in mu)
    out = [None]
    for l in range(1, d + 1):
        coefs = [np.prod([mu[r][k - 1] for k in range(1, d + 1) if k != l]) for r in range(len(V))]
        out.append(lambda x, l=l, coefs=coefs: sum(c * V[r][l - 1](x) for r, c in enumerate(coefs))
                   - (d - 1) / d * V0 + 0.0 * np.asarray(x))
    return out


def spatial_operators(disc, approximate=False):
    """G_l = nu L_l + M_{v_l} (restricted spatial bases), l = 1..d. approximate=True takes the ANOVA terms
    g_l in place of the v_l, for any separable potential."""
    if approximate:
        g = anova_factors(disc)
        return [None] + [disc.nu * disc.sp[l]["L"] + disc.weighted_space(l, g[l])["M"] for l in range(1, disc.d + 1)]
    v = additive_factors(disc)
    G = [None]
    for l in range(1, disc.d + 1):
        g = disc.nu * disc.sp[l]["L"]
        if v[l] is not None:
            g = g + disc.weighted_space(l, v[l])["M"]
        G.append(g)
    return G


def dense_P_potential(disc, approximate=False):
    """Assembled P_V (dense; tiny meshes only), straight from its definition above."""
    G = spatial_operators(disc, approximate)
    Ms = np.ones((1, 1))
    Hs = np.zeros((1, 1))
    for l in range(1, disc.d + 1):
        M = disc.sp[l]["M"]
        Hs = np.kron(M, Hs) + np.kron(G[l], Ms)
        Ms = np.kron(M, Ms)
    HMH = Hs.T @ np.linalg.solve(Ms, Hs)
    return np.kron(Ms, disc.Lt) + np.kron(HMH, disc.Mt) + np.kron(Hs, disc.Wsym)


class PotentialFastDiagonalization(FastDiagonalization):
    """Algorithm 1 for P_V: eigenpairs of (G_l, M_l) in step 1, H_i without the factor nu in step 3."""

    def __init__(self, disc, approximate=False):
        self.disc = disc
        self.U, self.lam = [None], [None]
        G = spatial_operators(disc, approximate)
        for l in range(1, disc.d + 1):
            lam, U = scipy.linalg.eigh(G[l], disc.sp[l]["M"])
            self.U.append(U)
            self.lam.append(lam)
        lam_s = np.zeros(disc.shape[:-1])
        for l in range(1, disc.d + 1):
            shp = [1] * disc.d
            shp[disc.d - l] = disc.n[l]
            lam_s = lam_s + self.lam[l].reshape(shp)
        self.lam_s = lam_s.ravel()

    def H(self, lam_i):
        """H_i = L_t + lambda_i^2 M_t + lambda_i (W_t + W_t^*)."""
        disc = self.disc
        return disc.Lt + lam_i ** 2 * disc.Mt + lam_i * disc.Wsym
