"""Load vector and liftings of non-homogeneous data (Sec. 2.2, Sec. 4.3).

Test infrastructure: part of the CPU oracle, see `oracle/__init__.py`.

[f]_i = F(S B_i) = int_Q f conj(S B_i); with real basis functions
conj(S B_i) = -i b_t' B_s - nu b_t Delta B_s (+ V b_t B_s with a potential).
(The printed formula in Sec. 4.3 drops nu in "- Delta v_h"; it is read as -nu Delta.)

Liftings (Sec. 2.2: u = u_bar + lifting, f_bar = f - S lifting):
* initial datum only (homogeneous Dirichlet data): u0 is L2-projected onto the
  Dirichlet-reduced spatial space, c = M_s^{-1} (u0, B_s), and attached to the
  first time basis function b_1(t) (the only one nonzero at t = 0). Then
  rhs_i = [f]_i - sum_j A_full(B_{(1,j)}, S B_i) c_j, using the first columns of
  the unrestricted time matrices.
* general Dirichlet and initial data (tiny meshes): the exact solution is
  L2-projected onto the whole space-time spline space and the coefficients of
  the basis functions that do not vanish on the initial face or the lateral
  boundary are kept as the lifting.
Integrals use the tensor Gauss rule of `bspline.element_quadrature`.
"""
import numpy as np

from .bspline import open_uniform_knots, basis_all
from .system import apply_terms, mode_product


def tables(disc, l, pts=None, full=False):
    """D[s, q, i] = d^s b_i(x_q) for direction l at its quadrature points (or `pts`)."""
    length = disc.T if l == 0 else 1.0
    x = disc.quad(l)[0] if pts is None else np.asarray(pts, dtype=float)
    D = basis_all(open_uniform_knots(disc.p[l], disc.n_el[l]), disc.p[l], x / length, nder=2)
    D = D / np.array([1.0, length, length ** 2])[:, None, None]
    if not full:
        if l == 0:
            D = D[:, :, :-1] if disc.formulation == "uw" else D[:, :, 1:]
        else:
            D = D[:, :, 1:-1]
    return D


def grid_coords(disc, pts=None, time=True):
    """Broadcastable coordinate arrays (t, x_1, ..., x_d) in the (Q_d, ..., Q_1, Q_t) layout."""
    d = disc.d
    pts = [disc.quad(l)[0] for l in range(d + 1)] if pts is None else pts
    nax = d + 1 if time else d
    out = []
    for l in range(0 if time else 1, d + 1):
        shp = [1] * nax
        ax = (d if l == 0 else d - l) if time else d - l
        shp[ax] = len(pts[l])
        out.append(np.asarray(pts[l]).reshape(shp))
    return out


def grid_weights(disc, time=True):
    d = disc.d
    W = np.ones([1] * (d + 1 if time else d))
    for l in range(0 if time else 1, d + 1):
        w = disc.quad(l)[1]
        shp = [1] * (d + 1 if time else d)
        shp[(d if l == 0 else d - l) if time else d - l] = len(w)
        W = W * w.reshape(shp)
    return W


def potential_fn(disc):
    """V(x) from its separable factors, or None."""
    if not disc.potential:
        return None

    def V(*xs):
        tot = 0.0
        for term in disc.potential:
            prod = 1.0
            for l, v in enumerate(term):
                prod = prod * v(xs[l])
            tot = tot + prod
        return tot
    return V


def load_vector(disc, f_fn):
    """[f]_i = int f conj(S B_i) (+ int f V B_i), by tensor quadrature and mode products."""
    d, nu = disc.d, disc.nu
    co = grid_coords(disc)
    F = f_fn(*co) * grid_weights(disc)
    F = np.broadcast_to(F, tuple(len(disc.quad(l)[0]) for l in range(d, 0, -1)) + (len(disc.quad(0)[0]),))
    T = [tables(disc, l) for l in range(d + 1)]

    def contract(G, tab_t, sp_ders):
        Z = mode_product(G, tab_t.T, d)
        for l in range(1, d + 1):
            Z = mode_product(Z, T[l][sp_ders[l - 1]].T, d - l)
        return Z

    out = -1j * contract(F, T[0][1], [0] * d)
    for l in range(d):
        ders = [0] * d
        ders[l] = 2
        out = out - nu * contract(F, T[0][0], ders)
    V = potential_fn(disc)
    if V is not None:
        out = out + contract(F * V(*co[1:]), T[0][0], [0] * d)
    return out.ravel()


def project_initial(disc, u0_fn):
    """c = M_s^{-1} (u0, B_s): L2 projection of u0 onto the Dirichlet-reduced spatial space."""
    d = disc.d
    co = grid_coords(disc, time=False)
    G = u0_fn(*co) * grid_weights(disc, time=False)
    for l in range(1, d + 1):
        G = mode_product(G, tables(disc, l)[0].T, d - l)
    for l in range(1, d + 1):
        G = mode_product(G, np.linalg.inv(disc.sp[l]["M"]), d - l)
    return G


def initial_lifting(disc, c):
    """The vector sum_j A_full(B_{(1,j)}, S B_i) c_j over the reduced rows i."""
    d = disc.d
    m_t = disc.n[0] + 1
    X0 = np.zeros(np.shape(c) + (m_t,), dtype=complex)
    X0[..., 0] = c
    Y = apply_terms(disc.terms(full_time=True), X0, d)
    return Y[..., 1:].ravel()


def rhs_initial(disc, f_fn=None, u0_fn=None):
    """rhs of the reduced system for forcing f and initial datum u0 with homogeneous Dirichlet data.

    Returns (rhs, c); the discrete solution is u_h = u_bar_h + b_1(t) sum_j c_j B_j(x).
    """
    rhs = np.zeros(disc.N_dof, dtype=complex) if f_fn is None else load_vector(disc, f_fn)
    c = None
    if u0_fn is not None:
        c = project_initial(disc, u0_fn)
        rhs = rhs - initial_lifting(disc, c)
    return rhs, c


def full_lifting(disc, u_fn, f_fn):
    """rhs and lifting coefficients for general Dirichlet/initial data taken from the exact solution u."""
    d = disc.d
    co = grid_coords(disc)
    G = u_fn(*co) * grid_weights(disc)
    for l in range(d + 1):
        G = mode_product(G, tables(disc, l, full=True)[0].T, d if l == 0 else d - l)
    for l in range(d + 1):
        G = mode_product(G, np.linalg.inv(disc.full[l]["M"]), d if l == 0 else d - l)
    mask = np.zeros(G.shape, dtype=bool)
    mask[..., 0] = True
    for l in range(1, d + 1):
        idx = [slice(None)] * (d + 1)
        idx[d - l] = 0
        mask[tuple(idx)] = True
        idx[d - l] = -1
        mask[tuple(idx)] = True
    XD = np.where(mask, G, 0.0)
    Y = apply_terms(disc.terms(full_time=True, full_space=True), XD, d)
    sl = tuple([slice(1, -1)] * d + [slice(1, None)])
    rhs = load_vector(disc, f_fn) - Y[sl].ravel()
    return rhs, XD


def embed_solution(disc, ubar, XD=None, c=None):
    """Full coefficient tensor (all basis functions) of u_h from the reduced solution and a lifting."""
    d = disc.d
    shape = tuple(disc.n[l] + 2 for l in range(d, 0, -1)) + (disc.n[0] + 1,)
    U = np.zeros(shape, dtype=complex) if XD is None else np.array(XD, dtype=complex)
    sl = tuple([slice(1, -1)] * d + [slice(1, None)])
    U[sl] += np.asarray(ubar).reshape(disc.shape)
    if c is not None:
        U[tuple([slice(1, -1)] * d + [0])] += c
    return U


def spatial_load(disc, u0_fn):
    """g_j = (u0, B_j)_{L2(Omega)} on the Dirichlet-reduced spatial basis (tensor Gauss rule)."""
    d = disc.d
    co = grid_coords(disc, time=False)
    G = u0_fn(*co) * grid_weights(disc, time=False)
    for l in range(1, d + 1):
        G = mode_product(G, tables(disc, l)[0].T, d - l)
    return G


def rhs_ultraweak(disc, f_fn=None, u0_fn=None):
    """Right-hand side of the ultraweak method (Sec. 4.4): b_i = (f, B_i) + i (u0, B_i(., 0)).

    The basis functions B_i = b_k(t) B_j(x) span the space with final conditions; the only time
    function nonzero at t = 0 is the first one, b_0(0) = 1, so the initial term sits on time index 0.
    With u_h = S z_h, the method reads (S z_h, S B_i) = b_i (the matrix of the least-squares form on
    this space)."""
    assert disc.formulation == "uw"
    d = disc.d
    out = np.zeros(disc.shape, dtype=complex)
    if f_fn is not None:
        co = grid_coords(disc)
        F = f_fn(*co) * grid_weights(disc)
        F = np.broadcast_to(F, tuple(len(disc.quad(l)[0]) for l in range(d, 0, -1)) + (len(disc.quad(0)[0]),))
        Z = mode_product(F, tables(disc, 0)[0].T, d)
        for l in range(1, d + 1):
            Z = mode_product(Z, tables(disc, l)[0].T, d - l)
        out = out + Z
    if u0_fn is not None:
        out[..., 0] += 1j * spatial_load(disc, u0_fn)
    return out.ravel()


def apply_S_on_grid(disc, z, V=None, extra=0):
    """Values of S z_h = i d_t z_h - nu Delta z_h (+ V z_h) on a tensor Gauss grid with `extra` more
    points per element than the library's rule, and that grid's points and weights (for L2(Q) errors of
    the ultraweak solution u_h = S z_h)."""
    from .bspline import element_quadrature
    d, nu = disc.d, disc.nu
    pts, wts, tabs = [], [], []
    for l in range(d + 1):
        length = disc.T if l == 0 else 1.0
        x, w = element_quadrature(disc.n_el[l], disc.nq[l] + extra, length)
        pts.append(x)
        wts.append(w)
        tabs.append(tables(disc, l, pts=x))
    Z = np.asarray(z, dtype=complex).reshape(disc.shape)

    def ev(tder, sders):
        Y = mode_product(Z, tabs[0][tder], d)
        for l in range(1, d + 1):
            Y = mode_product(Y, tabs[l][sders[l - 1]], d - l)
        return Y

    S = 1j * ev(1, [0] * d)
    for l in range(d):
        ders = [0] * d
        ders[l] = 2
        S = S - nu * ev(0, ders)
    if V is not None:
        co = np.meshgrid(*[pts[l] for l in range(d, 0, -1)], indexing="ij")
        S = S + V(*co[::-1])[..., None] * ev(0, [0] * d)
    return S, pts, wts
