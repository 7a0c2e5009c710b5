"""Helpers shared by the GPU parity tests: build both sides of a comparison from one workload."""
import numpy as np

from inputs import potential as cfg_potential, initial_factors, product_fn
from oracle.system import Discretization


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


def oracle_disc(n_el, p, T=1.0, nu=1.0, potential=None, formulation="ls"):
    d = len(n_el) - 1
    pl = [p] * (d + 1) if isinstance(p, int) else list(p)
    return Discretization(n_el, pl, T=T, nu=nu, potential=potential, formulation=formulation)


def sample_potential(prob, terms):
    """Pack the potential factors at the library's quadrature points (rank-major, then direction)."""
    import torch
    cols = []
    for term in terms:
        for l in range(1, prob.d + 1):
            x = prob.quad_points(l).cpu().numpy()
            cols.append(np.asarray(term[l - 1](x), dtype=np.float64) * np.ones_like(x))
    return torch.tensor(np.concatenate(cols), dtype=torch.float64, device="cuda")


def sample_initial(prob, factors):
    """u0 on the library's spatial quadrature grid, x_1 fastest."""
    import torch
    grids = [prob.quad_points(l).cpu().numpy() for l in range(1, prob.d + 1)]
    u = np.ones([1] * prob.d, dtype=complex)
    for l, g in enumerate(factors):
        shp = [1] * prob.d
        shp[prob.d - 1 - l] = len(grids[l])
        u = u * np.asarray(g(grids[l])).reshape(shp)
    return torch.tensor(np.ascontiguousarray(u).ravel(), dtype=torch.complex128, device="cuda")


def sample_forcing(prob, f):
    """f(t, x_1, ..., x_d) on the library's space-time quadrature grid, time fastest."""
    import torch
    grids = [prob.quad_points(l).cpu().numpy() for l in range(prob.d + 1)]
    d = prob.d
    co = []
    for l in range(d + 1):
        shp = [1] * (d + 1)
        shp[d if l == 0 else d - l] = len(grids[l])
        co.append(grids[l].reshape(shp))
    F = np.broadcast_to(f(*co), tuple(len(grids[l]) for l in range(d, 0, -1)) + (len(grids[0]),))
    return torch.tensor(np.ascontiguousarray(F).ravel(), dtype=torch.complex128, device="cuda")


def to_dev(v):
    import torch
    return torch.tensor(np.asarray(v, dtype=complex), dtype=torch.complex128, device="cuda")


def to_np(t):
    return t.detach().cpu().numpy()
