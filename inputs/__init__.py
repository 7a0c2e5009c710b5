"""Seeded synthetic inputs shared by the oracle tests and the CUDA-path tests / bench.

This module holds none of the solver's arithmetic: it only names the
workloads and draws their data (initial wavepackets, potentials, random
vectors) from fixed seeds. Every datum is returned as plain functions of the
coordinates; each consumer samples them at its own quadrature points.

Workloads (the paper's experiments are analytic, so these synthetic data
stand in for them exactly; sizes follow the 2D+t performance study, Table 1):
  c1     1D+t, p=2, 32 x 32 elements, V=0, u = exp(i pi^2 t) sin(pi x) (f = 0, u0 = sin(pi x)), tol 1e-10
  c2     2D+t, p=3, 64^2 x 64 elements, V = 10 |x - 1/2|^2 / (d/4), windowed Gaussian wavepacket (seed 0), tol 1e-8
  c3p2 / c3p4   3D+t, p=2 / 4, 32^3 x 64 elements, V = 0 or a Gaussian bump, wavepacket (seed 1)
  c4     128 2D+t instances, n_el in {16..96}^2 x {16..96}, p in {2,3,4}, seeded per instance (4 + i)
  c5     2D+t, p=3, 48^2 x 48, harmonic V, wavepackets with drawn centre/width/momentum/phase
  geometry (module inputs.geometry): analytic maps F of the unit box (identity, affine, quarter annulus,
         perturbed box) with their first and second derivatives, for the mapped-domain system
  tw     the travelling wave of the paper's performance study (Sec. 6.2, Table 1): 2D+t, V = 0,
         u = a exp(-i (|x|^2 + t^2) / w^2), w = 0.2, with its Dirichlet and initial values imposed
"""
import math

import numpy as np

CONFIGS = {
    "c1": dict(d=1, n_el=[32, 32], p=2, T=1.0, nu=1.0, potential=None, u0="sine", tol=1e-10),
    "c2": dict(d=2, n_el=[64, 64, 64], p=3, T=1.0, nu=1.0, potential="harmonic", u0=("wavepacket", 0), tol=1e-8),
    "c3p2": dict(d=3, n_el=[64, 32, 32, 32], p=2, T=1.0, nu=1.0, potential=None, u0=("wavepacket", 1), tol=1e-8),
    "c3p4": dict(d=3, n_el=[64, 32, 32, 32], p=4, T=1.0, nu=1.0, potential=None, u0=("wavepacket", 1), tol=1e-8),
    "c3p2_bump": dict(d=3, n_el=[64, 32, 32, 32], p=2, T=1.0, nu=1.0, potential="bump", u0=("wavepacket", 1), tol=1e-8),
    "c3p4_bump": dict(d=3, n_el=[64, 32, 32, 32], p=4, T=1.0, nu=1.0, potential="bump", u0=("wavepacket", 1), tol=1e-8),
    "c5": dict(d=2, n_el=[48, 48, 48], p=3, T=1.0, nu=1.0, potential="harmonic", u0=("wavepacket", 5), tol=1e-8),
    "tw": dict(d=2, n_el=[64, 64, 64], p=3, T=1.0, nu=1.0, potential=None, u0="travelling_wave", tol=1e-8),
}


def scaled(cfg, n_el):
    """The same workload on a smaller mesh (parity-test sizes)."""
    out = dict(cfg)
    out["n_el"] = list(n_el)
    return out


# ---- potentials: lists of rank-one terms, each a list of d real callables -------------------------
def harmonic_potential(d, vmax=10.0):
    """V(x) = vmax |x - 1/2|^2 / (d/4): the squared distance to the centre scaled to [0, vmax] on (0,1)^d."""
    s = vmax / (d / 4.0)
    one = lambda x: np.ones_like(np.asarray(x, dtype=float))
    terms = []
    for r in range(d):
        terms.append([(lambda x, s=s: s * (np.asarray(x) - 0.5) ** 2) if l == r else one for l in range(d)])
    return terms


def bump_potential(d, amp=10.0, width2=0.05):
    """V(x) = amp exp(-|x - 1/2|^2 / width2): one rank-one term."""
    f0 = lambda x, a=amp ** (1.0 / d): a * np.exp(-(np.asarray(x) - 0.5) ** 2 / width2)
    return [[f0 for _ in range(d)]]


def random_smooth_potential(rng, d, vmax=10.0):
    """Random separable smooth potential of rank <= 3 with values in [0, vmax] (batched instances)."""
    rank = int(rng.integers(1, 4))
    terms = []
    for _ in range(rank):
        amp = (vmax / rank) ** (1.0 / d)
        fs = []
        for _ in range(d):
            c = rng.uniform(0.2, 0.8)
            w = rng.uniform(0.05, 0.3)
            fs.append(lambda x, c=c, w=w, a=amp: a * np.exp(-(np.asarray(x) - c) ** 2 / (2 * w * w)))
        terms.append(fs)
    return terms


def potential(cfg):
    if cfg["potential"] is None:
        return None
    if cfg["potential"] == "harmonic":
        return harmonic_potential(cfg["d"])
    if cfg["potential"] == "bump":
        return bump_potential(cfg["d"])
    raise ValueError(cfg["potential"])


# ---- initial data ---------------------------------------------------------------------------------
def wavepacket_params(rng, d):
    """Centre c ~ U[0.3,0.7]^d, width sigma ~ U[0.05,0.15], momentum k ~ U[-20,20]^d, phase ~ U[0, 2 pi)."""
    c = rng.uniform(0.3, 0.7, size=d)
    sigma = rng.uniform(0.05, 0.15)
    k = rng.uniform(-20.0, 20.0, size=d)
    phi = rng.uniform(0.0, 2 * math.pi)
    return dict(c=c, sigma=sigma, k=k, phi=phi)


def wavepacket_factors(par):
    """u0 = prod_l g_l(x_l): g_l = exp(-(x-c_l)^2/(2 sigma^2) + i k_l x) sin(pi x), phase on g_1.

    The sin(pi x) window makes the datum vanish on the boundary (homogeneous Dirichlet data).
    """
    d = len(par["c"])
    out = []
    for l in range(d):
        ph = par["phi"] if l == 0 else 0.0
        out.append(lambda x, c=par["c"][l], s=par["sigma"], k=par["k"][l], ph=ph:
                   np.exp(-(np.asarray(x) - c) ** 2 / (2 * s * s) + 1j * (k * np.asarray(x) + ph)) * np.sin(np.pi * np.asarray(x)))
    return out


def initial_factors(cfg, seed_offset=0):
    """Separable factors of u0 for a workload (None for the travelling wave: its data come from u)."""
    d = cfg["d"]
    if cfg["u0"] == "travelling_wave":
        return None
    if cfg["u0"] == "sine":
        return [lambda x: np.sin(np.pi * np.asarray(x)) + 0j for _ in range(d)]
    kind, seed = cfg["u0"]
    rng = np.random.default_rng(seed + seed_offset)
    return wavepacket_factors(wavepacket_params(rng, d))


def product_fn(factors):
    """u(x_1, ..., x_d) = prod_l factors[l](x_l), broadcasting over its arguments."""
    def fn(*xs):
        out = 1.0
        for l, g in enumerate(factors):
            out = out * g(xs[l])
        return out
    return fn


def c4_instances(n=128):
    """Batched workload: per instance i, rng(4 + i) draws the mesh, degree, potential and wavepacket."""
    out = []
    for i in range(n):
        rng = np.random.default_rng(4 + i)
        ns = [int(v) for v in rng.integers(16, 97, size=3)]
        p = int(rng.integers(2, 5))
        V = random_smooth_potential(rng, 2)
        wp = wavepacket_params(rng, 2)
        out.append(dict(d=2, n_el=[ns[2], ns[0], ns[1]], p=p, T=1.0, nu=1.0, potential_terms=V,
                        u0_factors=wavepacket_factors(wp), tol=1e-8, params=wp))
    return out


def random_complex(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


# ---- the travelling wave of the performance study (Sec. 6.2, Table 1) ------------------------------
TW_OMEGA = 0.2


def travelling_wave(omega=TW_OMEGA, xp=np):
    """(u, f) for u = a exp(-i (x_1^2 + x_2^2 + t^2) / w^2), a = (2 / w^2)^(1/4), and the forcing the
    paper prints for it, f = i u_t - Delta u = a (4i / w^2 + 4 |x|^2 / w^4 + 2 t / w^2) exp(...) (nu = 1).
    xp: the array module the callables use (numpy, or torch for device grids)."""
    a = (2.0 / omega ** 2) ** 0.25
    w2 = omega ** 2

    def u(t, x1, x2):
        return a * xp.exp(-1j * (x1 ** 2 + x2 ** 2 + t ** 2) / w2)

    def f(t, x1, x2):
        r2 = x1 ** 2 + x2 ** 2
        return a * (4j / w2 + 4 * r2 / w2 ** 2 + 2 * t / w2) * xp.exp(-1j * (r2 + t ** 2) / w2)

    return u, f
