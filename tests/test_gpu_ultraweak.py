"""GPU parity of the ultraweak formulation (Sec. 4.4) against the oracle: system mat-vec, the
preconditioner, the right-hand side (both entry points), PCG, and the error of u_h = S z_h."""
import numpy as np
import pytest

import paper_2311_18461_gb300 as S
from inputs import harmonic_potential, random_complex
from oracle import fd as ofd, rhs as orhs
from tests._common import rel_err, oracle_disc, sample_potential, sample_initial, sample_forcing, to_dev, to_np

pytestmark = pytest.mark.gpu

CASES = [([6, 9], [2, 3], None), ([5, 7, 6], [3, 2, 3], None), ([4, 6, 5], [2, 3, 3], "harmonic")]


def _pair(n_el, p, pot, prec=S.STST_PREC_FP64, T=0.8, nu=1.2):
    d = len(n_el) - 1
    V = harmonic_potential(d) if pot else None
    disc = oracle_disc(n_el, p, T=T, nu=nu, potential=V, formulation="uw")
    prob = S.Problem(d, n_el, p, T=T, nu=nu, prec_mode=prec, formulation=S.STST_FORM_UW)
    if V:
        prob.set_potential(sample_potential(prob, V), len(V))
    return disc, prob


@pytest.mark.parametrize("n_el,p,pot", CASES)
def test_apply_sys_matches_oracle(n_el, p, pot):
    disc, prob = _pair(n_el, p, pot)
    x = random_complex(disc.N_dof, 1)
    y = to_np(prob.apply_sys(to_dev(x)))
    assert rel_err(y, disc.apply(x)) < 1e-12
    prob.close()


@pytest.mark.parametrize("prec,tol", [(S.STST_PREC_FP64, 1e-11), (S.STST_PREC_FP32, 5e-5)])
@pytest.mark.parametrize("n_el,p,pot", CASES[:2])
def test_apply_prec_matches_oracle(n_el, p, pot, prec, tol):
    disc, prob = _pair(n_el, p, pot, prec)
    assert prob.build_fd() == 0
    r = random_complex(disc.N_dof, 2)
    s = to_np(prob.apply_prec(to_dev(r)))
    assert rel_err(s, ofd.FastDiagonalization(disc).apply(r)) < tol
    prob.close()


@pytest.mark.parametrize("entry", ["rhs", "noalloc"])
def test_rhs_matches_oracle(entry):
    nu = 1.2
    f = lambda t, x1, x2: (1 + 2j * t) * np.sin(np.pi * x1) * np.sin(np.pi * x2) + 0.3 * t * t
    u0 = [lambda x: np.sin(np.pi * np.asarray(x)) * (1 + 0.5j * np.asarray(x)),
          lambda x: np.asarray(x) * (1 - np.asarray(x)) + 0j]
    disc, prob = _pair([5, 7, 6], [3, 2, 3], None, nu=nu)
    fq = sample_forcing(prob, f)
    uq = sample_initial(prob, u0)
    b = prob.vec()
    fn = S.stst_rhs if entry == "rhs" else S.stst_rhs_noalloc
    fn(prob.h, fq, uq, b, None)
    ref = orhs.rhs_ultraweak(disc, f, lambda x1, x2: u0[0](x1) * u0[1](x2))
    assert rel_err(to_np(b), ref) < 1e-12
    prob.close()


def test_pcg_matches_dense_solve_and_u_h_error():
    """C1-like ultraweak solve: u = e^{i pi^2 t} sin(pi x); PCG z against the dense solve, and the
    L2(Q) error of u_h = S z_h from the GPU's z against the oracle's own."""
    n, p = 16, 3
    disc, prob = _pair([n, n], [p, p], None, T=1.0, nu=1.0)
    u0 = lambda x: np.sin(np.pi * x) + 0j
    b = prob.rhs(u0_qp=sample_initial(prob, [lambda x: np.sin(np.pi * np.asarray(x)) + 0j]))
    assert prob.build_fd() == 0
    x, st, it, rr = prob.pcg(b, tol=1e-12, maxit=200)
    assert st == 0 and rr <= 1e-12
    bo = orhs.rhs_ultraweak(disc, None, u0)
    assert rel_err(to_np(b), bo) < 1e-12
    z_ref = np.linalg.solve(disc.dense(), bo)
    assert rel_err(to_np(x), z_ref) < 1e-8

    def l2err(z):
        Sz, pts, wts = orhs.apply_S_on_grid(disc, z, extra=3)
        U = np.exp(1j * np.pi ** 2 * pts[0][None, :]) * np.sin(np.pi * pts[1][:, None])
        W = np.outer(wts[1], wts[0])
        return np.sqrt(np.sum(W * np.abs(Sz - U) ** 2) / np.sum(W * np.abs(U) ** 2))
    e_gpu, e_ref = l2err(to_np(x)), l2err(z_ref)
    assert e_gpu < 2e-2 and abs(e_gpu - e_ref) <= 1e-6 * e_ref
    prob.close()
