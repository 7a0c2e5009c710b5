"""The potential-aware preconditioner P_V (stst_set_prec_operator(h, 1); an extension of Eq.
prec_definition to S_V = i d_t + sum_l (-nu d_ll + v_l)) against the oracle's
PotentialFastDiagonalization, and its PCG against the oracle's PCG with P_V.

Tolerances as for P-hat: the FP64 Fast Diagonalization 1e-10 relative (eigenpairs of (G_l, M_l) refined
in FP64, banded solves with kappa(H_i) ~ 1e2), FP32 5e-5; PCG iterates within one iteration of the
oracle's and solutions within 1e-9.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2311_18461_gb300 as S
from inputs import CONFIGS, harmonic_potential, bump_potential, initial_factors, product_fn, random_complex
from oracle import fd as ofd, pcg as opcg, rhs as orhs
from tests._common import rel_err, oracle_disc, sample_potential, to_dev, to_np

pytestmark = pytest.mark.gpu


def _problem(n_el, p, prec=S.STST_PREC_FP64, T=1.0, nu=1.0, V=None):
    d = len(n_el) - 1
    pl = [p] * (d + 1) if isinstance(p, int) else list(p)
    V = harmonic_potential(d) if V is None else V
    prob = S.Problem(d, n_el, pl, T=T, nu=nu, prec_mode=prec)
    prob.set_potential(sample_potential(prob, V), len(V))
    S.stst_set_prec_operator(prob.h, 1)
    disc = oracle_disc(n_el, pl, T=T, nu=nu, potential=V)
    return prob, disc


@pytest.mark.parametrize("n_el,p", [([6, 9], [2, 3]), ([9, 11, 7], [2, 3, 2]), ([5, 6, 5, 4], [2, 2, 3, 2])])
def test_apply_prec_potential_fp64(n_el, p):
    prob, disc = _problem(n_el, p, T=0.9, nu=1.1)
    assert prob.build_fd() == 0
    r = random_complex(prob.n_dof, 31)
    s = to_np(prob.apply_prec(to_dev(r)))
    assert rel_err(s, ofd.PotentialFastDiagonalization(disc).apply(r)) < 1e-10
    prob.close()


@pytest.mark.parametrize("same", [True, False])
def test_apply_prec_potential_equal_meshes(same):
    """Equal meshes in both directions: with the same factor the two G_l are equal and share one
    eigendecomposition; with different factors they must not."""
    f1 = lambda x: 6.0 * (x - 0.5) ** 2
    f2 = f1 if same else (lambda x: 3.0 + 4.0 * x)
    one = lambda x: 1.0 + 0.0 * x
    prob, disc = _problem([8, 10, 10], [2, 3, 3], V=[[f1, one], [one, f2]])
    assert prob.build_fd() == 0
    r = random_complex(prob.n_dof, 34)
    s = to_np(prob.apply_prec(to_dev(r)))
    assert rel_err(s, ofd.PotentialFastDiagonalization(disc).apply(r)) < 1e-10
    prob.close()


@pytest.mark.parametrize("n_el,p,V", [
    ([6, 9], [2, 3], [[lambda x: -100.0 * x * (1 - x)]]),
    ([8, 10, 9], [2, 3, 2], [[lambda x: -100.0 * x * (1 - x), lambda x: 1.0 + 0.0 * x],
                             [lambda x: 1.0 + 0.0 * x, lambda x: 3.0 + 4.0 * x]]),
])
def test_apply_prec_potential_with_negative_eigenvalues(n_el, p, V):
    """A negative factor makes G_l = nu L_l + M_{v_l} indefinite: some eigenvalues of (G_l, M_l) are
    negative (the Sturm-count bracket of the eigensolver and the lambda < 0 sign of the advection term
    in H_i). H_i stays Hermitian positive definite for every real lambda."""
    prob, disc = _problem(n_el, p, V=V)
    F = ofd.PotentialFastDiagonalization(disc)
    assert F.lam[1].min() < 0 < F.lam[1].max()
    assert prob.build_fd() == 0
    r = random_complex(prob.n_dof, 35)
    s = to_np(prob.apply_prec(to_dev(r)))
    assert rel_err(s, F.apply(r)) < 1e-10
    prob.close()


def test_apply_prec_potential_fp32():
    prob, disc = _problem([9, 11, 7], [2, 3, 2], prec=S.STST_PREC_FP32)
    assert prob.build_fd() == 0
    r = random_complex(prob.n_dof, 32)
    s = to_np(prob.apply_prec(to_dev(r)))
    assert rel_err(s, ofd.PotentialFastDiagonalization(disc).apply(r)) < 5e-5
    prob.close()


def test_pcg_with_potential_prec_follows_the_oracle():
    """2D+t p = 3, harmonic V, wavepacket datum at n_el = 16: to 1e-10 the oracle takes 10 iterations with
    P_V (to 1e-8: 8, against 11 with P-hat); the GPU's FP64 solve follows it."""
    cfg = dict(CONFIGS["c2"])
    n_el = [16, 16, 16]
    prob, disc = _problem(n_el, cfg["p"])
    b = orhs.rhs_initial(disc, None, product_fn(initial_factors(cfg)))[0]
    assert prob.build_fd() == 0
    x, st, it, rr = prob.pcg(to_dev(b), tol=1e-10, maxit=200)
    xo, ito, _, _ = opcg.pcg(disc.apply, ofd.PotentialFastDiagonalization(disc).apply, b, tol=1e-10, maxit=200)
    assert st == 0 and abs(it - ito) <= 1
    assert rel_err(to_np(x), xo) < 1e-9
    prob.close()


def test_prec_operator_switch_and_errors():
    prob, disc = _problem([6, 7, 5], [2, 3, 2])
    with pytest.raises(S.StstError):
        S.stst_set_prec_operator(prob.h, 2)
    assert prob.build_fd() == 0
    r = to_dev(random_complex(prob.n_dof, 33))
    s1 = to_np(prob.apply_prec(r))
    S.stst_set_prec_operator(prob.h, 0)                 # back to P-hat: rebuild needed
    with pytest.raises(S.StstError) as e:
        prob.apply_prec(r)
    assert e.value.status == -5
    assert prob.build_fd() == 0
    s0 = to_np(prob.apply_prec(r))
    assert rel_err(s0, ofd.FastDiagonalization(disc).apply(to_np(r))) < 1e-10
    assert rel_err(s1, s0) > 1e-3                       # the two preconditioners differ
    # a product potential is not a sum of one-direction factors
    bump = bump_potential(2)
    with pytest.raises(S.StstError):
        prob.set_potential(sample_potential(prob, bump), 1)
        S.stst_set_prec_operator(prob.h, 1)
    S.stst_set_prec_operator(prob.h, 0)
    prob.set_potential(sample_potential(prob, harmonic_potential(2)), 2)
    S.stst_set_prec_operator(prob.h, 1)
    prob.set_potential(sample_potential(prob, bump), 1)  # installed after selecting P_V
    with pytest.raises(S.StstError) as e:
        prob.build_fd()
    assert e.value.status == -5
    prob.close()
