"""The flexible CG of the mixed-precision path (FP32 or BF16x3 preconditioner inside the FP64 solve)
against the oracle's flexible CG (`oracle.pcg.fcg`, pinned in tests/test_oracle_fcg_pins.py).

1. Iterates: the oracle's flexible CG is driven by the library's own preconditioner (stst_apply_prec,
   called through the C ABI on each oracle residual), so both sides run the same method with the same
   low-precision operator and x_k after k iterations can be compared directly. The two residuals differ
   only by the mat-vec's summation order (<= 1e-12 relative, test_apply_sys), which changes the FP32
   (or BF16) rounding of a small fraction of the preconditioner's inputs; the iterates then agree to
   ~1e-10 and the differences grow by at most ~30x per iteration (the CG sensitivity measured in the
   oracle pins): 1e-7 over six iterations.
2. A-orthogonality: x_{k+1} - x_k = alpha_k p_k, so consecutive steps of the library's solve must be
   A-orthogonal (the oracle's A), up to the mat-vec's 1e-12 relative difference: 1e-9 (the Polak-Ribiere
   beta used before leaves ~1e-7 with the FP32 and ~1e-5 with the BF16x3 preconditioner).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2311_18461_gb300 as S
from inputs import harmonic_potential, random_complex
from oracle import pcg as opcg
from tests._common import rel_err, oracle_disc, sample_potential, to_dev, to_np

pytestmark = pytest.mark.gpu

K = 6


def _problem(prec):
    n_el, p = [9, 11, 7], [2, 3, 2]
    V = harmonic_potential(2)
    prob = S.Problem(2, n_el, p, prec_mode=prec)
    prob.set_potential(sample_potential(prob, V), len(V))
    disc = oracle_disc(n_el, p, potential=V)
    assert prob.build_fd() == 0
    return prob, disc


def _gpu_iterates(prob, b):
    xs = [np.zeros(prob.n_dof, dtype=complex)]
    for k in range(1, K + 2):
        x, st, it, rr = prob.pcg(to_dev(b), tol=0.0, maxit=k)
        assert it == k
        xs.append(to_np(x))
    return xs


@pytest.mark.parametrize("prec", [S.STST_PREC_FP32, S.STST_PREC_BF16])
def test_flexible_cg_iterates_follow_the_oracle(prec):
    prob, disc = _problem(prec)
    b = random_complex(prob.n_dof, 71)
    xs = _gpu_iterates(prob, b)
    P = lambda r: to_np(prob.apply_prec(to_dev(r)))
    trace = []
    opcg.fcg(disc.apply, P, b, tol=0.0, maxit=K, trace=trace)
    for k in range(1, K + 1):
        assert rel_err(xs[k], trace[k - 1]["x"]) < 1e-7, k
    prob.close()


@pytest.mark.parametrize("prec", [S.STST_PREC_FP32, S.STST_PREC_BF16])
def test_flexible_cg_steps_are_A_orthogonal(prec):
    prob, disc = _problem(prec)
    b = random_complex(prob.n_dof, 72)
    xs = _gpu_iterates(prob, b)
    steps = [xs[k + 1] - xs[k] for k in range(K + 1)]
    an = lambda v: np.sqrt(np.vdot(v, disc.apply(v)).real)
    worst = max(abs(np.vdot(steps[k + 1], disc.apply(steps[k]))) / (an(steps[k + 1]) * an(steps[k]))
                for k in range(K))
    assert worst < 1e-9, worst
    prob.close()
