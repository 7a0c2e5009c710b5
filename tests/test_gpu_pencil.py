"""The pencil kernel (stst_set_pencil): Algorithm 1 steps 2-4 along the last spatial direction with the
banded time solves of step 3 in one kernel, one CTA per pencil or a cluster of two CTAs exchanging their
solved rows through distributed shared memory.

Against the FP64 oracle's Fast Diagonalization (tolerance 5e-5, as for every FP32 preconditioner: FP32 mode
products over n_l <= 65 terms and banded solves with kappa(H_i) ~ 1e2) and against the separate FP32
kernels (1e-5: the same FP32 sums, with the time solves' recurrences run by another kernel), for d = 1, 2,
3, time degrees 1 to 4 (the band widths of the solves), odd and even sizes; PCG with it reaches the
oracle's solution.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2311_18461_gb300 as S
from inputs import harmonic_potential, random_complex
from oracle import fd as ofd, pcg as opcg
from tests._common import rel_err, oracle_disc, sample_potential, to_dev, to_np

pytestmark = pytest.mark.gpu

SHAPES = [
    ([9, 12], [2, 3]),              # d = 1: one pencil (the whole problem)
    ([7, 9, 11], [3, 2, 3]),        # d = 2, n_2 = 12
    ([6, 8, 13], [1, 3, 2]),        # time degree 1, n_2 = 13 (odd: the two CTAs get 7 and 6 rows)
    ([11, 6, 10], [4, 2, 3]),       # time degree 4
    ([5, 6, 5, 7], [2, 2, 3, 2]),   # d = 3
]


def _apply(n_el, p, mode, potential=False):
    S.stst_set_pencil(mode)
    try:
        prob = S.Problem(len(n_el) - 1, n_el, p, prec_mode=S.STST_PREC_FP32)
        V = harmonic_potential(prob.d) if potential else None
        if V:
            prob.set_potential(sample_potential(prob, V), len(V))
        assert prob.build_fd() == 0
        used = S.stst_pencil_info(prob.h)
        r = random_complex(prob.n_dof, 51)
        z = to_np(prob.apply_prec(to_dev(r)))
    finally:
        S.stst_set_pencil(0)
    return prob, r, z, used


@pytest.mark.parametrize("n_el,p", SHAPES)
@pytest.mark.parametrize("ctas", [1, 2])
def test_pencil_matches_oracle_and_separate_kernels(n_el, p, ctas):
    prob, r, z, used = _apply(n_el, p, 1 + ctas)
    assert used == ctas
    disc = oracle_disc(n_el, p)
    assert rel_err(z, ofd.FastDiagonalization(disc).apply(r)) < 5e-5
    prob0, r0, z0, used0 = _apply(n_el, p, 1)
    assert used0 == 0 and np.array_equal(r, r0)
    assert rel_err(z, z0) < 1e-5
    prob.close()
    prob0.close()


def test_pencil_pcg_reaches_the_oracle_solution():
    """2D+t with the harmonic potential: the flexible CG with the pencil preconditioner to 1e-12."""
    n_el, p = [12, 14, 13], [3, 3, 3]
    S.stst_set_pencil(3)
    try:
        prob = S.Problem(2, n_el, p, prec_mode=S.STST_PREC_FP32)
        V = harmonic_potential(2)
        prob.set_potential(sample_potential(prob, V), len(V))
        assert prob.build_fd() == 0
        assert S.stst_pencil_info(prob.h) == 2
        b = random_complex(prob.n_dof, 52)
        x, st, it, rr = prob.pcg(to_dev(b), tol=1e-12, maxit=300)
    finally:
        S.stst_set_pencil(0)
    disc = oracle_disc(n_el, p, potential=V)
    xo, _, _, _ = opcg.pcg(disc.apply, ofd.FastDiagonalization(disc).apply, b, tol=1e-13, maxit=300)
    assert st == 0 and rel_err(to_np(x), xo) < 1e-8
    prob.close()


def test_pencil_not_used_where_it_does_not_apply():
    """FP64 and BF16 preconditioners, time degree above 4: the separate kernels run."""
    S.stst_set_pencil(3)
    try:
        for n_el, p, prec in [([4, 6, 7], 2, S.STST_PREC_FP64), ([4, 6, 7], 2, S.STST_PREC_BF16),
                              ([6, 6, 7], [5, 2, 2], S.STST_PREC_FP32)]:
            prob = S.Problem(len(n_el) - 1, n_el, p, prec_mode=prec)
            prob.build_fd()
            assert S.stst_pencil_info(prob.h) == 0, (n_el, p, prec)
            prob.close()
    finally:
        S.stst_set_pencil(0)
    for bad in (-1, 4):
        with pytest.raises(S.StstError):
            S.stst_set_pencil(bad)
