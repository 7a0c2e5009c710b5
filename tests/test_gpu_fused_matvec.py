"""The sum-factorised mat-vec with all levels in one launch (grid barriers between levels; opt-in) against
one launch per level: every output and every per-CTA partial sum is computed by the same thread arithmetic
over the same elements of the last level, so the two are bitwise equal, and so are the PCG solves built
on them (same iterations, same solutions). Handles in a batch keep one launch per level."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2311_18461_gb300 as S
from inputs import random_complex
from tests._common import to_dev, to_np

pytestmark = pytest.mark.gpu


def _apply(prob, x):
    y = torch.empty_like(x)
    S.stst_apply_sys(prob.h, x, y)
    return y.cpu().numpy()


def _kernels(prob, fn):
    S.stst_profile(prob.h, 1)
    fn()
    names = set(S.stst_profile_read(prob.h))
    S.stst_profile(prob.h, 0)
    return names


@pytest.mark.parametrize("n_el,p,prec", [([9, 11, 7], [2, 3, 2], S.STST_PREC_FP64),
                                         ([5, 6, 5, 7], [2, 2, 3, 2], S.STST_PREC_FP64),
                                         ([32, 32], 2, S.STST_PREC_FP64),
                                         ([12, 20, 16], 3, S.STST_PREC_FP32),
                                         ([64, 64, 64], 3, S.STST_PREC_FP32)])
def test_fused_mat_vec_is_bitwise_the_per_level_one(n_el, p, prec):
    out = {}
    try:
        for mode in (0, 1):
            S.stst_set_fused_matvec(mode)
            prob = S.Problem(len(n_el) - 1, n_el, p, prec_mode=prec)
            x = to_dev(random_complex(prob.n_dof, 3))
            names = _kernels(prob, lambda: _apply(prob, x))
            assert ("pass_fused_f64" in names) == (mode == 1), names
            y = _apply(prob, x)
            assert prob.build_fd() == 0
            xs, st, it, rr = prob.pcg(to_dev(random_complex(prob.n_dof, 4)), tol=1e-10, maxit=300)
            out[mode] = (y, to_np(xs), st, it, rr)
            prob.close()
    finally:
        S.stst_set_fused_matvec(0)
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert out[0][2:] == out[1][2:]


def test_opt_in_fuses_the_c2_mat_vec_and_batches_do_not():
    S.stst_set_fused_matvec(1)
    prob = S.Problem(2, [64, 64, 64], 3)
    x = to_dev(random_complex(prob.n_dof, 5))
    assert "pass_fused_f64" in _kernels(prob, lambda: _apply(prob, x))
    b = to_dev(random_complex(prob.n_dof, 6))
    sol = torch.zeros_like(b)
    prob.build_fd()
    batch = S.stst_batch_create([prob.h], [b], [sol])
    names = _kernels(prob, lambda: _apply(prob, x))
    assert "pass_fused_f64" not in names and "pass_f64" in names, names
    S.stst_batch_destroy(batch)
    prob.close()
    S.stst_set_fused_matvec(0)


def test_mode_argument_is_checked():
    for bad in (-1, 2):
        with pytest.raises(S.StstError):
            S.stst_set_fused_matvec(bad)
    S.stst_set_fused_matvec(0)
