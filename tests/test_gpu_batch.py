"""Batched solves: one graph launch solves many heterogeneous problems; each branch reproduces the
single-problem solve (same kernels in the same order) and the oracle's solution."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2311_18461_gb300 as S
from inputs import random_smooth_potential, wavepacket_factors, wavepacket_params, random_complex
from oracle import fd as ofd, pcg as opcg
from tests._common import rel_err, oracle_disc, sample_potential, sample_initial, to_dev, to_np

pytestmark = pytest.mark.gpu

SPECS = [([9, 7, 8], [2, 2, 2], S.STST_PREC_FP32), ([12, 10, 9], [3, 3, 3], S.STST_PREC_FP64),
         ([6, 11, 5], [4, 4, 4], S.STST_PREC_FP32), ([10, 8, 8], [2, 3, 3], S.STST_PREC_BF16),
         ([16, 6], [3, 3], S.STST_PREC_FP32)]


def _instances(seed0):
    out = []
    for k, (n_el, p, prec) in enumerate(SPECS):
        d = len(n_el) - 1
        rng = np.random.default_rng(seed0 + k)
        V = random_smooth_potential(rng, d)
        prob = S.Problem(d, n_el, p, prec_mode=prec)
        prob.set_potential(sample_potential(prob, V), len(V))
        b = prob.rhs(None, sample_initial(prob, wavepacket_factors(wavepacket_params(rng, d))))
        out.append((prob, V, b, n_el, p))
    return out


def test_batch_matches_single_solves_and_oracle():
    inst = _instances(100)
    xs = [prob.vec() for prob, *_ in inst]
    batch = S.stst_batch_create([prob.h for prob, *_ in inst], [b for _, _, b, _, _ in inst], xs)
    try:
        for rep in range(2):  # the graph is reusable: a second launch redoes setup and solve
            for x in xs:
                x.zero_()
            status, iters, relres, sts = S.stst_batch_solve(batch, len(inst), 1e-10, 300)
            assert status == 0 and all(s == 0 for s in sts)
            assert all(r <= 1e-10 for r in relres)
            for (prob, V, b, n_el, p), x, it in zip(inst, xs, iters):
                prob.build_fd()
                x1, st1, it1, rr1 = prob.pcg(b, tol=1e-10, maxit=300)
                assert it1 == it
                assert rel_err(to_np(x), to_np(x1)) < 1e-12
    finally:
        S.stst_batch_destroy(batch)
    prob, V, b, n_el, p = inst[1]
    disc = oracle_disc(n_el, p, potential=V)
    xo, _, _, _ = opcg.pcg(disc.apply, ofd.FastDiagonalization(disc).apply, to_np(b), tol=1e-13, maxit=300)
    assert rel_err(to_np(xs[1]), xo) < 1e-8


def test_batch_reports_per_problem_outcomes():
    inst = _instances(200)[:3]
    xs = [prob.vec() for prob, *_ in inst]
    rhs = [b.clone() for _, _, b, _, _ in inst]
    rhs[1][3] = complex(float("nan"), 0.0)
    batch = S.stst_batch_create([prob.h for prob, *_ in inst], rhs, xs)
    try:
        status, iters, relres, sts = S.stst_batch_solve(batch, len(inst), 1e-10, 300)
        assert sts[0] == 0 and sts[2] == 0 and sts[1] in (1, 2)
        assert status == sts[1]
        status, iters, relres, sts = S.stst_batch_solve(batch, len(inst), 0.0, 2)
        assert sts[0] == 1 and sts[2] == 1 and iters[0] == 2 and iters[2] == 2
    finally:
        S.stst_batch_destroy(batch)
    with pytest.raises(S.StstError):
        S.stst_batch_create([inst[0][0].h, inst[0][0].h], rhs[:2], xs[:2])


def test_batch_c4_mesh_range_against_the_oracle():
    """The ends of the batched workload's range (n_el in {16..96}^2 x {16..96}, p in {2, 3, 4}, a random
    separable potential and a wavepacket per instance): a 96^2 x 96, p = 4 instance (950,796 unknowns) with
    the FP32 preconditioner and 16^2 x 16 instances with the BF16x3 and FP32 ones, solved in one launch to
    relative residual 1e-11; every solution within 1e-8 of the oracle's (PCG with the exact P-hat to 1e-13
    on the same right-hand side)."""
    specs = [([96, 96, 96], 4, S.STST_PREC_FP32), ([16, 16, 16], 2, S.STST_PREC_BF16),
             ([16, 16, 16], 3, S.STST_PREC_FP32)]
    inst = []
    for k, (n_el, p, prec) in enumerate(specs):
        rng = np.random.default_rng(4 + k)
        V = random_smooth_potential(rng, 2)
        prob = S.Problem(2, n_el, p, prec_mode=prec)
        prob.set_potential(sample_potential(prob, V), len(V))
        b = prob.rhs(None, sample_initial(prob, wavepacket_factors(wavepacket_params(rng, 2))))
        inst.append((prob, V, b, n_el, p))
    xs = [prob.vec() for prob, *_ in inst]
    batch = S.stst_batch_create([prob.h for prob, *_ in inst], [b for _, _, b, _, _ in inst], xs)
    try:
        status, iters, relres, sts = S.stst_batch_solve(batch, len(inst), 1e-11, 400)
    finally:
        S.stst_batch_destroy(batch)
    assert status == 0 and all(s == 0 for s in sts) and all(r <= 1e-11 for r in relres)
    for (prob, V, b, n_el, p), x in zip(inst, xs):
        disc = oracle_disc(n_el, p, potential=V)
        bn = to_np(b)
        xo, _, _, _ = opcg.pcg(disc.apply, ofd.FastDiagonalization(disc).apply, bn, tol=1e-13, maxit=400)
        assert rel_err(to_np(x), xo) < 1e-8, (n_el, p)
        prob.close()
