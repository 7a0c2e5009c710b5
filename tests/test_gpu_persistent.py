"""The persistent PCG (stst_persistent_solve: a whole solve per thread-block cluster, many problems in one
launch) against the oracle's PCG with the exact P-hat (Sec. 5.3, Sec. 6) and against the library's graph
solve. Both GPU forms run the same plain CG with the FP64 preconditioner; their sums run in different
orders, so the iteration counts agree within one and the solutions to rounding amplified by the solve:
1e-10 relative (the FP64 path's bound against the oracle)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2311_18461_gb300 as S
from inputs import harmonic_potential, random_complex
from oracle import fd as ofd, pcg as opcg
from tests._common import oracle_disc, rel_err, sample_potential, to_dev, to_np

pytestmark = pytest.mark.gpu


def _problem(n_el, p, V=None, formulation=S.STST_FORM_LS, prec=S.STST_PREC_FP64):
    prob = S.Problem(len(n_el) - 1, n_el, p, prec_mode=prec, formulation=formulation)
    if V is not None:
        prob.set_potential(sample_potential(prob, V), len(V))
    assert prob.build_fd() == 0
    return prob


CASES = [([8, 8], [2, 2], None), ([9, 11, 7], [2, 3, 2], "harmonic"), ([8, 8, 8], 3, None),
         ([5, 6, 5, 7], [2, 2, 3, 2], None), ([6, 5, 4, 5], [4, 2, 3, 2], "harmonic")]


@pytest.mark.parametrize("n_el,p,pot", CASES)
def test_persistent_solve_matches_oracle_and_graph_solve(n_el, p, pot):
    d = len(n_el) - 1
    V = harmonic_potential(d) if pot else None
    prob = _problem(n_el, p, V)
    b = random_complex(prob.n_dof, 21)
    x = torch.zeros(prob.n_dof, dtype=torch.complex128, device="cuda")
    st, its, rrs, sts = S.stst_persistent_solve([prob.h], [to_dev(b)], [x], tol=1e-12, maxit=300)
    assert st == 0 and sts == [0]
    disc = oracle_disc(n_el, p, potential=V)
    xo, ito, rro, _ = opcg.pcg(disc.apply, ofd.FastDiagonalization(disc).apply, b, tol=1e-12, maxit=300)
    assert abs(its[0] - ito) <= 1, (its, ito)
    assert rel_err(to_np(x), xo) < 1e-10
    xg, stg, itg, rrg = prob.pcg(to_dev(b), tol=1e-12, maxit=300)
    assert abs(itg - its[0]) <= 1
    assert rel_err(to_np(x), to_np(xg)) < 1e-10
    prob.close()


def test_many_problems_of_different_sizes_in_one_launch():
    shapes = [([8, 8, 8], 2), ([12, 9, 10], 3), ([6, 7], 4), ([5, 4, 6, 5], 2), ([16, 16, 16], 3)]
    probs = [_problem(n, p) for n, p in shapes]
    bs = [to_dev(random_complex(pr.n_dof, 30 + i)) for i, pr in enumerate(probs)]
    xs = [torch.zeros_like(b) for b in bs]
    st, its, rrs, sts = S.stst_persistent_solve([pr.h for pr in probs], bs, xs, tol=1e-10, maxit=300,
                                                cluster_ctas=4)
    assert st == 0 and all(s == 0 for s in sts)
    for pr, b, x, it, rr in zip(probs, bs, xs, its, rrs):
        assert rr <= 1e-10
        xg, stg, itg, rrg = pr.pcg(b, tol=1e-10, maxit=300)
        assert abs(itg - it) <= 1
        assert rel_err(to_np(x), to_np(xg)) < 1e-8
        pr.close()


@pytest.mark.parametrize("C", [1, 2, 8, 16])
def test_cluster_sizes_agree(C):
    prob = _problem([10, 12, 12], 3)
    b = to_dev(random_complex(prob.n_dof, 40))
    x = torch.zeros_like(b)
    st, its, rrs, _ = S.stst_persistent_solve([prob.h], [b], [x], tol=1e-10, maxit=300, cluster_ctas=C)
    xg, stg, itg, rrg = prob.pcg(b, tol=1e-10, maxit=300)
    assert st == 0 and abs(its[0] - itg) <= 1
    assert rel_err(to_np(x), to_np(xg)) < 1e-8
    prob.close()


def test_ultraweak_and_edge_cases():
    prob = _problem([7, 8, 6], [3, 2, 2], formulation=S.STST_FORM_UW)
    disc = oracle_disc([7, 8, 6], [3, 2, 2], formulation="uw")
    b = random_complex(prob.n_dof, 50)
    x = torch.zeros(prob.n_dof, dtype=torch.complex128, device="cuda")
    st, its, _, _ = S.stst_persistent_solve([prob.h], [to_dev(b)], [x], tol=1e-12, maxit=300)
    xo, ito, _, _ = opcg.pcg(disc.apply, ofd.FastDiagonalization(disc).apply, b, tol=1e-12, maxit=300)
    assert st == 0 and abs(its[0] - ito) <= 1 and rel_err(to_np(x), xo) < 1e-10
    # a zero right-hand side: x = 0 after no iteration; maxit = 0: not converged, x = 0
    z = torch.zeros_like(x)
    x.fill_(1.0)
    st, its, rrs, _ = S.stst_persistent_solve([prob.h], [z], [x], tol=1e-10, maxit=300)
    assert st == 0 and its == [0] and rrs == [0.0] and bool((x == 0).all())
    st, its, rrs, sts = S.stst_persistent_solve([prob.h], [to_dev(b)], [x], tol=1e-10, maxit=0)
    assert st == S.STST_NOT_CONVERGED and its == [0] and sts == [S.STST_NOT_CONVERGED] and rrs == [1.0]
    prob.close()


def test_refused_handles_and_arguments():
    p64 = _problem([6, 6, 6], 2)
    p32 = _problem([6, 6, 6], 2, prec=S.STST_PREC_FP32)
    b = to_dev(random_complex(p64.n_dof, 60))
    x = torch.zeros_like(b)
    for hs, kw, code in [([p32.h], {}, S.STST_ERR_STATE), ([p64.h, p64.h], {}, S.STST_ERR_ARG),
                         ([p64.h], {"cluster_ctas": 3}, S.STST_ERR_ARG), ([p64.h], {"maxit": -1}, S.STST_ERR_ARG)]:
        with pytest.raises(S.StstError) as e:
            S.stst_persistent_solve(hs, [b] * len(hs), [x] * len(hs), **kw)
        assert e.value.status == code
    fresh = S.Problem(2, [6, 6, 6], 2)  # not built
    with pytest.raises(S.StstError) as e:
        S.stst_persistent_solve([fresh.h], [b], [x])
    assert e.value.status == S.STST_ERR_STATE
    for pr in (p64, p32, fresh):
        pr.close()
