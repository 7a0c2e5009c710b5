"""The system on a mapped domain (Sec. 3.2, Eq. syst_mat with the spatial matrices of Eq. space_mat over
Omega = F((0,1)^d)) on the GPU against the oracle (`oracle.geometry`, pinned in
tests/test_oracle_geometry_pins.py).

The library assembles M_s, L_s, B_s by the same quadrature as the oracle but sums in another order, so the
mat-vec agrees to rounding: 1e-12 relative (the parametric mat-vec's bound, test_apply_sys). PCG keeps
the parametric P-hat (the paper's fast solver is for F = id only): the FP64-preconditioned solution is held
to 1e-10 of the oracle's sparse direct solution, the FP32-preconditioned one (flexible CG) to 1e-8.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

torch = pytest.importorskip("torch")

import paper_2311_18461_gb300 as S
from inputs import random_complex
from inputs.geometry import Affine, Identity, Perturbed, QuarterAnnulus, geometry_at
from oracle import fd as ofd, geometry as ogeo, pcg as opcg
from oracle.system import Discretization
from tests._common import rel_err, to_dev, to_np

pytestmark = pytest.mark.gpu


def _set_map(prob, gmap):
    grids = [prob.quad_points(l).cpu().numpy() for l in range(1, prob.d + 1)]
    J, H = geometry_at(gmap, grids)
    jac = torch.tensor(np.ascontiguousarray(J), dtype=torch.float64, device="cuda")
    hess = torch.tensor(np.ascontiguousarray(H), dtype=torch.float64, device="cuda")
    return prob.set_geometry(jac, hess)


def _apply(prob, v):
    x = to_dev(v)
    y = torch.empty_like(x)
    S.stst_apply_sys(prob.h, x, y)
    return to_np(y)


CASES = [
    (QuarterAnnulus(1.0, 2.0), [5, 6, 7], [2, 3, 2]),
    (QuarterAnnulus(0.5, 1.5), [4, 9, 5], [3, 2, 4]),
    (Perturbed(0.1, 1), [6, 9], [2, 3]),
    (Perturbed(0.08, 2), [4, 7, 6], [2, 2, 3]),
    (Perturbed(0.05, 3), [3, 4, 5, 3], [2, 2, 3, 2]),
]


@pytest.mark.parametrize("gmap,n_el,p", CASES)
def test_mapped_apply_sys_matches_oracle(gmap, n_el, p):
    prob = S.Problem(len(n_el) - 1, n_el, p)
    _set_map(prob, gmap)
    assert S.stst_geometry_info(prob.h)[0] == 1
    g = ogeo.GeoDiscretization(n_el, p, gmap)
    for seed in (1, 2):
        x = random_complex(prob.n_dof, seed)
        assert rel_err(_apply(prob, x), g.apply(x)) < 1e-12
    prob.close()


@pytest.mark.parametrize("n_el,p", [([4, 7], [2, 3]), ([3, 5, 4], [2, 3, 2]), ([2, 3, 4, 3], [1, 2, 2, 2])])
def test_identity_map_reproduces_the_parametric_operator(n_el, p):
    d = len(n_el) - 1
    prob = S.Problem(d, n_el, p)
    x = random_complex(prob.n_dof, 5)
    y0 = _apply(prob, x)
    _set_map(prob, Identity(d))
    y1 = _apply(prob, x)
    assert rel_err(y1, y0) < 1e-12
    S.stst_set_geometry(prob.h, None, None)  # removed: the parametric operator again, unchanged
    assert S.stst_geometry_info(prob.h) == (0, 0)
    assert np.array_equal(_apply(prob, x), y0)
    prob.close()


@pytest.mark.parametrize("prec,tol", [(S.STST_PREC_FP64, 1e-10), (S.STST_PREC_FP32, 1e-8)])
@pytest.mark.parametrize("gmap,n_el,p", [(QuarterAnnulus(1.0, 2.0), [6, 7, 6], [2, 3, 2]),
                                         (Perturbed(0.05, 3), [3, 4, 3, 4], [2, 2, 2, 2])])
def test_pcg_on_the_mapped_domain_reaches_the_direct_solution(gmap, n_el, p, prec, tol):
    """The scaled P-hat (eigenvalue scales from the geometry, as the oracle's prec_scales) preconditions PCG
    to the sparse direct solution; with the FP64 preconditioner the iteration count is the oracle's."""
    prob = S.Problem(len(n_el) - 1, n_el, p, prec_mode=prec)
    _set_map(prob, gmap)
    assert prob.build_fd() == 0
    g = ogeo.GeoDiscretization(n_el, p, gmap)
    disc = Discretization(n_el, p)
    sc = ogeo.prec_scales(gmap, disc)
    assert np.allclose(S.stst_geometry_info(prob.h, with_scales=True)[2][:len(sc)], sc, rtol=1e-12, atol=0)
    b = random_complex(prob.n_dof, 7)
    x, st, it, rr = prob.pcg(to_dev(b), tol=1e-12, maxit=500)
    assert st == 0, (st, it, rr)
    xd = spla.spsolve(g.sparse(), b)
    assert rel_err(to_np(x), xd) < tol
    if prec == S.STST_PREC_FP64:
        _, ito, _, _ = opcg.pcg(g.apply, ofd.FastDiagonalization(disc, scales=sc).apply, b, tol=1e-12, maxit=500)
        assert abs(it - ito) <= 1, (it, ito)
    prob.close()


def test_affine_box_takes_the_parametric_iteration_count():
    """On a box with sides 1 x pi/2 the scaled P-hat is the box's own preconditioner (up to a constant):
    PCG takes the unit box's iterations, where the unscaled one needs several times more."""
    n_el, p = [16, 16, 16], 3
    sides = [1.0, 0.5 * np.pi]
    its = {}
    for mapped in (False, True):
        prob = S.Problem(2, n_el, p)
        if mapped:
            _set_map(prob, Affine(sides))
        assert prob.build_fd() == 0
        bb = random_complex(prob.n_dof, 9)
        _, st, its[mapped], _ = prob.pcg(to_dev(bb), tol=1e-8, maxit=2000)
        assert st == 0
        prob.close()
    assert abs(its[True] - its[False]) <= 2, its


def test_geometry_states_and_errors():
    n_el, p = [4, 5, 6], [2, 2, 2]
    prob = S.Problem(2, n_el, p)
    # a map that folds: det J changes sign inside the box
    grids = [prob.quad_points(l).cpu().numpy() for l in (1, 2)]
    J, H = geometry_at(Perturbed(0.5, 2), grids)
    det = np.linalg.det(J)
    assert det.min() < 0 < det.max()
    with pytest.raises(S.StstError) as e:
        prob.set_geometry(torch.tensor(J, device="cuda"), torch.tensor(H, device="cuda"))
    assert e.value.status == S.STST_ERR_ARG
    assert S.stst_geometry_info(prob.h)[0] == 0
    with pytest.raises(S.StstError):
        prob.set_geometry(torch.tensor(J, device="cuda"), None)
    # a mapped handle refuses a potential and the parametric load vectors
    _set_map(prob, QuarterAnnulus())
    V = torch.ones(sum(len(g) for g in grids), dtype=torch.float64, device="cuda")
    with pytest.raises(S.StstError) as e:
        prob.set_potential(V, 1)
    assert e.value.status == S.STST_ERR_STATE
    nq = int(np.prod([len(prob.quad_points(l)) for l in range(3)]))
    f = torch.zeros(nq, dtype=torch.complex128, device="cuda")
    with pytest.raises(S.StstError) as e:
        prob.rhs(f, None)
    assert e.value.status == S.STST_ERR_STATE
    # nor does it join a batch (refused before any device work)
    bb = torch.zeros(prob.n_dof, dtype=torch.complex128, device="cuda")
    xx = torch.zeros(prob.n_dof, dtype=torch.complex128, device="cuda")
    with pytest.raises(S.StstError) as e:
        S.stst_batch_create([prob.h], [bb], [xx])
    assert e.value.status == S.STST_ERR_STATE
    prob.close()
    # a handle with a potential, or the ultraweak formulation, refuses a geometry
    prob = S.Problem(2, n_el, p)
    prob.set_potential(V, 1)
    with pytest.raises(S.StstError) as e:
        _set_map(prob, QuarterAnnulus())
    assert e.value.status == S.STST_ERR_STATE
    prob.close()
    prob = S.Problem(2, n_el, p, formulation=S.STST_FORM_UW)
    with pytest.raises(S.StstError) as e:
        _set_map(prob, QuarterAnnulus())
    assert e.value.status == S.STST_ERR_STATE
    prob.close()


def test_full_size_annulus_mat_vec_and_solve():
    """2D+t, p = 3, 64^2 x 64 elements (278,850 unknowns, the c2 mesh) on the quarter annulus: the mat-vec
    against the oracle's sparse assembly, and the FP32-preconditioned solve to relative residual 1e-8 (282
    iterations with the scaled P-hat, bounded here by 400; the unscaled one did not converge in 3,000) with
    its true residual checked by the oracle's operator."""
    n_el, p = [64, 64, 64], 3
    prob = S.Problem(2, n_el, p, prec_mode=S.STST_PREC_FP32)
    _set_map(prob, QuarterAnnulus(1.0, 2.0))
    g = ogeo.GeoDiscretization(n_el, p, QuarterAnnulus(1.0, 2.0))
    x = random_complex(prob.n_dof, 11)
    assert rel_err(_apply(prob, x), g.apply(x)) < 1e-12
    assert prob.build_fd() == 0
    b = random_complex(prob.n_dof, 12)
    xs, st, it, rr = prob.pcg(to_dev(b), tol=1e-8, maxit=1000)
    assert st == 0 and it < 400, (st, it)
    true_res = np.linalg.norm(b - g.apply(to_np(xs))) / np.linalg.norm(b)
    assert true_res < 2e-8, true_res
    prob.close()
