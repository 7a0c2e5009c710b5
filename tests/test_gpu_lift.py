"""General Dirichlet and initial data on the GPU (stst_rhs_lift, the lifting of Sec. 2.2 with data
taken from a function on the whole cylinder) against the oracle's full lifting, and the paper's
performance study (Sec. 6.2, Table 1) run through the CUDA path: P-hat-CG iterations on the
travelling wave.

Tolerances: the right-hand side and the lifting coefficients are FP64 sums of the same terms in a
different order (quadrature of S_V g_h against the Kronecker operator with exactly integrated
matrices): 1e-12 relative. Iteration counts: within one of the paper's (Table 1), as the oracle's are.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2311_18461_gb300 as S
from inputs import harmonic_potential, travelling_wave
from oracle import fd as ofd, pcg as opcg, rhs as orhs
from tests._common import rel_err, oracle_disc, sample_potential, sample_forcing, to_np

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _smooth_1d(t, x):
    return np.exp(1j * (2.0 * t + x)) * (1.0 + x ** 2) + 0.3 * t


def _forcing_1d(t, x):
    return np.cos(3.0 * x) * (1.0 + 1j * t)


def _smooth_2d(t, x1, x2):
    return np.exp(1j * (t + 2.0 * x1 - x2)) * (1.0 + x1 * x2) + 0.2j * t * x2


def _forcing_2d(t, x1, x2):
    return (x1 - 0.3) * np.exp(-1j * t) + 0.5 * x2 ** 2


def _lift_case(n_el, p, u_fn, f_fn, T=1.0, nu=1.0, V=None):
    d = len(n_el) - 1
    pl = [p] * (d + 1) if isinstance(p, int) else list(p)
    prob = S.Problem(d, n_el, pl, T=T, nu=nu)
    if V is not None:
        prob.set_potential(sample_potential(prob, V), len(V))
    disc = oracle_disc(n_el, pl, T=T, nu=nu, potential=V)
    b_gpu, xd_gpu = prob.rhs_lift(sample_forcing(prob, f_fn) if f_fn else None, sample_forcing(prob, u_fn),
                                  want_xd=True)
    b_ref, xd_ref = orhs.full_lifting(disc, u_fn, f_fn if f_fn else (lambda *a: 0.0 * a[0]))
    return prob, to_np(b_gpu), to_np(xd_gpu), b_ref, np.asarray(xd_ref).ravel()


@pytest.mark.parametrize("n_el,p,T,nu", [([5, 7], [2, 3], 1.0, 1.0), ([9, 4], [3, 2], 0.7, 1.3),
                                         ([4, 5, 6], [2, 3, 2], 1.0, 1.0), ([3, 6, 4], [3, 2, 3], 1.4, 0.8)])
def test_rhs_lift_matches_oracle(n_el, p, T, nu):
    d = len(n_el) - 1
    u_fn, f_fn = (_smooth_1d, _forcing_1d) if d == 1 else (_smooth_2d, _forcing_2d)
    prob, b, xd, b_ref, xd_ref = _lift_case(n_el, p, u_fn, f_fn, T=T, nu=nu)
    assert rel_err(xd, xd_ref) < 1e-12
    assert rel_err(b, b_ref) < 1e-12
    prob.close()


def _smooth_3d(t, x1, x2, x3):
    return np.exp(1j * (t + x1 - 2.0 * x3)) * (1.0 + x2 * x3) + 0.1 * t * x1


def _forcing_3d(t, x1, x2, x3):
    return (x1 + 1j * x2) * np.exp(-1j * t) + x3 ** 2


def test_rhs_lift_3d_matches_oracle():
    prob, b, xd, b_ref, xd_ref = _lift_case([3, 3, 4, 2], [2, 2, 3, 2], _smooth_3d, _forcing_3d, T=0.8, nu=1.1)
    assert rel_err(xd, xd_ref) < 1e-12
    assert rel_err(b, b_ref) < 1e-12
    prob.close()


def test_rhs_lift_with_potential_and_no_forcing():
    prob, b, xd, b_ref, xd_ref = _lift_case([5, 6, 4], [2, 2, 3], _smooth_2d, None, V=harmonic_potential(2))
    assert rel_err(xd, xd_ref) < 1e-12
    assert rel_err(b, b_ref) < 1e-12
    prob.close()


def test_rhs_lift_keeps_only_boundary_and_initial_coefficients():
    """g_h lives on the basis functions that do not vanish at t = 0 or on the spatial boundary."""
    n_el, p = [4, 5, 6], [2, 3, 2]
    prob, b, xd, _, _ = _lift_case(n_el, p, _smooth_2d, _forcing_2d)
    m = [n_el[l] + p[l] for l in range(3)]
    X = xd.reshape(m[2], m[1], m[0])
    assert np.all(X[1:-1, 1:-1, 1:] == 0)
    assert np.abs(X[:, :, 0]).min() > 0 and np.abs(X[0]).min() > 0 and np.abs(X[:, -1]).min() > 0
    prob.close()


def test_rhs_lift_rejects_ultraweak_and_missing_data():
    prob = S.Problem(1, [4, 5], 2, formulation=S.STST_FORM_UW)
    u = sample_forcing(prob, _smooth_1d)
    with pytest.raises(S.StstError):
        prob.rhs_lift(None, u)
    prob.close()
    prob = S.Problem(1, [4, 5], 2)
    with pytest.raises(S.StstError):
        S.stst_rhs_lift(prob.h, None, None, prob.vec(), None)
    prob.close()


def test_rhs_lift_solution_reproduces_a_discrete_function():
    """If u is itself in the spline space (here a polynomial of degree <= p in each variable), the
    lifted problem's discrete solution is u: u_h = u_bar + g_h matches u's projection everywhere."""
    n_el, p = [3, 4, 3], [2, 2, 2]
    u_fn = lambda t, x1, x2: (1 + 1j * t) * (1 + x1 - 0.5 * x2 ** 2) + 0 * t * x1 * x2
    f_fn = lambda t, x1, x2: 1j * (1j) * (1 + x1 - 0.5 * x2 ** 2) - (1 + 1j * t) * (-1.0) + 0 * t * x1 * x2
    prob = S.Problem(2, n_el, p)
    b, xd = prob.rhs_lift(sample_forcing(prob, f_fn), sample_forcing(prob, u_fn), want_xd=True)
    prob.build_fd()
    x, st, it, rr = prob.pcg(b, tol=1e-13, maxit=200)
    assert st == 0
    # full projection of u (no mask) from the oracle: the interior part must equal the solution
    disc = oracle_disc(n_el, p)
    _, xd_ref = orhs.full_lifting(disc, u_fn, f_fn)
    full = orhs.embed_solution(disc, to_np(x), XD=to_np(xd).reshape(np.asarray(xd_ref).shape))
    co = orhs.grid_coords(disc)
    G = u_fn(*co) * orhs.grid_weights(disc)
    for l in range(3):
        G = orhs.mode_product(G, orhs.tables(disc, l, full=True)[0].T, 2 if l == 0 else 2 - l)
    for l in range(3):
        G = orhs.mode_product(G, np.linalg.inv(disc.full[l]["M"]), 2 if l == 0 else 2 - l)
    assert rel_err(full, G) < 1e-9
    prob.close()


def _table1():
    rows = []
    for line in open(os.path.join(GOLDEN, "table1_iterations.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            p, n_el, it = (int(v) for v in line.split())
            rows.append((p, n_el, it))
    return rows


@pytest.mark.parametrize("p,n_el,iters", [r for r in _table1() if r[1] <= 32])
@pytest.mark.parametrize("prec", [S.STST_PREC_FP64, S.STST_PREC_FP32])
def test_table1_iterations_on_gpu(p, n_el, iters, prec):
    """Sec. 6.2 / Table 1: P-hat-CG from x0 = 0 to 1e-8 on the travelling wave takes the paper's
    iteration count (within one) with the FP64 preconditioner, and with the FP32 one in the FP64 solve."""
    u_fn, f_fn = travelling_wave()
    prob = S.Problem(2, [n_el] * 3, p, prec_mode=prec)
    b = prob.rhs_lift(sample_forcing(prob, f_fn), sample_forcing(prob, u_fn))
    prob.build_fd()
    x, st, it, rr = prob.pcg(b, tol=1e-8, maxit=200)
    assert st == 0 and rr <= 1e-8
    assert abs(it - iters) <= 1, (it, iters)
    prob.close()


def test_table1_smallest_case_matches_oracle_solve():
    """p = 3, n_el = 8: the GPU P-hat-CG solution of the travelling wave equals the oracle's."""
    u_fn, f_fn = travelling_wave()
    prob = S.Problem(2, [8, 8, 8], 3)
    b = prob.rhs_lift(sample_forcing(prob, f_fn), sample_forcing(prob, u_fn))
    prob.build_fd()
    x, st, it, rr = prob.pcg(b, tol=1e-12, maxit=200)
    disc = oracle_disc([8, 8, 8], 3)
    b_ref, _ = orhs.full_lifting(disc, u_fn, f_fn)
    x_ref, it_ref, _, _ = opcg.pcg(disc.apply, ofd.FastDiagonalization(disc).apply, b_ref, tol=1e-12, maxit=200)
    assert rel_err(to_np(b), b_ref) < 1e-12
    assert rel_err(to_np(x), x_ref) < 1e-9
    prob.close()
