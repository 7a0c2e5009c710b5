"""Planted mistakes in the oracle (on the CPU) must be caught by its pins.

Each test copies the oracle's state, plants one plausible error (a sign,
a dropped term, a transposed operand, a wrong power) and checks that the
corresponding pin fails by a wide margin. This shows the pins are sharp.
"""
import numpy as np

from oracle import direct, fd
from oracle.system import Discretization


def _mismatch(disc):
    A = disc.dense()
    Ad = direct.dense_A(disc)
    return np.abs(A - Ad).max() / np.abs(Ad).max()


def test_wrong_sign_of_W_is_caught():
    disc = Discretization([2, 3, 2], [2, 2], T=0.7, nu=1.3)
    assert _mismatch(disc) < 1e-12
    disc.Wsym = -disc.Wsym
    assert _mismatch(disc) > 1e-3


def test_dropped_cross_term_of_Bs_is_caught():
    disc = Discretization([2, 3, 2], [2, 2], T=0.7, nu=1.3)
    K2 = disc.sp[1]["K2"]
    all_terms = disc.terms()
    kept = [t for t in all_terms if not (np.allclose(t[1][1], K2) or np.allclose(t[1][1], K2.T))]
    assert len(kept) == len(all_terms) - 2
    disc.terms = lambda *a, **k: kept
    assert _mismatch(disc) > 1e-3


def test_transposed_eigenvectors_are_caught():
    disc = Discretization([4, 5, 6], [2, 3])
    P = fd.dense_P(disc)
    F = fd.FastDiagonalization(disc)
    r = np.random.default_rng(0).standard_normal(disc.N_dof) + 0j
    good = np.abs(F.apply(r) - np.linalg.solve(P, r)).max()
    F.U = [None] + [U.T for U in F.U[1:]]
    bad = np.abs(F.apply(r) - np.linalg.solve(P, r)).max()
    assert good < 1e-12 * np.abs(r).max() * 1e3 and bad > 1e3 * good


def test_lambda_instead_of_lambda_squared_is_caught():
    disc = Discretization([4, 5, 6], [2, 3])
    P = fd.dense_P(disc)
    F = fd.FastDiagonalization(disc)
    r = np.random.default_rng(1).standard_normal(disc.N_dof) + 0j
    ref = np.linalg.solve(P, r)
    F.H = lambda li, F=F: disc.Lt + disc.nu ** 2 * li * disc.Mt + disc.nu * li * disc.Wsym
    assert np.abs(F.apply(r) - ref).max() > 1e-3 * np.abs(ref).max()
