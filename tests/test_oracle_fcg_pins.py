"""Pins of the oracle's flexible CG (`oracle.pcg.fcg`, Notay's flexible conjugate gradients with one kept
direction; the solver's form when the preconditioner is applied in low precision).

What the method fixes whatever the preconditioner does at each iteration:
  * consecutive directions are A-orthogonal: <p_{k+1}, A p_k> = 0;
  * every step is the exact line search along its direction: <r_{k+1}, p_k> = 0;
  * hence the A-norm of the error never grows;
  * with a fixed Hermitian positive definite preconditioner the iterates are plain PCG's (Sec. 5.3).
The preconditioners that vary are P-hat^{-1} (Algorithm 1) with a fresh random diagonal scaling at every
iteration: a Hermitian one, D_k P-hat^{-1} D_k with D_k in [0.8, 1.25], and a non-Hermitian one,
P-hat^{-1} diag(c_k) with complex c_k near 1 (it makes <r, z> complex, so the complex alpha is exercised).
Planted mistakes (the real part of beta only, a conjugated beta, the Polak-Ribiere beta, a real or
conjugated alpha) fail these pins by orders of magnitude.
"""
import numpy as np
import pytest

from oracle import fd, pcg
from oracle.system import Discretization


def _bump(d):
    return [[(lambda x: 10.0 * np.exp(-(x - 0.5) ** 2 / 0.05)) for _ in range(d)]]


@pytest.fixture(scope="module")
def system():
    disc = Discretization([4, 5, 4], [2, 3], potential=_bump(2))
    A = disc.dense()
    F = fd.FastDiagonalization(disc)
    rng = np.random.default_rng(11)
    f = rng.standard_normal(disc.N_dof) + 1j * rng.standard_normal(disc.N_dof)
    return disc, A, F, f


def _varying(F, n, hermitian, seed):
    """B_k(r): P-hat^{-1} with a new random diagonal scaling at every iteration k."""
    rng = np.random.default_rng(seed)
    scales = {}

    def B(r, k):
        if k not in scales:
            if hermitian:
                scales[k] = rng.uniform(0.8, 1.25, n)
            else:
                scales[k] = rng.uniform(0.8, 1.25, n) * np.exp(0.3j * rng.uniform(-1, 1, n))
        c = scales[k]
        return c * F.apply(c * r) if hermitian else F.apply(c * r)
    return B


def _anorm(A, v):
    return np.sqrt(np.vdot(v, A @ v).real)


def _check(A, f, trace, tol=1e-12):
    """Largest relative violation of A-orthogonality and of the line search, and whether the A-norm of the
    error ever grew."""
    xs = np.linalg.solve(A, f)
    conj = 0.0
    line = 0.0
    e_prev = _anorm(A, xs)
    grew = False
    for k, t in enumerate(trace):
        r, p, q = t["r"], t["p"], t["q"]
        r_before = f if k == 0 else trace[k - 1]["r"]
        line = max(line, abs(np.vdot(p, r)) / abs(np.vdot(p, r_before)))
        e = _anorm(A, xs - t["x"])
        grew = grew or e > e_prev * (1 + 1e-12)
        e_prev = e
        if k + 1 < len(trace):
            pn = trace[k + 1]["p"]
            conj = max(conj, abs(np.vdot(q, pn)) / (_anorm(A, pn) * _anorm(A, p)))
    return conj, line, grew


@pytest.mark.parametrize("hermitian", [True, False])
def test_fcg_directions_A_orthogonal_and_exact_line_searches_under_a_varying_preconditioner(system, hermitian):
    disc, A, F, f = system
    trace = []
    B = _varying(F, disc.N_dof, hermitian, 5)
    x, it, rr, _ = pcg.fcg(lambda v: A @ v, B, f, tol=1e-13, maxit=200, trace=trace, with_iteration=True)
    conj, line, grew = _check(A, f, trace)
    assert len(trace) >= 8
    assert conj < 1e-12, conj
    assert line < 1e-12, line
    assert not grew
    xs = np.linalg.solve(A, f)
    assert np.abs(x - xs).max() <= 1e-10 * np.abs(xs).max()


def test_fcg_is_plain_pcg_for_a_fixed_preconditioner(system):
    disc, A, F, f = system
    trace = []
    xf, itf, _, hf = pcg.fcg(lambda v: A @ v, F.apply, f, tol=1e-12, maxit=200, trace=trace)
    xp, itp, _, hp = pcg.pcg(lambda v: A @ v, F.apply, f, tol=1e-12, maxit=200)
    assert abs(itf - itp) <= 1
    # Equal in exact arithmetic. In floating point the two recurrences differ by rounding, and CG
    # amplifies such differences geometrically (here by ~30x per iteration after the tenth, where the
    # residual histories part at the 1e-4 level and then meet again): the first eight residuals agree to
    # 1e-12, the solutions to 1e-11.
    hf, hp = np.array(hf[:9]), np.array(hp[:9])
    assert np.max(np.abs(hf - hp) / hp) < 1e-12
    assert np.abs(xf - xp).max() <= 1e-11 * np.abs(xp).max()
    # fixed Hermitian B: <r, z> is real and positive, so alpha is real up to rounding
    assert max(abs(t["alpha"].imag) / abs(t["alpha"]) for t in trace) < 1e-12


def test_sigma_recurrence_of_the_device_form(system):
    """The device computes alpha's numerator <r_{k+1}, p_{k+1}> as <r_{k+1}, z_{k+1}> + conj(beta_k)
    <r_{k+1}, p_k> (both read from partial sums of kernels it runs anyway): an identity for any complex
    beta, whose second term is the rounding-level residue of the line search."""
    disc, A, F, f = system
    B = _varying(F, disc.N_dof, False, 9)
    trace = []
    pcg.fcg(lambda v: A @ v, B, f, tol=1e-10, maxit=6, trace=trace, with_iteration=True)
    worst = 0.0
    for k in range(len(trace) - 1):
        r, p, beta = trace[k]["r"], trace[k]["p"], trace[k]["beta"]
        pn = trace[k + 1]["p"]
        z = pn - beta * p
        exact = pcg.inner(r, pn)
        dev = pcg.inner(r, z) + np.conj(beta) * pcg.inner(r, p)
        worst = max(worst, abs(dev - exact) / abs(exact))
        assert abs(beta.imag) > 1e-3 * abs(beta)   # the non-Hermitian B makes beta complex
    assert worst < 1e-13


def _mutated(monkeypatch, which):
    if which == "beta_real":
        monkeypatch.setattr(pcg, "fcg_beta", lambda z, p, q: -pcg.inner(z, q).real / pcg.inner(p, q).real)
    elif which == "beta_conj":
        monkeypatch.setattr(pcg, "fcg_beta", lambda z, p, q: -np.conj(pcg.inner(z, q)) / pcg.inner(p, q).real)
    elif which == "alpha_real":
        monkeypatch.setattr(pcg, "fcg_alpha", lambda r, p, q: pcg.inner(r, p).real / pcg.inner(p, q).real)
    elif which == "alpha_conj":
        monkeypatch.setattr(pcg, "fcg_alpha", lambda r, p, q: pcg.inner(p, r) / pcg.inner(p, q).real)


@pytest.mark.parametrize("which,pin", [("beta_real", "conj"), ("beta_conj", "conj"), ("alpha_real", "line"),
                                       ("alpha_conj", "line")])
def test_planted_mistakes_in_fcg_fail_its_pins(system, monkeypatch, which, pin):
    disc, A, F, f = system
    _mutated(monkeypatch, which)
    trace = []
    pcg.fcg(lambda v: A @ v, _varying(F, disc.N_dof, False, 5), f, tol=1e-13, maxit=30, trace=trace,
             with_iteration=True)
    conj, line, grew = _check(A, f, trace)
    assert (conj if pin == "conj" else line) > 1e-6


def test_polak_ribiere_beta_is_not_A_orthogonal(system):
    """The real Polak-Ribiere form beta = Re <r_{k+1}, z_{k+1} - z_k> / <r_k, z_k> (a common flexible
    choice) leaves consecutive directions A-orthogonal only for a fixed preconditioner."""
    disc, A, F, f = system
    B = _varying(F, disc.N_dof, False, 5)
    r = f.copy()
    z = B(r, 0)
    p = z.copy()
    rho = np.vdot(r, z).real
    x = np.zeros_like(f)
    trace = []
    for k in range(12):
        q = A @ p
        alpha = rho / np.vdot(p, q).real
        x = x + alpha * p
        r = r - alpha * q
        trace.append({"x": x.copy(), "r": r.copy(), "p": p.copy(), "q": q})
        zn = B(r, k + 1)
        rho_n = np.vdot(r, zn).real
        beta = (rho_n - np.vdot(r, z).real) / rho
        p = zn + beta * p
        z, rho = zn, rho_n
    conj, _, _ = _check(A, f, trace)
    assert conj > 1e-6
