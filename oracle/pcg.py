"""Preconditioned conjugate gradients for the HPD least-squares system (Sec. 5.3, Sec. 6).

Test infrastructure: part of the CPU oracle, see `oracle/__init__.py`.

The paper solves A u = f by CG preconditioned with P-hat, tolerance 1e-8,
zero initial guess, at most 200 iterations. A is Hermitian positive definite
(the paper says "symmetric"; read Hermitian), inner products are
<a, b> = b^H a. Stopping test: ||f - A x_k||_2 <= tol ||f||_2 on the
recursively updated residual (the paper does not name its norm; for x_0 = 0
this equals ||r_k|| / ||r_0||).

`pcg(..., flexible=False)` is the paper's method: plain PCG with a fixed
Hermitian positive definite preconditioner.

`fcg` (and `pcg(..., flexible=True)`) is the flexible conjugate gradient
method of Notay (SIAM J. Sci. Comput. 22 (2000) 1444-1460) with one kept
direction, written for a complex Hermitian A. It is not in the paper: it is
the form the solver uses when the preconditioner is applied in low precision,
which makes it a slightly different operator at every iteration. Each new
direction is the preconditioned residual made A-orthogonal to the previous
direction, and each step is the exact line search along its direction:
    q_k = A p_k,  alpha_k = <r_k, p_k> / <p_k, q_k>,
    x_{k+1} = x_k + alpha_k p_k,  r_{k+1} = r_k - alpha_k q_k,
    z_{k+1} = B_{k+1}(r_{k+1}),
    beta_k = -<z_{k+1}, q_k> / <p_k, q_k>,  p_{k+1} = z_{k+1} + beta_k p_k.
alpha and beta are complex. Whatever the B_k are, consecutive directions are
A-orthogonal, <r_{k+1}, p_k> = 0 and the A-norm of the error never grows;
for a fixed Hermitian positive definite B the iterates are those of `pcg`.
"""
import numpy as np


def pcg(apply_A, apply_P, f, x0=None, tol=1e-8, maxit=200, flexible=False):
    """Returns (x, iterations, relative residual, history of relative residuals)."""
    if flexible:
        return fcg(apply_A, apply_P, f, x0=x0, tol=tol, maxit=maxit)
    f = np.asarray(f, dtype=complex)
    x = np.zeros_like(f) if x0 is None else np.array(x0, dtype=complex)
    nf = np.linalg.norm(f)
    if nf == 0.0:
        return np.zeros_like(f), 0, 0.0, [0.0]
    r = f - apply_A(x) if x0 is not None else f.copy()
    hist = [np.linalg.norm(r) / nf]
    if hist[-1] <= tol:
        return x, 0, hist[-1], hist
    z = apply_P(r)
    p = z.copy()
    rho = np.vdot(r, z).real
    it = 0
    while it < maxit:
        q = apply_A(p)
        pq = np.vdot(p, q).real
        alpha = rho / pq
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        hist.append(np.linalg.norm(r) / nf)
        if hist[-1] <= tol:
            break
        z = apply_P(r)
        rho_new = np.vdot(r, z).real
        beta = rho_new / rho
        p = z + beta * p
        rho = rho_new
    return x, it, hist[-1], hist


def inner(a, b):
    """<a, b> = b^H a."""
    return np.vdot(b, a)


def fcg_alpha(r, p, q):
    """Exact line search along p: <r, p> / <p, A p> (q = A p; <p, A p> is real for Hermitian A)."""
    return inner(r, p) / inner(p, q).real


def fcg_beta(z, p, q):
    """Coefficient that makes z + beta p A-orthogonal to p: -<z, A p> / <p, A p> (q = A p)."""
    return -inner(z, q) / inner(p, q).real


def fcg(apply_A, apply_P, f, x0=None, tol=1e-8, maxit=200, trace=None, with_iteration=False):
    """Flexible CG (Notay 2000, one kept direction). with_iteration: apply_P is called as apply_P(r, k)
    at iteration k (a preconditioner that changes from one iteration to the next), else apply_P(r).
    trace: a list that receives, per iteration, the dict of x, r, p, q, alpha, beta after the update.
    Returns (x, iterations, relative residual, history)."""
    B = (lambda r, k: apply_P(r, k)) if with_iteration else (lambda r, k: apply_P(r))
    f = np.asarray(f, dtype=complex)
    x = np.zeros_like(f) if x0 is None else np.array(x0, dtype=complex)
    nf = np.linalg.norm(f)
    if nf == 0.0:
        return np.zeros_like(f), 0, 0.0, [0.0]
    r = f - apply_A(x) if x0 is not None else f.copy()
    hist = [np.linalg.norm(r) / nf]
    if hist[-1] <= tol:
        return x, 0, hist[-1], hist
    p = B(r, 0)
    it = 0
    while it < maxit:
        q = apply_A(p)
        alpha = fcg_alpha(r, p, q)
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        hist.append(np.linalg.norm(r) / nf)
        beta = None
        if hist[-1] > tol:
            z = B(r, it)
            beta = fcg_beta(z, p, q)
        if trace is not None:
            trace.append({"x": x.copy(), "r": r.copy(), "p": p.copy(), "q": q.copy(), "alpha": alpha,
                          "beta": beta})
        if beta is None:
            break
        p = z + beta * p
    return x, it, hist[-1], hist
