"""Preconditioned conjugate gradients for the HPD least-squares system (Sec. 5.3, Sec. 6).

Test infrastructure: part of the CPU oracle, see `oracle/__init__.py`.

The paper solves A u = f by CG preconditioned with P-hat, tolerance 1e-8,
zero initial guess, at most 200 iterations. A is Hermitian positive definite
(the paper says "symmetric"; read Hermitian), inner products are
<a, b> = b^H a. Stopping test: ||f - A x_k||_2 <= tol ||f||_2 on the
recursively updated residual (the paper does not name its norm; for x_0 = 0
this equals ||r_k|| / ||r_0||).

`flexible=True` replaces beta = <r_k+1, z_k+1>/<r_k, z_k> by the
Polak-Ribiere form <r_k+1, z_k+1 - z_k>/<r_k, z_k>, the standard choice when
the preconditioner is applied inexactly (not in the paper; parity unpinned
beyond the exact-preconditioner case, where both forms coincide: the extra term
<r_k+1, z_k> vanishes in exact arithmetic for a fixed Hermitian preconditioner
or one rescaled at each step, so no closed form checks it).
"""
import numpy as np


def pcg(apply_A, apply_P, f, x0=None, tol=1e-8, maxit=200, flexible=False):
    """Returns (x, iterations, relative residual, history of relative residuals)."""
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
        z_new = apply_P(r)
        rho_new = np.vdot(r, z_new).real
        beta = (rho_new - np.vdot(r, z).real) / rho if flexible else rho_new / rho
        z = z_new
        p = z + beta * p
        rho = rho_new
    return x, it, hist[-1], hist
