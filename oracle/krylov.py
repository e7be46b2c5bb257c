"""Restarted GMRES with Givens rotations (complex128).

Oracle (test infrastructure only).  The paper runs full GMRES with a
relative-residual stopping tolerance (Section 4) and names restarted GMRES
as the natural next step (Sections 4 and 5).  This is GMRES(m): Arnoldi
with modified Gram-Schmidt, the small least-squares problem reduced by
complex Givens rotations, x0 given, restart every m steps.

Preconditioning, eq. (2): left (P^{-1} A x = P^{-1} b, the residual tested is
the preconditioned one) or right (A P^{-1} u = b, x = P^{-1} u, the residual
tested is the true ||b - A x|| / ||b||).  Right is the default reading.
"""
from __future__ import annotations

import numpy as np


def _givens(a: complex, b: complex):
    """Rotation [c s; -conj(s) c] with real c mapping (a, b) to (r, 0)."""
    if b == 0:
        return 1.0, 0.0 + 0.0j, a
    if a == 0:
        return 0.0, 1.0 + 0.0j, b
    rho = np.sqrt(abs(a) ** 2 + abs(b) ** 2)
    c = abs(a) / rho
    s = (a / abs(a)) * np.conj(b) / rho
    r = (a / abs(a)) * rho
    return c, s, r


def gmres(matvec, b: np.ndarray, x0: np.ndarray | None = None, tol: float = 1e-6,
          restart: int = 50, maxiter: int = 2000, precond=None, side: str = "right"):
    """Solve A x = b.  Returns (x, info) with info = {iters, restarts, history, converged}.

    ``history`` holds the relative residual estimate after every iteration
    (preconditioned residual for side='left').
    """
    shape = b.shape
    bf = b.reshape(-1).astype(np.complex128)
    n = bf.size
    M = precond if precond is not None else (lambda v: v)
    A = lambda v: matvec(v.reshape(shape)).reshape(-1)
    Mv = lambda v: M(v.reshape(shape)).reshape(-1)
    x = np.zeros(n, dtype=np.complex128) if x0 is None else x0.reshape(-1).astype(np.complex128).copy()

    if side == "left":
        op = lambda v: Mv(A(v))
        rhs = Mv(bf)
    else:
        op = lambda v: A(Mv(v))
        rhs = bf
    bnorm = np.linalg.norm(rhs)
    if bnorm == 0:
        return np.zeros(shape, dtype=np.complex128), dict(iters=0, restarts=0, history=[], converged=True)

    iters = 0
    restarts = 0
    history = []
    converged = False
    while iters < maxiter:
        if side == "left":
            r = Mv(bf - A(x))
        else:
            r = bf - A(x)
        beta = np.linalg.norm(r)
        if beta / bnorm <= tol:
            converged = True
            break
        V = np.zeros((restart + 1, n), dtype=np.complex128)
        H = np.zeros((restart + 1, restart), dtype=np.complex128)
        cs = np.zeros(restart)
        sn = np.zeros(restart, dtype=np.complex128)
        g = np.zeros(restart + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(restart):
            w = op(V[j])
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            for i in range(j):
                hi, hi1 = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * hi + sn[i] * hi1
                H[i + 1, j] = -np.conj(sn[i]) * hi + cs[i] * hi1
            c, s, rr = _givens(H[j, j], H[j + 1, j])
            cs[j], sn[j] = c, s
            H[j, j] = rr
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(s) * g[j]
            g[j] = c * g[j]
            iters += 1
            j_done = j + 1
            res = abs(g[j + 1]) / bnorm
            history.append(res)
            hnext = np.linalg.norm(w)
            if res <= tol or hnext == 0 or iters >= maxiter:
                break
            V[j + 1] = w / hnext
        y = np.zeros(j_done, dtype=np.complex128)
        for i in range(j_done - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:j_done] @ y[i + 1:j_done]) / H[i, i]
        upd = V[:j_done].T @ y
        if side == "left":
            x = x + upd
        else:
            x = x + Mv(upd)
        restarts += 1
    else:
        pass
    if not converged:
        if side == "left":
            r = Mv(bf - A(x))
        else:
            r = bf - A(x)
        converged = np.linalg.norm(r) / bnorm <= tol
    return x.reshape(shape), dict(iters=iters, restarts=restarts, history=history,
                                  converged=bool(converged))


def bicgstab(matvec, b: np.ndarray, x0: np.ndarray | None = None, tol: float = 1e-6,
             maxiter: int = 4000, precond=None):
    """Right-preconditioned BiCG-Stab (van der Vorst), the paper's second solver (Section 4).

    Solves A M u = b, x = M u, with the shadow residual r_hat = r0 and the
    conjugated inner product.  Stops when the true-residual recurrence
    ||r|| / ||b|| <= tol (checked after each half step).  Returns
    (x, info) with info = {iters, half_steps, history, converged}; one
    iteration is two matvecs and two preconditioner applies, half_steps counts
    the half steps taken (2 iters, one less when the first half converged).
    """
    shape = b.shape
    bf = b.reshape(-1).astype(np.complex128)
    M = precond if precond is not None else (lambda v: v)
    A = lambda v: matvec(v.reshape(shape)).reshape(-1)
    Mv = lambda v: M(v.reshape(shape)).reshape(-1)
    x = np.zeros_like(bf) if x0 is None else x0.reshape(-1).astype(np.complex128).copy()
    bnorm = np.linalg.norm(bf)
    if bnorm == 0:
        return np.zeros(shape, dtype=np.complex128), dict(iters=0, half_steps=0, history=[],
                                                          converged=True)
    r = bf - A(x)
    rhat = r.copy()
    half = 0
    rho = alpha = omega = 1.0 + 0j
    v = np.zeros_like(bf)
    p = np.zeros_like(bf)
    history = []
    converged = np.linalg.norm(r) / bnorm <= tol
    it = 0
    while not converged and it < maxiter:
        rho_new = np.vdot(rhat, r)
        beta = (rho_new / rho) * (alpha / omega)
        p = r + beta * (p - omega * v)
        ph = Mv(p)
        v = A(ph)
        alpha = rho_new / np.vdot(rhat, v)
        s = r - alpha * v
        it += 1
        half += 1
        if np.linalg.norm(s) / bnorm <= tol:
            x = x + alpha * ph
            history.append(np.linalg.norm(s) / bnorm)
            converged = True
            break
        half += 1
        sh = Mv(s)
        t = A(sh)
        omega = np.vdot(t, s) / np.vdot(t, t)
        x = x + alpha * ph + omega * sh
        r = s - omega * t
        rho = rho_new
        res = np.linalg.norm(r) / bnorm
        history.append(res)
        converged = res <= tol
    return x.reshape(shape), dict(iters=it, half_steps=half, history=history,
                                  converged=bool(converged))
