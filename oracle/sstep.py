"""s-step (Newton-basis) restarted GMRES (complex128).

Oracle (test infrastructure only).  The paper solves with GMRES and names
restarted GMRES as the next step (Sections 4 and 5); this is the same
GMRES(m) computed in blocks of s basis vectors, the published s-step form:

- the Krylov vectors of a block come from the Newton recurrence
  v_{t+1} = (A P^{-1} - theta_t) v_t started at the block's last orthonormal
  vector (Bai, Hu & Reichel, IMA J. Numer. Anal. 14 (1994) 563);
- the shifts theta are Ritz values of the first cycle ordered as Leja points
  (Reichel, BIT 30 (1990) 332): the first of largest modulus, each next one
  maximising the product of its distances to those already taken;
- the block is orthogonalised against the basis by block classical
  Gram-Schmidt run twice, then within itself by a Cholesky QR of its Gram
  matrix;
- the Hessenberg columns of the block follow from the change of basis
  (Hoemmen, "Communication-avoiding Krylov subspace methods", UC Berkeley
  2010, Section 3.3): with [v_0 .. v_s] = [Q_j, Q_new] Rc and
  A P^{-1} [v_0 .. v_{s-1}] = [v_0 .. v_s] B (B: shifts on the diagonal,
  ones below), H_new = (Rc B - [H_j Rc_top; 0]) Rc_bot^{-1}.

In exact arithmetic the cycle spans the same Krylov space with the same
orthonormal basis and Hessenberg matrix as Arnoldi (the Arnoldi
factorisation with a positive subdiagonal is unique), so the iterates are
GMRES(m)'s.  The first cycle of a solve is plain Arnoldi (it supplies the Ritz
values).  Right preconditioning, x0 = 0 unless given; the residual tested
after each column is the Givens estimate, and the cycle stops at the first
column that meets the tolerance, so iterations are counted per column while
matrix-vector products come in whole blocks.
"""
from __future__ import annotations

import numpy as np

from .krylov import _givens


def leja_order(points, count: int) -> list[int]:
    """Indices of the first ``count`` Leja points of ``points`` in order.

    The first is the point of largest modulus; each next one maximises the
    product of its distances to the points already chosen (sum of logarithms;
    a point already chosen has distance zero).  Ties (within a relative
    1e-12, rounding) go to the first point in the input order."""
    z = np.asarray(points, dtype=np.complex128)
    n = z.size
    count = min(count, n)
    if count <= 0:
        return []

    def first_max(v):
        top = v.max()
        return int(np.flatnonzero(v >= top - 1e-12 * max(1.0, abs(top)))[0])

    mod = np.abs(z)
    chosen = [int(np.flatnonzero(mod >= mod.max() * (1 - 1e-12))[0])]
    score = np.zeros(n)
    while len(chosen) < count:
        with np.errstate(divide="ignore"):
            score = score + np.log(np.abs(z - z[chosen[-1]]))
        score[chosen[-1]] = -np.inf
        chosen.append(first_max(score))
    return chosen


def ritz_shifts(Hraw: np.ndarray, jl: int, s: int) -> np.ndarray:
    """s Newton shifts from an Arnoldi cycle of jl columns: the eigenvalues of
    the leading k x k block of its Hessenberg matrix, k = min(jl, 4 s), in
    Leja order (fewer than s when k < s; the rest are zero)."""
    k = min(jl, 4 * s)
    theta = np.zeros(s, dtype=np.complex128)
    if k == 0:
        return theta
    ev = np.linalg.eigvals(Hraw[:k, :k])
    idx = leja_order(ev, s)
    theta[:len(idx)] = ev[idx]
    return theta


def block_hessenberg(Hraw: np.ndarray, j: int, C: np.ndarray, R: np.ndarray,
                     theta: np.ndarray) -> np.ndarray:
    """Hessenberg columns j .. j+s-1 of a Newton block (Hoemmen 2010, Sec. 3.3).

    Hraw: the (unrotated) Hessenberg matrix, columns < j filled.  C: (j+1) x s
    coefficients of the block against Q_j = [q_0 .. q_j]; R: s x s upper
    triangular with (W - Q_j C) = Q_new R; theta: the block's s shifts.
    Returns the (j+s+1) x s block of new columns."""
    s = R.shape[0]
    n = j + s + 1
    Rc = np.zeros((n, s + 1), dtype=np.complex128)   # [v_0 .. v_s] = [Q_j, Q_new] Rc
    Rc[j, 0] = 1.0
    Rc[:j + 1, 1:] = C
    Rc[j + 1:, 1:] = R
    B = np.zeros((s + 1, s), dtype=np.complex128)    # A P^-1 [v_0..v_{s-1}] = [v_0..v_s] B
    B[np.arange(s), np.arange(s)] = theta
    B[np.arange(1, s + 1), np.arange(s)] = 1.0
    M = Rc @ B
    if j > 0:
        M[:j + 1] -= Hraw[:j + 1, :j] @ Rc[:j, :s]
    Rbot = Rc[j:j + s, :s]                           # upper triangular, unit (0, 0)
    Hn = np.linalg.solve(Rbot.T, M.T).T              # M Rbot^{-1}
    for t in range(s):                               # Hessenberg: nothing below row j+t+1
        Hn[j + t + 2:, t] = 0.0
    return Hn


def newton_block(op, v0: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """W[t] = (op - theta_t) W[t-1], W[-1] = v0: the s Newton vectors."""
    W = np.zeros((theta.size, v0.size), dtype=np.complex128)
    prev = v0
    for t, th in enumerate(theta):
        W[t] = op(prev) - th * prev
        prev = W[t]
    return W


def orthogonalise_block(Q: np.ndarray, W: np.ndarray):
    """Block CGS twice against the rows of Q, then Cholesky QR of the block.

    Returns (Qn, C, R) with W = Q^T C + Qn^T R (rows are vectors), or None
    when the block's Gram matrix is not numerically positive definite."""
    C1 = Q.conj() @ W.T
    W = W - (Q.T @ C1).T
    C2 = Q.conj() @ W.T
    W = W - (Q.T @ C2).T
    G = W.conj() @ W.T                                # G[a, b] = <W_a, W_b>
    try:
        L = np.linalg.cholesky(G)                     # G = L L^H, R = L^H
    except np.linalg.LinAlgError:
        return None
    R = L.conj().T
    Qn = np.linalg.solve(R.T, W)                      # rows of W^T R^{-1}
    return Qn, C1 + C2, R


def sstep_gmres(matvec, b: np.ndarray, x0: np.ndarray | None = None, tol: float = 1e-6,
                restart: int = 50, maxiter: int = 2000, precond=None, s: int = 5):
    """Solve A x = b (right preconditioning).  Returns (x, info) with info =
    {iters, matvecs, restarts, history, converged, shifts}."""
    shape = b.shape
    bf = b.reshape(-1).astype(np.complex128)
    n = bf.size
    M = precond if precond is not None else (lambda v: v)
    A = lambda v: matvec(v.reshape(shape)).reshape(-1)
    Mv = lambda v: M(v.reshape(shape)).reshape(-1)
    op = lambda v: A(Mv(v))
    x = np.zeros(n, dtype=np.complex128) if x0 is None else x0.reshape(-1).astype(np.complex128).copy()
    bnorm = np.linalg.norm(bf)
    info = dict(iters=0, matvecs=0, restarts=0, history=[], converged=True, shifts=None)
    if bnorm == 0:
        return np.zeros(shape, dtype=np.complex128), info
    m = restart
    theta = None
    converged = False
    while info["iters"] < maxiter:
        r = bf - A(x)
        beta = np.linalg.norm(r)
        if beta / bnorm <= tol:
            converged = True
            break
        V = np.zeros((m + 1, n), dtype=np.complex128)
        Hraw = np.zeros((m + 1, m), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)  # rotated copy
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        steps = min(m, maxiter - info["iters"])
        j = 0
        jl = 0
        stop = False
        while j < steps and not stop:
            if theta is None:                          # first cycle: Arnoldi (one column)
                w = op(V[j])
                info["matvecs"] += 1
                for i in range(j + 1):
                    Hraw[i, j] = np.vdot(V[i], w)
                    w = w - Hraw[i, j] * V[i]
                Hraw[j + 1, j] = np.linalg.norm(w)
                if Hraw[j + 1, j] != 0:
                    V[j + 1] = w / Hraw[j + 1, j]
                ncol = 1
            else:
                sb = min(s, m - j)
                Wb = newton_block(op, V[j], theta[:sb])
                info["matvecs"] += sb
                res = orthogonalise_block(V[:j + 1], Wb)
                if res is None:                        # breakdown: end the cycle here
                    break
                Qn, C, R = res
                Hraw[:j + sb + 1, j:j + sb] = block_hessenberg(Hraw, j, C, R, theta[:sb])
                V[j + 1:j + sb + 1] = Qn
                ncol = min(sb, steps - j)
            for t in range(ncol):
                c = j + t
                H[:c + 2, c] = Hraw[:c + 2, c]
                for i in range(c):
                    hi, hi1 = H[i, c], H[i + 1, c]
                    H[i, c] = cs[i] * hi + sn[i] * hi1
                    H[i + 1, c] = -np.conj(sn[i]) * hi + cs[i] * hi1
                cc, ss, rr = _givens(H[c, c], H[c + 1, c])
                cs[c], sn[c] = cc, ss
                H[c, c] = rr
                H[c + 1, c] = 0.0
                g[c + 1] = -np.conj(ss) * g[c]
                g[c] = cc * g[c]
                info["iters"] += 1
                jl = c + 1
                est = abs(g[c + 1]) / bnorm
                info["history"].append(est)
                if est <= tol or Hraw[c + 1, c] == 0 or info["iters"] >= maxiter:
                    stop = True
                    break
            j += ncol
        if theta is None:
            theta = ritz_shifts(Hraw, jl, s)
            info["shifts"] = theta
        y = np.zeros(jl, dtype=np.complex128)
        for i in range(jl - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:jl] @ y[i + 1:jl]) / H[i, i]
        x = x + Mv(V[:jl].T @ y)
        info["restarts"] += 1
        if jl == 0:
            break
    if not converged:
        converged = np.linalg.norm(bf - A(x)) / bnorm <= tol
    info["converged"] = bool(converged)
    return x.reshape(shape), info
