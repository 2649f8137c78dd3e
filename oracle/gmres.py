"""Right-preconditioned restarted GMRES(k) with modified Gram-Schmidt.

Oracle module (test infrastructure only).  §2.4 of the paper wraps the
sweeping preconditioner in GMRES(k); §3 starts from the zero vector and stops
at a relative residual of 1e-5.  Readings of what it leaves open: right
preconditioning (so the residual monitored is the true one of the symmetrised
system), modified Gram-Schmidt, complex Givens rotations, convergence tested
on the Arnoldi estimate and confirmed with the true residual at every restart;
the iteration count is the total number of inner iterations; several
right-hand sides are independent solves.
"""
from __future__ import annotations

import numpy as np


def givens(a, b):
    """c (real), s with [[c, s], [-conj(s), c]] @ [a, b] = [r, 0]."""
    if b == 0:
        return 1.0, 0.0
    if a == 0:
        return 0.0, 1.0
    rho = np.hypot(abs(a), abs(b))
    c = abs(a) / rho
    s = (a / abs(a)) * np.conj(b) / rho
    return c, s


def gmres(matvec, precond, b, tol=1e-5, k=20, maxit=500, history=False, basis=None):
    """Solve A x = b with x = M^{-1} y, x0 = 0.  Returns (x, iters, relres[, hist]).

    ``basis``, if a list, receives the Arnoldi basis V of every cycle.
    """
    b = np.asarray(b, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    n = b.shape[0]
    x = np.zeros(n, dtype=np.complex128)
    hist = []
    if bnorm == 0:
        return (x, 0, 0.0, hist) if history else (x, 0, 0.0)
    r = b.copy()
    iters = 0
    relres = 1.0
    while True:
        beta = np.linalg.norm(r)
        V = np.zeros((k + 1, n), dtype=np.complex128)
        Z = np.zeros((k, n), dtype=np.complex128)
        Hm = np.zeros((k + 1, k), dtype=np.complex128)
        cs = np.zeros(k)
        sn = np.zeros(k, dtype=np.complex128)
        g = np.zeros(k + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        j_end = 0
        for j in range(k):
            Z[j] = precond(V[j])
            w = matvec(Z[j])
            for i in range(j + 1):                       # modified Gram-Schmidt
                Hm[i, j] = np.vdot(V[i], w)
                w = w - Hm[i, j] * V[i]
            Hm[j + 1, j] = np.linalg.norm(w)
            if Hm[j + 1, j] != 0:
                V[j + 1] = w / Hm[j + 1, j]
            for i in range(j):                           # earlier rotations
                t = cs[i] * Hm[i, j] + sn[i] * Hm[i + 1, j]
                Hm[i + 1, j] = -np.conj(sn[i]) * Hm[i, j] + cs[i] * Hm[i + 1, j]
                Hm[i, j] = t
            cs[j], sn[j] = givens(Hm[j, j], Hm[j + 1, j])
            Hm[j, j] = cs[j] * Hm[j, j] + sn[j] * Hm[j + 1, j]
            Hm[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            iters += 1
            j_end = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) / bnorm < tol or iters >= maxit:
                break
        y = np.zeros(j_end, dtype=np.complex128)
        for i in range(j_end - 1, -1, -1):              # back substitution
            y[i] = (g[i] - np.dot(Hm[i, i + 1:j_end], y[i + 1:j_end])) / Hm[i, i]
        if basis is not None:
            basis.append(V[:j_end + 1].copy())
        x = x + y @ Z[:j_end]
        r = b - matvec(x)
        relres = np.linalg.norm(r) / bnorm
        if relres < tol or iters >= maxit:
            break
    return (x, iters, relres, hist) if history else (x, iters, relres)
