"""Algs. 1.1 and 1.2: the naive block tridiagonal LDL^T factorisation and solve.

Oracle module (test infrastructure only), dense plane blocks, tiny grids.
With one plane per block, S_0 := A_{0,0} and S_{i+1} := A_{i+1,i+1} -
A_{i+1,i} S_i^{-1} A_{i+1,i}^T; the solve applies L^{-1}, D^{-1} and L^{-T}
loop by loop.  The blocks are taken from a global sparse matrix in the
ordering of Eq. (1.2) (plane i = unknowns [i n1 n2, (i+1) n1 n2)).
"""
from __future__ import annotations

import numpy as np


def block_ldlt(M, plane: int):
    """Alg. 1.1 on the dense version of M; returns the list of S_i."""
    M = M.toarray() if hasattr(M, "toarray") else np.asarray(M)
    nb = M.shape[0] // plane
    B = lambda i, j: M[i * plane:(i + 1) * plane, j * plane:(j + 1) * plane]
    S = [B(0, 0).copy()]
    for i in range(nb - 1):
        A10 = B(i + 1, i)
        S.append(B(i + 1, i + 1) - A10 @ np.linalg.solve(S[i], A10.T))
    return S


def block_solve(M, plane: int, S, f):
    """Alg. 1.2 with the S_i of ``block_ldlt``."""
    M = M.toarray() if hasattr(M, "toarray") else np.asarray(M)
    nb = M.shape[0] // plane
    B = lambda i, j: M[i * plane:(i + 1) * plane, j * plane:(j + 1) * plane]
    u = [np.array(f[i * plane:(i + 1) * plane], dtype=np.complex128) for i in range(nb)]
    for i in range(nb - 1):                 # L^{-1}
        u[i + 1] = u[i + 1] - B(i + 1, i) @ np.linalg.solve(S[i], u[i])
    for i in range(nb):                     # D^{-1}
        u[i] = np.linalg.solve(S[i], u[i])
    for i in range(nb - 2, -1, -1):         # L^{-T}
        u[i] = u[i] - np.linalg.solve(S[i], B(i + 1, i).T @ u[i + 1])
    return np.concatenate(u)
