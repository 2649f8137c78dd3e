"""Multifrontal complex-symmetric LDL^T factorisation and solve.

Oracle module (test infrastructure only).  Follows §2.2 of the paper:

* front F of supernode S is partitioned as [F_TL *; F_BL F_BR]; F_TL holds the
  Schur complement of S with respect to its descendants, F_BL the coupling to
  the ancestors, F_BR the descendants' updates for the ancestors;
* partial factorisation, in the paper's order:
    F_TL = L_F D_F L_F^T          (unit lower L_F, diagonal D_F, no pivoting)
    F_BL := F_BL L_F^{-T}
    Z_BL := F_BL
    F_BL := F_BL D_F^{-1}
    F_BR := F_BR - Z_BL F_BL^T
  after which F_BR is added into the parent front (extend-add);
* solve: up the tree x_S := L_F^{-1} x_S and x_U -= F_BL x_S added into the
  ancestors' entries, then D^{-1}, then down the tree
  x_S := L_F^{-T} (x_S - F_BL^T x_U).

The factorisation is unpivoted (the paper's solver has no pivoting); a pivot
with |d| < 1e-300 raises ZeroPivot.  Transposes are plain transposes, never
conjugates: the matrices are complex symmetric.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .symbolic import Symbolic

PIVOT_TINY = 1e-300


class ZeroPivot(ArithmeticError):
    def __init__(self, front, j, d):
        super().__init__(f"pivot {j} of front {front} is {d!r}")
        self.front, self.j, self.d = front, j, d


@dataclass
class Front:
    L_TL: np.ndarray   # s x s, unit lower (diagonal stored as ones)
    d: np.ndarray      # s
    L_BL: np.ndarray   # u x s  (final F_BL = F_BL L^{-T} D^{-1})


def ldlt_unpivoted(A: np.ndarray, front: int = -1):
    """Textbook column-by-column LDL^T of a complex symmetric matrix.

    d_j    = A_jj - sum_{k<j} L_jk^2 d_k
    L_ij   = (A_ij - sum_{k<j} L_ik L_jk d_k) / d_j,   i > j
    """
    s = A.shape[0]
    L = np.eye(s, dtype=np.complex128)
    d = np.zeros(s, dtype=np.complex128)
    for j in range(s):
        ld = L[j, :j] * d[:j]
        d[j] = A[j, j] - np.dot(L[j, :j], ld)
        if abs(d[j]) < PIVOT_TINY:
            raise ZeroPivot(front, j, d[j])
        L[j + 1:, j] = (A[j + 1:, j] - L[j + 1:, :j] @ ld) / d[j]
    return L, d


def assemble_front(H: sp.csr_matrix, rows: np.ndarray, s: int) -> np.ndarray:
    """F with F_TL = H[S, S], F_BL = H[U, S] (mirrored into the top right) and F_BR = 0."""
    F = np.zeros((len(rows), len(rows)), dtype=np.complex128)
    F[:, :s] = H[rows][:, rows[:s]].toarray()
    F[:s, s:] = F[s:, :s].T
    return F


def factor(H: sp.csr_matrix, sym: Symbolic, return_assembled: bool = False):
    """Multifrontal factorisation of H (natural node numbering of its box).

    Returns a list of Front in postorder; with ``return_assembled`` also the
    assembled F of every supernode before its partial factorisation.
    """
    fronts = []
    assembled = []
    pending = {}
    for f, sn in enumerate(sym.supernodes):
        s = len(sn.nodes)
        rows = np.concatenate([sn.nodes, sn.struct])
        F = assemble_front(H, rows, s)
        erows = sym.elim[rows]
        for c in sn.children:
            Uc, crows = pending.pop(c)
            rel = np.searchsorted(erows, sym.elim[crows])
            assert np.array_equal(erows[rel], sym.elim[crows])
            F[np.ix_(rel, rel)] += Uc
        if return_assembled:
            assembled.append(F.copy())
        # partial factorisation (§2.2, steps in the paper's order)
        L, d = ldlt_unpivoted(F[:s, :s], f)
        FBL = F[s:, :s]
        FBL = sla.solve_triangular(L, FBL.T, lower=True, unit_diagonal=True).T   # F_BL := F_BL L^{-T}
        Z = FBL.copy()                                                           # Z_BL := F_BL
        FBL = FBL / d[None, :]                                                   # F_BL := F_BL D^{-1}
        FBR = F[s:, s:] - Z @ FBL.T                                              # F_BR -= Z_BL F_BL^T
        fronts.append(Front(L, d, FBL))
        if sn.parent >= 0:
            pending[f] = (FBR, sn.struct)
    assert not pending
    return (fronts, assembled) if return_assembled else fronts


def solve(fronts, sym: Symbolic, b: np.ndarray) -> np.ndarray:
    """x = H^{-1} b from the factorisation; b has shape (N,) or (N, nrhs)."""
    x = np.array(b, dtype=np.complex128, copy=True)
    vec = x.ndim == 1
    if vec:
        x = x[:, None]
    # L^{-1}: up the tree
    for sn, fr in zip(sym.supernodes, fronts):
        xs = sla.solve_triangular(fr.L_TL, x[sn.nodes], lower=True, unit_diagonal=True)
        x[sn.nodes] = xs
        if len(sn.struct):
            x[sn.struct] -= fr.L_BL @ xs
    # D^{-1}
    for sn, fr in zip(sym.supernodes, fronts):
        x[sn.nodes] /= fr.d[:, None]
    # L^{-T}: down the tree
    for sn, fr in zip(reversed(sym.supernodes), reversed(fronts)):
        rhs = x[sn.nodes]
        if len(sn.struct):
            rhs = rhs - fr.L_BL.T @ x[sn.struct]
        x[sn.nodes] = sla.solve_triangular(fr.L_TL.T, rhs, lower=False, unit_diagonal=True)
    return x[:, 0] if vec else x


def assembled_L(fronts, sym: Symbolic):
    """The global unit lower factor L and D, in elimination order (for pins)."""
    N = sym.N
    rows, cols, vals = [], [], []
    dvec = np.zeros(N, dtype=np.complex128)
    for sn, fr in zip(sym.supernodes, fronts):
        s = len(sn.nodes)
        e_s = sym.elim[sn.nodes]
        e_u = sym.elim[sn.struct]
        dvec[e_s] = fr.d
        ii, jj = np.tril_indices(s)
        rows.append(e_s[ii]); cols.append(e_s[jj]); vals.append(fr.L_TL[ii, jj])
        if len(e_u):
            r, c = np.meshgrid(np.arange(len(e_u)), np.arange(s), indexing="ij")
            rows.append(e_u[r.ravel()]); cols.append(e_s[c.ravel()]); vals.append(fr.L_BL.ravel())
    L = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N)).tocsr()
    return L, dvec
