"""Pins of the oracle's multifrontal LDL^T (§2.2) against dense linear algebra."""
import math

import numpy as np
import pytest

from oracle import discretize as dz
from oracle import multifrontal as mf
from oracle import panels as pn
from oracle import symbolic as sy


def _aux(n=6, nz=10, gamma=2, depth=3, pad=2, panel=1, seed=0):
    h = 1.0 / (n + 1)
    rng = np.random.default_rng(seed)
    c = 1.0 + 0.6 * rng.random((nz, n, n))
    p = dz.Helmholtz(c, h, 2 * math.pi / (10 * h) * 0.9, gamma, 4.0, 2 * math.pi)
    z0, z1 = pn.panel_plan(nz, gamma, depth)[panel]
    return p, pn.aux_problem(p, z0, z1, pad)


@pytest.mark.parametrize("leaf", [4, 16, 64])
def test_solve_matches_dense_solve(leaf):
    p, ap = _aux()
    sym = sy.nested_dissection(ap.nx, ap.ny, ap.depth, leaf)
    fr = mf.factor(ap.H, sym)
    rng = np.random.default_rng(3)
    b = rng.normal(size=(ap.H.shape[0], 3)) + 1j * rng.normal(size=(ap.H.shape[0], 3))
    x = mf.solve(fr, sym, b)
    xd = np.linalg.solve(ap.H.toarray(), b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-12


def test_factor_reconstructs_matrix():
    p, ap = _aux(n=5)
    sym = sy.nested_dissection(ap.nx, ap.ny, ap.depth, 10)
    fr = mf.factor(ap.H, sym)
    L, d = mf.assembled_L(fr, sym)
    L = L.toarray()
    assert np.allclose(np.diag(L), 1.0) and np.all(np.triu(L, 1) == 0)
    Hp = ap.H.toarray()[np.ix_(sym.order, sym.order)]
    R = L @ np.diag(d) @ L.T
    assert np.linalg.norm(R - Hp) / np.linalg.norm(Hp) < 1e-13


def test_assembled_front_is_schur_complement():
    # F_TL, F_BL: Schur complement of the front rows w.r.t. the descendants; F_BR: descendants' update only
    p, ap = _aux(n=6)
    sym = sy.nested_dissection(ap.nx, ap.ny, ap.depth, 12)
    _, assembled = mf.factor(ap.H, sym, return_assembled=True)
    H = ap.H.toarray()
    for sn, F in zip(sym.supernodes, assembled):
        s = len(sn.nodes)
        R = np.concatenate([sn.nodes, sn.struct])
        desc = sym.order[sn.subtree_first:sn.first]
        Sch = H[np.ix_(R, R)]
        if len(desc):
            Sch = Sch - H[np.ix_(R, desc)] @ np.linalg.solve(H[np.ix_(desc, desc)], H[np.ix_(desc, R)])
        expect = Sch.copy()
        U = sn.struct
        expect[s:, s:] -= H[np.ix_(U, U)]
        scale = np.max(np.abs(H))
        assert np.max(np.abs(F[:, :s] - expect[:, :s])) < 1e-11 * scale
        if len(U):
            assert np.max(np.abs(F[s:, s:] - expect[s:, s:])) < 1e-11 * scale


def test_ldlt_textbook_properties():
    rng = np.random.default_rng(5)
    A = rng.normal(size=(30, 30)) + 1j * rng.normal(size=(30, 30))
    A = A + A.T + 40 * np.eye(30)                 # complex symmetric, not Hermitian
    L, d = mf.ldlt_unpivoted(A)
    assert np.allclose(np.triu(L, 1), 0) and np.allclose(np.diag(L), 1)
    assert np.linalg.norm(L @ np.diag(d) @ L.T - A) / np.linalg.norm(A) < 1e-14
    # the pivots are ratios of leading principal minors
    minors = [np.linalg.det(A[:k, :k]) for k in range(1, 31)]
    ratios = [minors[0]] + [minors[k] / minors[k - 1] for k in range(1, 30)]
    assert np.allclose(d, ratios, rtol=1e-9)


def test_zero_pivot_is_reported():
    A = np.array([[0.0, 1.0], [1.0, 2.0]], dtype=complex)
    with pytest.raises(mf.ZeroPivot):
        mf.ldlt_unpivoted(A)
