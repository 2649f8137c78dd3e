"""Pins of the oracle's sweep (Algs. 1.1-1.5) and GMRES(k) (§2.4)."""
import math

import numpy as np
import pytest

from oracle import discretize as dz
from oracle import gmres as gm
from oracle import naive
from oracle import sweep as sw
from paper_1204_0111_gb300 import workloads as wl


def _prob(n=6, nz=12, gamma=2, alpha=2 * math.pi, seed=0, C=4.0):
    h = 1.0 / (n + 1)
    rng = np.random.default_rng(seed)
    c = 1.0 + 0.5 * rng.random((nz, n, n))
    return dz.Helmholtz(c, h, 2 * math.pi * 0.8 / (10 * h), gamma, C, alpha)


def test_T_is_panel_block_of_dense_inverse():
    # Eqs. (1.3)-(1.4), Alg. 1.3: T_i u = (H_i^{-1})_{panel,panel} u
    p = _prob()
    P = sw.SweepingPreconditioner(p, 3, pad=3, leaf=8)
    rng = np.random.default_rng(1)
    plane = p.nx * p.ny
    for i in range(P.m):
        ap = P.aux[i]
        off = ap.lead * plane
        v = rng.normal(size=(ap.n_panel, 2)) + 1j * rng.normal(size=(ap.n_panel, 2))
        ref = np.linalg.inv(ap.H.toarray())[off:, off:] @ v
        got = P.T(i, v)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12


def test_exact_mode_inverts_J():
    # Fig. 2 (middle): with the exact auxiliary problems the sweep is an exact block LDL^T solve
    p = _prob(n=5, nz=13)
    P = sw.SweepingPreconditioner(p, 3, leaf=8, mode="exact")
    J = dz.operator_J(p)
    x = wl.random_vector(p.N, 2, seed=4)
    y = P.apply(np.asarray((J @ x.T).T))
    assert np.linalg.norm(y - x) / np.linalg.norm(x) < 1e-11


def test_exact_mode_single_planes_is_naive_block_ldlt():
    # Algs. 1.1 / 1.2 (one plane per block) give the same result as the exact sweep and J^{-1}
    n, nz = 4, 7
    h = 1.0 / (n + 1)
    rng = np.random.default_rng(2)
    p = dz.Helmholtz(1 + 0.3 * rng.random((nz, n, n)), h, 6.0, 0, 4.0, 2 * math.pi)
    J = dz.operator_J(p)
    f = wl.random_vector(p.N, 1, seed=5)[0]
    S = naive.block_ldlt(J, n * n)
    u_naive = naive.block_solve(J, n * n, S, f)
    u_dense = np.linalg.solve(J.toarray(), f)
    assert np.linalg.norm(u_naive - u_dense) / np.linalg.norm(u_dense) < 1e-12
    P = sw.SweepingPreconditioner(p, 1, leaf=4, mode="exact")
    assert P.m == nz
    u_sweep = P.apply(f)
    assert np.linalg.norm(u_sweep - u_dense) / np.linalg.norm(u_dense) < 1e-12


def test_single_panel_is_J_inverse_and_gmres_one_step():
    # panel depth >= n: m = 1, M^{-1} = J^{-1}; with alpha = 0, J = A and GMRES needs one iteration
    p = _prob(n=5, nz=8, alpha=0.0)
    P = sw.SweepingPreconditioner(p, 50, leaf=16)
    assert P.m == 1
    A = dz.operator_A(p)
    f = wl.random_vector(p.N, 1, seed=6)[0]
    assert np.linalg.norm(P.apply(f) - np.linalg.solve(A.toarray(), f)) / np.linalg.norm(P.apply(f)) < 1e-12
    x, it, rr = gm.gmres(lambda v: A @ v, P.apply, f, tol=1e-10, k=10)
    assert it == 1 and rr < 1e-10


def test_apply_is_linear_and_batched():
    p = _prob()
    P = sw.SweepingPreconditioner(p, 3, leaf=16)
    X = wl.random_vector(p.N, 3, seed=7)
    Y = P.apply(X)
    for j in range(3):
        assert np.allclose(Y[j], P.apply(X[j]), rtol=0, atol=1e-13 * np.abs(Y).max())
    assert np.allclose(P.apply(2 * X[0] - 1j * X[1]), 2 * Y[0] - 1j * Y[1], atol=1e-12 * np.abs(Y).max())


def test_gmres_matches_dense_solve_with_full_krylov_space():
    rng = np.random.default_rng(8)
    n = 25
    A = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)) + 6 * np.eye(n)
    Mi = np.linalg.inv(A + 0.3 * rng.normal(size=(n, n)))
    b = rng.normal(size=n) + 1j * rng.normal(size=n)
    basis = []
    x, it, rr, hist = gm.gmres(lambda v: A @ v, lambda v: Mi @ v, b, tol=1e-13, k=n, history=True, basis=basis)
    assert np.linalg.norm(x - np.linalg.solve(A, b)) / np.linalg.norm(x) < 1e-10
    basis = []
    gm.gmres(lambda v: A @ v, lambda v: v, b, tol=1e-13, k=8, maxit=8, basis=basis)
    V = basis[0]
    assert V.shape[0] == 9
    assert np.max(np.abs(V.conj() @ V.T - np.eye(V.shape[0]))) < 1e-12
    assert all(hist[i + 1] <= hist[i] * (1 + 1e-12) for i in range(len(hist) - 1))


def test_gmres_restarts_reach_tolerance():
    rng = np.random.default_rng(9)
    n = 60
    A = np.diag(np.linspace(1, 3, n)).astype(complex) + 0.05 * (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))
    b = rng.normal(size=n).astype(complex)
    x, it, rr = gm.gmres(lambda v: A @ v, lambda v: v, b, tol=1e-8, k=5, maxit=400)
    assert rr < 1e-8 and it > 5
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) < 1e-8


def test_manufactured_discrete_solution_is_recovered():
    # f := A u_m; the sweeping preconditioner inside GMRES recovers u_m to the tolerance
    p = _prob(n=8, nz=14, gamma=3)
    P = sw.SweepingPreconditioner(p, 3, pad=3, leaf=32)
    A = dz.operator_A(p)
    um = wl.random_vector(p.N, 1, seed=10)[0]
    f = A @ um
    x, it, rr = gm.gmres(lambda v: A @ v, P.apply, f, tol=1e-9, k=20, maxit=200)
    assert rr < 1e-9
    assert np.linalg.norm(x - um) / np.linalg.norm(um) < 1e-5


def test_moving_pml_beats_a_reflecting_pad():
    # §1.1: the PML next to the panel is what makes the Schur complement approximation good; a pad
    # without absorption (C = 0 in the pad only is not expressible, so compare to no pad at all)
    w = wl.cube_constant(12, gamma=3, panel_depth=3)
    p = dz.Helmholtz(w.c, w.h, w.omega, w.gamma, w.pml_C, w.alpha)
    A = dz.operator_A(p)
    b = dz.rhs_scale(p) * w.rhs()[0]
    its = {}
    for pad in (3, 0):
        P = sw.SweepingPreconditioner(p, w.panel_depth, pad=pad, leaf=w.leaf)
        _, its[pad], rr = gm.gmres(lambda v: A @ v, P.apply, b, tol=1e-5, k=20, maxit=300)
        assert rr < 1e-5
    assert its[3] < its[0]


def test_cube_constant_20_converges_in_few_iterations():
    # the CPU-seconds workload: 20^3, c = 1, gamma = 5, panels of 4 planes, pad 5, GMRES(20) to 1e-5
    w = wl.cube_constant(20)
    p = dz.Helmholtz(w.c, w.h, w.omega, w.gamma, w.pml_C, w.alpha)
    P = sw.SweepingPreconditioner(p, w.panel_depth, w.pad, w.leaf)
    assert P.m == 4
    A = dz.operator_A(p)
    b = dz.rhs_scale(p) * w.rhs()[0]
    x, it, rr = gm.gmres(lambda v: A @ v, P.apply, b, tol=1e-5, k=20, maxit=200)
    assert rr < 1e-5 and it <= 20


def test_apply_is_complex_symmetric():
    # Alg. 1.5 applies L^{-T} D^{-1} L^{-1} with L's blocks J_{i+1,i} T_i and D's blocks T_i^{-1}; each T_i
    # is a diagonal block of H_i^{-1} with H_i = H_i^T (§1.1), and J_{i,i+1} = J_{i+1,i}^T, so the whole
    # preconditioner is complex symmetric (transpose, not conjugate transpose)
    p = _prob(n=5, nz=11, seed=4)
    P = sw.SweepingPreconditioner(p, 2, pad=2, leaf=8)
    M = P.apply(np.eye(p.N, dtype=np.complex128)).T
    assert np.linalg.norm(M - M.T) / np.linalg.norm(M) < 1e-12
    assert np.linalg.norm(M - M.conj().T) / np.linalg.norm(M) > 1e-3
