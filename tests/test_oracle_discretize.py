"""Pins of the oracle's discretisation (Eq. (1.1), Eq. (1.5), §1.1) to facts outside it."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import discretize as dz
from oracle import panels as pn


def _prob(n=6, gamma=2, c=None, omega=7.0, alpha=2 * math.pi, C=4.0, faces=dz.ALL_FACES, nz=None):
    nz = n if nz is None else nz
    h = 1.0 / (n + 1)
    if c is None:
        rng = np.random.default_rng(1)
        c = 1.0 + 0.5 * rng.random((nz, n, n))
    return dz.Helmholtz(c, h, omega, gamma, C, alpha, faces)


def test_operator_is_complex_symmetric_bitwise():
    # §1.1: the PML makes the matrix complex symmetric, not Hermitian
    p = _prob()
    for M in (dz.operator_A(p), dz.operator_J(p)):
        D = (M - M.T).tocoo()
        assert np.count_nonzero(D.data) == 0
        H = (M - M.conj().T).tocoo()
        assert np.max(np.abs(H.data)) > 1e-3   # not Hermitian


def test_textbook_laplacian_without_pml_or_damping():
    # gamma = 0 and alpha = 0: the Kronecker-sum 7-point Laplacian minus omega^2/c^2 (library construction)
    n = 5
    h = 1.0 / (n + 1)
    rng = np.random.default_rng(7)
    c = 1.0 + rng.random((n, n, n))
    p = dz.Helmholtz(c, h, 9.0, 0, 4.0, 0.0)
    T = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]) / h ** 2
    I = sp.identity(n)
    lap = sp.kron(I, sp.kron(I, T)) + sp.kron(I, sp.kron(T, I)) + sp.kron(T, sp.kron(I, I))
    ref = (lap - sp.diags((9.0 ** 2 / c ** 2).ravel())).toarray()
    for M in (dz.operator_A(p), dz.operator_J(p)):
        assert np.max(np.abs(M.toarray() - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_block_tridiagonal_in_planes():
    # Eq. (1.2): with index i1 + i2 n + i3 n^2, only neighbouring planes couple
    p = _prob(n=4)
    M = dz.operator_A(p).tocoo()
    plane = 16
    assert np.all(np.abs(M.row // plane - M.col // plane) <= 1)


def test_damping_only_changes_the_mass_term():
    # Eq. (1.5): J - A = -((omega + i alpha)^2 - omega^2) / c^2 * s1 s2 s3 on the diagonal only
    p = _prob()
    D = (dz.operator_J(p) - dz.operator_A(p)).tocoo()
    assert np.all(D.row == D.col)
    expect = -(((p.omega + 1j * p.alpha) ** 2 - p.omega ** 2) / p.c ** 2).ravel() * dz.rhs_scale(p)
    got = np.zeros(p.N, dtype=complex)
    got[D.row] = D.data
    assert np.allclose(got, expect, rtol=1e-12, atol=0)


def test_pml_profile_closed_form():
    n, gamma, C, h = 12, 4, 3.0, 1.0 / 13
    sig = dz.pml_sigma(np.arange(n), n, gamma, C, h)
    eta = gamma * h
    assert sig[0] == pytest.approx(C / eta)                         # t = 1 at the outermost node
    assert sig[gamma - 1] == pytest.approx(C / eta / gamma ** 2)     # t = 1/gamma
    assert np.all(sig[gamma:n - gamma] == 0)                         # region of interest untouched
    assert np.allclose(sig, sig[::-1])                               # both faces alike
    half = dz.pml_sigma(np.array([-0.5]), n, gamma, C, h)[0]
    assert half == pytest.approx(C / eta * ((gamma + 0.5) / gamma) ** 2)


def test_manufactured_solution_second_order():
    # gamma = 0: u = sin(pi x) sin(pi y) sin(pi z) solves -Lap u - k^2 u = (3 pi^2 - k^2) u; error O(h^2)
    errs = []
    for n in (7, 15):
        h = 1.0 / (n + 1)
        p = dz.Helmholtz(np.ones((n, n, n)), h, 3.0, 0, 4.0, 0.0)
        x = (np.arange(n) + 1) * h
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        u = (np.sin(np.pi * X) * np.sin(np.pi * Y) * np.sin(np.pi * Z)).ravel()
        f = (3 * np.pi ** 2 - 9.0) * u
        uh = spla.spsolve(dz.operator_A(p).tocsc(), f)
        errs.append(np.max(np.abs(uh - u)))
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_pml_absorbs_outgoing_wave_1d():
    # A waveguide with one lateral node is the 1D operator -d_zz - (k^2 - 4/h^2).  With PML at both
    # ends the solution for a point source must be the OUTGOING discrete Green's function
    # C exp(+i theta |j - j0|), 2 - 2 cos(theta) = kz^2 h^2 (time convention exp(-i omega t)).
    nz = 240
    h = 1.0 / (nz + 1)
    kz = 2 * math.pi * 12.0
    omega = math.sqrt(kz ** 2 + 4.0 / h ** 2)
    p = dz.Helmholtz(np.ones((nz, 1, 1)), h, omega, 40, 40.0 * omega * h, 0.0,
                     dz.FACE_Z_LO | dz.FACE_Z_HI)
    A = dz.operator_A(p).tocsc()
    j0 = nz // 2
    f = np.zeros(nz, dtype=complex)
    f[j0] = 1.0
    u = spla.spsolve(A, f)
    theta = math.acos(1 - (kz * h) ** 2 / 2)
    Cg = h ** 2 / (-2j * math.sin(theta))
    j = np.arange(60, nz - 60)
    green = Cg * np.exp(1j * theta * np.abs(j - j0))
    assert np.max(np.abs(u[j] - green)) < 0.03 * abs(Cg)
    wrong = Cg * np.exp(-1j * theta * np.abs(j - j0))      # incoming wave: must NOT match
    assert np.max(np.abs(u[j] - wrong)) > 0.5 * abs(Cg)


def test_panel_plan():
    assert pn.panel_plan(20, 5, 4) == [(0, 9), (9, 13), (13, 17), (17, 20)]
    assert len(pn.panel_plan(100, 8, 4)) == 23
    assert pn.panel_plan(10, 2, 20) == [(0, 10)]


def test_aux_problem_panel_block_is_J_block():
    # Alg. 1.4: H_i is J_{i,i} with PML prefixed; its panel block equals J's except the a_3
    # term of the panel's first plane at the half-point shared with the pad
    p = _prob(n=5, gamma=2, nz=14)
    J = dz.operator_J(p)
    plan = pn.panel_plan(p.nz, p.gamma, 3)
    plane = p.nx * p.ny
    for (z0, z1) in plan[1:]:
        ap = pn.aux_problem(p, z0, z1, pad=3)
        off = ap.lead * plane
        Hp = ap.H[off:, off:].toarray()
        Jp = J[z0 * plane:z1 * plane][:, z0 * plane:z1 * plane].toarray()
        D = Hp - Jp
        D[np.arange(plane), np.arange(plane)] = 0.0           # first plane's diagonal differs
        assert np.max(np.abs(D)) == 0.0
        diag_diff = np.diag(Hp - Jp)[:plane]
        assert np.max(np.abs(diag_diff)) > 0.0
        # the pad's mass term is J's, with c copied from the panel's first plane: changing alpha
        # shifts the pad diagonal by -((w + i a')^2 - (w + i a)^2) / c(z0)^2 * s1 s2 s3
        p2 = dz.Helmholtz(p.c, p.h, p.omega, p.gamma, p.pml_C, p.alpha + 1.0, p.pml_faces)
        ap2 = pn.aux_problem(p2, z0, z1, pad=3)
        dd = (ap2.H.diagonal() - ap.H.diagonal())[:off].reshape(ap.lead, p.ny, p.nx)
        s1, s2, s3 = dz.global_stretches(p)
        lat = s2.node[:, None] * s1.node[None, :]
        shift = -((p.omega + 1j * (p.alpha + 1.0)) ** 2 - (p.omega + 1j * p.alpha) ** 2) / p.c[z0] ** 2
        for k in range(ap.lead):
            ratio = dd[k] / (shift * lat)          # = s3 at pad node k, the same over the plane
            assert np.allclose(ratio, ratio.flat[0], rtol=1e-12)
            sig = (ratio.flat[0] - 1).imag * p.omega
            assert sig == pytest.approx(p.pml_C / (3 * p.h) * ((3 - k) / 3) ** 2, rel=1e-9)


def test_pad_profile_closed_form():
    # the pad's x3-stretch at its nodes: sigma = C/(p h) ((p - k)/p)^2, zero on the panel
    p = _prob(n=4, gamma=2, nz=12, C=5.0)
    pad = 4
    z0, z1 = pn.panel_plan(p.nz, p.gamma, 3)[1]
    ap = pn.aux_problem(p, z0, z1, pad)
    plane = p.nx * p.ny
    # read sigma_3 back from the coupling between plane k and k+1 at lateral node (1, 1):
    # H[k, k+1] = -s1 s2 / s3(k + 1/2) / h^2
    s1 = 1.0 + 1j * dz.pml_sigma(np.arange(4), 4, 2, 5.0, p.h) / p.omega
    i = 1 + 4 * 1
    for k in range(pad + (z1 - z0) - 1):
        a3 = -ap.H[k * plane + i, (k + 1) * plane + i] * p.h ** 2
        s3h = s1[1] * s1[1] / a3
        sigma = (s3h - 1.0).imag * p.omega
        t = max(0.0, (pad - (k + 0.5)) / pad)
        assert sigma == pytest.approx(5.0 / (pad * p.h) * t * t, abs=1e-9)
