"""Batches of independent problems (psp_setup_batch) through the C ABI.

A batch factors all problems' panels level by level in shared launches, runs their sweeps side by
side in one persistent launch, and solves them with one lockstep GMRES whose columns are the
(problem, right-hand side) pairs.  Each problem's arithmetic is the same as in its own handle, so
factors, applications and GMRES iterates must equal those of separate handles bit for bit; the
separate handles are themselves held to the oracle in test_gpu_parity.py, and each batched
problem is also checked against the oracle directly.
"""
import math

import numpy as np
import pytest

from oracle import discretize as dz
from oracle import sweep as osw
from paper_1204_0111_gb300 import workloads as wl

from _cases import random_velocity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1204_0111_gb300 import psp  # noqa: E402


def problems_small():
    out = []
    w = wl.cube_constant(20)
    out.append(dict(c=w.c, h=w.h, omega=w.omega, gamma=w.gamma, panel_depth=w.panel_depth))
    for (nx, ny, nz, gam, d, seed) in ((16, 12, 18, 3, 3, 5), (24, 20, 22, 4, 4, 6)):
        h = 1.0 / (max(nx, ny, nz) + 1)
        out.append(dict(c=random_velocity(nx, ny, nz, seed), h=h, omega=2 * math.pi / (10 * h), gamma=gam,
                        panel_depth=d))
    return out


def problems_tc():
    # fronts large enough for the 128 x 128 tensor-core tiles, next to a small problem
    n = 40
    h = 1.0 / (n + 1)
    return [dict(c=random_velocity(n, n, 14, 2, 1.0, 1.4), h=h, omega=2 * math.pi / (10 * h), gamma=2, panel_depth=2),
            problems_small()[1]]


def single(pr, **kw):
    return psp.SweepingPreconditioner(torch.from_numpy(pr["c"]).cuda(), pr["h"], pr["omega"], pr["gamma"],
                                      pr["panel_depth"], **kw)


def batched(prs, **kw):
    return psp.SweepingPreconditionerBatch([dict(p, c=torch.from_numpy(p["c"]).cuda()) for p in prs], **kw)


def oracle_problem(pr):
    return dz.Helmholtz(pr["c"], pr["h"], pr["omega"], pr["gamma"], 4.0, 2 * math.pi)


def assert_same_factors(B, singles):
    panel = 0
    for P in singles:
        for i in range(P.info()["panels"]):
            nf = len(psp.parse_symbolic(P.symbolic(i))[1])
            for f in range(nf):
                Gs, s, u = P.export_front(i, f)
                Gb, sb, ub = B.export_front(panel, f)
                assert (s, u) == (sb, ub)
                assert np.array_equal(Gs, Gb), (panel, f)
            assert np.array_equal(P.symbolic(i), B.symbolic(panel))
            panel += 1
    assert B.info()["panels"] == panel


@pytest.mark.parametrize("precision,si", [("c128", "extended"), ("c64", "extended"), ("c128", "paper"),
                                          ("c64", "paper"), ("c128", "none")])
def test_batch_equals_separate_handles(precision, si):
    prs = problems_small() if precision == "c128" else problems_tc()
    B = batched(prs, precision=precision, selective_inversion=si)
    singles = [single(p, precision=precision, selective_inversion=si) for p in prs]
    assert B.points == [p["c"].size for p in prs]
    assert_same_factors(B, singles)
    nrhs = 2
    rs = [wl.random_vector(p["c"].size, nrhs, seed=70 + q) for q, p in enumerate(prs)]
    flat = torch.from_numpy(B.pack(rs)).cuda()
    out = torch.empty_like(flat)
    B.apply(flat, out)
    got = B.unpack(out.cpu().numpy(), nrhs)
    for q, (P, r) in enumerate(zip(singles, rs)):
        o = np.zeros_like(r)
        P.apply(r, o)
        assert np.array_equal(got[q], o), q
    # matvec with A and J, per problem
    for which in (0, 1):
        y = torch.empty_like(flat)
        B.matvec(flat, y, which)
        yb = B.unpack(y.cpu().numpy(), nrhs)
        for q, (pr, r) in enumerate(zip(prs, rs)):
            M = dz.operator_A(oracle_problem(pr)) if which == 0 else dz.operator_J(oracle_problem(pr))
            ref = (M @ r.T).T
            assert np.linalg.norm(yb[q] - ref) / np.linalg.norm(ref) < 1e-13


def test_batch_apply_matches_oracle_per_problem():
    prs = problems_small()
    B = batched(prs)
    nrhs = 1
    rs = [wl.random_vector(p["c"].size, nrhs, seed=90 + q) for q, p in enumerate(prs)]
    out = np.zeros(B.N * nrhs, dtype=np.complex128)
    B.apply(B.pack(rs), out)
    for q, (pr, r) in enumerate(zip(prs, rs)):
        O = osw.SweepingPreconditioner(oracle_problem(pr), pr["panel_depth"], pr["gamma"], 64)
        ref = O.apply(r)
        got = B.unpack(out, nrhs)[q]
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-10, q


def test_batch_solve_equals_separate_solves_and_reaches_tolerance():
    prs = problems_small()
    B = batched(prs)
    nrhs = 2
    fs = []
    for pr in prs:
        nz, ny, nx = pr["c"].shape
        fs.append(np.stack([wl.gaussian_source(nx, ny, nz, pr["h"], x0) for x0 in ((0.5, 0.5, 0.5), (0.3, 0.6, 0.4))]))
    fd = torch.from_numpy(B.pack(fs)).cuda()
    ud = torch.zeros_like(fd)
    info = B.solve(fd, ud, tol=1e-6, k=10, maxit=400)
    assert info["converged"] == 1
    ub = B.unpack(ud.cpu().numpy(), nrhs)
    its = []
    for q, (pr, f) in enumerate(zip(prs, fs)):
        P = single(pr)
        u = np.zeros_like(f)
        inf_q = P.solve(f, u, tol=1e-6, k=10, maxit=400)
        its.append(inf_q["iterations"])
        assert np.array_equal(ub[q], u), q
        p = oracle_problem(pr)
        A = dz.operator_A(p)
        b = dz.rhs_scale(p)[None, :] * f
        for j in range(nrhs):
            assert np.linalg.norm(b[j] - A @ ub[q][j]) / np.linalg.norm(b[j]) < 1e-6
    assert info["iterations"] == max(its)


def test_level_groups_under_a_small_temporary_budget_give_the_same_factors():
    pr = problems_tc()[0]
    for precision in ("c128", "c64"):
        P = single(pr, precision=precision)
        Q = single(pr, precision=precision, setup_temp_mb=1)
        assert_same_factors(Q, [P])


def test_batch16_uneven_problems_eight_shots_complex64():
    # the batching workload: 16 independent problems, n = 40 + 8 (k mod 11), smooth random velocity,
    # gamma 8, complex64 fronts, 8 shots each solved as one block; every (problem, shot) column to
    # a true relative residual of 1e-5, and the two smallest problems equal to their own handles
    ws = [wl.cube_smooth(k) for k in range(16)]
    prs = [dict(c=w.c, h=w.h, omega=w.omega, gamma=w.gamma, panel_depth=w.panel_depth) for w in ws]
    B = batched(prs, precision="c64", pml_C=ws[0].pml_C)   # one amplitude for the whole batch
    nrhs = 8
    fs = [w.rhs() for w in ws]
    fd = torch.from_numpy(B.pack(fs)).cuda()
    ud = torch.zeros_like(fd)
    info = B.solve(fd, ud, tol=1e-5, k=20, maxit=400)
    assert info["converged"] == 1
    ub = B.unpack(ud.cpu().numpy(), nrhs)
    for q, w in enumerate(ws):
        p = dz.Helmholtz(w.c, w.h, w.omega, w.gamma, w.pml_C, w.alpha)
        A = dz.operator_A(p)
        b = dz.rhs_scale(p)[None, :] * fs[q]
        for j in range(nrhs):
            assert np.linalg.norm(b[j] - A @ ub[q][j]) / np.linalg.norm(b[j]) < 1e-5, (q, j)
    B.close()
    del fd, ud
    small = [0, 11]   # n = 40 twice (seeds 400 and 411)
    Bs = batched([prs[q] for q in small], precision="c64", pml_C=ws[0].pml_C)
    flat = np.zeros(Bs.N * nrhs, dtype=np.complex128)
    Bs.solve(Bs.pack([fs[q] for q in small]), flat, tol=1e-5, k=20, maxit=400)
    for i, q in enumerate(small):
        P = single(prs[q], precision="c64", pml_C=ws[0].pml_C)
        u = np.zeros_like(fs[q])
        P.solve(fs[q], u, tol=1e-5, k=20, maxit=400)
        assert np.array_equal(Bs.unpack(flat, nrhs)[i], u)
