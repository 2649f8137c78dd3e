"""Selective-inversion variants (§2.2) through the C ABI against the oracle.

After the partial LDL^T of a front, F_TL = L_TL D L_TL^T and L_BL = F_BL L_TL^{-T} D^{-1}.  The
handle keeps, per front, G = [inv(L_TL); L_BL inv(L_TL)] (extended, the default), the paper's
G = [inv(L_TL); L_BL], or G = [L_TL; L_BL] without inversion, D on the top block's diagonal, or the
paper's G with a second inverse of L_TL built row by row for the down sweep (§2.2's two inverses).
All four apply the same preconditioner: the sweep takes one pass per front and direction for the
first, two dependent phases for the second and fourth, and triangular substitution for the third.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from paper_1204_0111_gb300 import parallel as par
from paper_1204_0111_gb300 import workloads as wl

from _cases import small_cases

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1204_0111_gb300 import psp  # noqa: E402

CASES = small_cases()
MODES = ["paper", "none", "two"]
_oracles = {}


def oracle_for(case):
    from oracle import sweep as osw
    if case.name not in _oracles:
        _oracles[case.name] = osw.SweepingPreconditioner(case.oracle_problem(), case.depth, case.pad, case.leaf)
    return _oracles[case.name]


def gpu_for(case, si, precision="c128", **kw):
    c = torch.from_numpy(case.c).cuda()
    return psp.SweepingPreconditioner(c, case.h, case.omega, case.gamma, case.depth, pad=case.pad, leaf=case.leaf,
                                      pml_C=case.C, alpha=case.alpha, faces=case.faces, precision=precision,
                                      selective_inversion=si, **kw)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("si", MODES)
@pytest.mark.parametrize("case", CASES, ids=lambda c: c.name)
def test_front_factors_in_each_form(case, si):
    O = oracle_for(case)
    P = gpu_for(case, si)
    worst = 0.0
    for i in range(O.m):
        for f, fr in enumerate(O.fronts[i]):
            G, s, u = P.export_front(i, f)
            if si in ("paper", "two"):
                top = sla.solve_triangular(fr.L_TL, np.eye(s), lower=True, unit_diagonal=True)
            else:
                top = fr.L_TL
            exp = np.vstack([np.tril(top, -1) + np.diag(fr.d), fr.L_BL])
            got = G.copy()
            got[:s] = np.tril(got[:s])
            worst = max(worst, rel(got, exp))
    P.close()
    assert worst < 1e-10, worst


@pytest.mark.parametrize("precision,tol", [("c128", 1e-10), ("c64", 1e-4)])
@pytest.mark.parametrize("case", CASES, ids=lambda c: c.name)
def test_second_inverse_by_rows(case, precision, tol):
    # the two-inverse form keeps a second inverse of L_TL, built row by row (X L_TL = I), besides the
    # first (built column by column): both equal the oracle's inv(L_TL); they are separate
    # computations (their rounding differs somewhere), and the first stays the paper's form's
    O = oracle_for(case)
    P = gpu_for(case, "two", precision=precision)
    Q = gpu_for(case, "paper", precision=precision)
    worst, differ = 0.0, False
    for i in range(O.m):
        for f, fr in enumerate(O.fronts[i]):
            X = P.export_second_inverse(i, f)
            G, s, _ = P.export_front(i, f)
            Gq, _, _ = Q.export_front(i, f)
            assert np.array_equal(G, Gq)
            inv = sla.solve_triangular(fr.L_TL, np.eye(s), lower=True, unit_diagonal=True)
            worst = max(worst, rel(X, inv))
            assert np.array_equal(np.triu(X, 1), np.zeros_like(X)) and np.all(np.diag(X) == 1)
            differ = differ or not np.array_equal(np.tril(X, -1), np.tril(G[:s], -1))
    assert worst < tol, worst
    assert differ
    with pytest.raises(psp.PSPError) as e:
        Q.export_second_inverse(0, 0)
    assert e.value.name == "PSP_ERR_STATE"
    P.close()
    Q.close()


@pytest.mark.parametrize("si", MODES)
@pytest.mark.parametrize("nrhs", [1, 3])
@pytest.mark.parametrize("case", CASES, ids=lambda c: c.name)
def test_apply_matches_oracle_in_each_form(case, si, nrhs):
    O = oracle_for(case)
    P = gpu_for(case, si)
    r = wl.random_vector(case.N, nrhs, seed=17)
    out = torch.empty((nrhs, case.N), dtype=torch.complex128, device="cuda")
    P.apply(torch.from_numpy(r).cuda(), out)
    torch.cuda.synchronize()
    assert rel(out.cpu().numpy(), O.apply(r)) < 1e-10
    P.close()


@pytest.mark.parametrize("si", MODES)
def test_forms_solve_like_the_extended_one(si):
    case = CASES[1]
    f = np.stack([wl.gaussian_source(case.nx, case.ny, case.nz, case.h, s) for s in ((0.5, 0.5, 0.5), (0.3, 0.6, 0.2))])
    E = gpu_for(case, "extended")
    S = gpu_for(case, si)
    ue, us = np.zeros_like(f), np.zeros_like(f)
    ie = E.solve(f, ue, tol=1e-8, k=10, maxit=300)
    is_ = S.solve(f, us, tol=1e-8, k=10, maxit=300)
    assert is_["converged"] == 1 and abs(is_["iterations"] - ie["iterations"]) <= 1
    assert rel(us, ue) < 1e-6
    # the paper's form and no inversion skip the products of L_BL inv(L_TL) (and, without inversion,
    # the inverse itself): less executed setup work for the same algorithmic work
    se = {k: v for k, v in E.stats().items() if not k.startswith("host:")}
    ss = {k: v for k, v in S.stats().items() if not k.startswith("host:")}
    ex = sum(v["extra_flops"] for v in se.values())
    sx = sum(v["extra_flops"] for v in ss.values())
    if si == "two":   # the second inverse costs about what the first does
        assert ss["k_panel_rsolve"]["launches"] > 0 and sx > 0
    else:
        assert sx < ex and (si == "paper" or sx == 0)
    E.close()
    S.close()


@pytest.mark.parametrize("si", MODES)
def test_complex64_forms_against_complex128(si):
    case = CASES[2]
    r = wl.random_vector(case.N, 2, seed=23)
    outs = {}
    for prec in ("c128", "c64"):
        P = gpu_for(case, si, precision=prec, tc_min_dim=32)
        o = torch.empty((2, case.N), dtype=torch.complex128, device="cuda")
        P.apply(torch.from_numpy(r).cuda(), o)
        torch.cuda.synchronize()
        outs[prec] = o.cpu().numpy()
        P.close()
    assert rel(outs["c64"], outs["c128"]) < 1e-4


@pytest.mark.parametrize("si", MODES)
def test_blocks_in_each_form(si):
    w = wl.cube_lens(32, gamma=3, panel_depth=3)
    plan, cost = psp.plan_panels(w.n, w.n, w.n, w.h, w.gamma, w.panel_depth, pad=w.pad, leaf=w.leaf)
    blocks = par.partition(cost, 3)
    c = torch.from_numpy(w.c).cuda()
    kw = dict(pad=w.pad, leaf=w.leaf, pml_C=w.pml_C, alpha=w.alpha, selective_inversion=si)
    full = psp.SweepingPreconditioner(c, w.h, w.omega, w.gamma, w.panel_depth, **kw)
    x = torch.from_numpy(wl.random_vector(w.N, 2, seed=2)).cuda()
    ref = torch.empty_like(x)
    full.apply(x, ref)
    parts = [psp.SweepingPreconditioner(c, w.h, w.omega, w.gamma, w.panel_depth, panels=b, **kw) for b in blocks]
    u = x.clone()
    for P in parts:
        P.sweep_part(u, 0)
    for P in reversed(parts):
        P.sweep_part(u, 1)
    torch.cuda.synchronize()
    assert float(torch.linalg.norm(u - ref) / torch.linalg.norm(ref)) < 1e-13
    for P in parts + [full]:
        P.close()


@pytest.mark.parametrize("precision,ncand", [("c128", 3), ("c64", 7)])
def test_setup_autotuner_keeps_results(precision, ncand):
    # psp_tune_setup re-factors the handle under each form (and tensor-core threshold) and keeps the
    # cheapest for the expected number of applications; the preconditioner stays the same
    case = CASES[2]
    P = gpu_for(case, "extended", precision=precision)
    r = wl.random_vector(case.N, 1, seed=29)
    before = torch.empty((1, case.N), dtype=torch.complex128, device="cuda")
    P.apply(torch.from_numpy(r).cuda(), before)
    t = P.tune_setup(nrhs=1, expected_applies=25)
    assert t["candidates"] == ncand and t["best_total_ms"] <= t["initial_total_ms"]
    assert t["selective_inversion"] in ("extended", "paper", "none")
    after = torch.empty_like(before)
    P.apply(torch.from_numpy(r).cuda(), after)
    torch.cuda.synchronize()
    tol = 1e-10 if precision == "c128" else 1e-4
    assert float(torch.linalg.norm(after - before) / torch.linalg.norm(before)) < tol
    if precision == "c128":
        assert rel(after.cpu().numpy(), oracle_for(case).apply(r)) < 1e-10
    P.close()
