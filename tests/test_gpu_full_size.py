"""Full-size checks in the configuration bench.py times, through the C ABI.

At these sizes the oracle cannot run a whole preconditioner application, so the checks are:
* fronts of one interior panel factored by the oracle, element by element (complex128, 1e-10);
* properties that hold at any size: the preconditioner is complex symmetric (it applies
  L^{-T} D^{-1} L^{-1}, Alg. 1.5, with H_i = H_i^T), and GMRES reaches a true relative residual of
  1e-5, measured on the host with the oracle's sparse operator;
* complex64 fronts against the complex128 GPU path on the same input (the mixed-precision error of
  one application).
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import discretize as dz
from oracle import multifrontal as omf
from oracle import panels as opn
from oracle import symbolic as osy
from paper_1204_0111_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1204_0111_gb300 import psp  # noqa: E402

_cache = {}


def lens100():
    if "w" not in _cache:
        _cache["w"] = wl.cube_lens(100)
        w = _cache["w"]
        _cache["A"] = dz.operator_A(dz.Helmholtz(w.c, w.h, w.omega, w.gamma, w.pml_C, w.alpha))
    return _cache["w"], _cache["A"]


def handle(w, precision="c128", **kw):
    c = torch.from_numpy(w.c).cuda()
    return psp.SweepingPreconditioner(c, w.h, w.omega, w.gamma, w.panel_depth, pad=w.pad, leaf=w.leaf,
                                      pml_C=w.pml_C, alpha=w.alpha, precision=precision, **kw)


def bilinear_asymmetry(P, N, seed):
    x = wl.random_vector(N, 1, seed=seed)
    y = wl.random_vector(N, 1, seed=seed + 1)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    Mx, My = torch.empty_like(xd), torch.empty_like(yd)
    P.apply(xd, Mx)
    P.apply(yd, My)
    a = (yd * Mx).sum().item()
    b = (xd * My).sum().item()
    return abs(a - b) / abs(a), Mx.cpu().numpy()


def true_residual(A, w, f, u):
    b = dz.rhs_scale(dz.Helmholtz(w.c, w.h, w.omega, w.gamma, w.pml_C, w.alpha))[None, :] * f
    return max(np.linalg.norm(b[j] - A @ u[j]) / np.linalg.norm(b[j]) for j in range(f.shape[0]))


def test_lens100_complex128_fronts_of_one_panel_match_oracle():
    w, _ = lens100()
    P = handle(w)
    p = dz.Helmholtz(w.c, w.h, w.omega, w.gamma, w.pml_C, w.alpha)
    plan = opn.panel_plan(p.nz, p.gamma, w.panel_depth)
    i = len(plan) // 2
    z0, z1 = plan[i]
    ap = opn.aux_problem(p, z0, z1, w.pad)
    sym = osy.nested_dissection(ap.nx, ap.ny, ap.depth, w.leaf)
    fronts = omf.factor(ap.H, sym)
    worst = 0.0
    for f, fr in enumerate(fronts):
        G, s, u = P.export_front(i, f)
        Linv = sla.solve_triangular(fr.L_TL, np.eye(s), lower=True, unit_diagonal=True)
        exp = np.vstack([np.tril(Linv, -1) + np.diag(fr.d), fr.L_BL @ Linv])
        got = G.copy()
        got[:s] = np.tril(got[:s])
        worst = max(worst, np.linalg.norm(got - exp) / np.linalg.norm(exp))
    assert worst < 1e-10, worst


def test_lens100_complex128_apply_symmetric_and_solve_to_tolerance():
    w, A = lens100()
    P = handle(w)
    asym, _ = bilinear_asymmetry(P, w.N, 31)
    assert asym < 1e-10, asym
    f = w.rhs()
    fd = torch.from_numpy(f).cuda()
    ud = torch.zeros_like(fd)
    info = P.solve(fd, ud, tol=w.tol, k=w.k, maxit=400)
    assert info["converged"] == 1
    assert true_residual(A, w, f, ud.cpu().numpy()) < w.tol
    assert 5 <= info["iterations"] <= 40


def test_lens100_complex64_apply_error_and_solve_to_tolerance():
    w, A = lens100()
    P128 = handle(w)
    _, ref = bilinear_asymmetry(P128, w.N, 41)
    P128.close()
    P64 = handle(w, precision="c64")
    asym, got = bilinear_asymmetry(P64, w.N, 41)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < 1e-4, err        # complex64 fronts (tensor-core TF32 splits): measured ~2e-6
    assert asym < 1e-4, asym
    f = w.rhs()
    u = np.zeros_like(f)
    info = P64.solve(f, u, tol=w.tol, k=w.k, maxit=400)
    assert info["converged"] == 1 and true_residual(A, w, f, u) < w.tol


def test_layered30_matches_oracle_iterations():
    # the layered and faulted family where the method still converges quickly: GMRES iteration count
    # equal to the oracle's (+-1), true residual below 1e-5, complex128 and complex64 fronts
    from oracle import gmres as ogm
    from oracle import sweep as osw
    w = wl.cube_layered(30, gamma=5)
    p = dz.Helmholtz(w.c, w.h, w.omega, w.gamma, w.pml_C, w.alpha)
    A = dz.operator_A(p)
    O = osw.SweepingPreconditioner(p, w.panel_depth, w.pad, w.leaf)
    b = dz.rhs_scale(p) * w.rhs()[0]
    _, it_oracle, _ = ogm.gmres(lambda v: A @ v, O.apply, b, tol=w.tol, k=w.k, maxit=300)
    for precision in ("c128", "c64"):
        P = handle(w, precision=precision)
        f = w.rhs()
        u = np.zeros_like(f)
        info = P.solve(f, u, tol=w.tol, k=w.k, maxit=300)
        assert info["converged"] == 1 and true_residual(A, w, f, u) < w.tol
        assert abs(info["iterations"] - it_oracle) <= 1, (precision, info["iterations"], it_oracle)


def test_layered200_complex64_solve_to_tolerance():
    # the 200^3 layered and faulted model, gamma 10, complex64 fronts (116 GB of factors, level
    # groups under the temporary budget), FP64 GMRES(20) to 1e-5; the application is complex
    # symmetric and the solution's true residual is measured with the oracle's operator
    w = wl.cube_layered(200)
    P = handle(w, precision="c64")
    asym, _ = bilinear_asymmetry(P, w.N, 51)
    assert asym < 1e-4, asym
    f = w.rhs()
    fd = torch.from_numpy(f).cuda()
    ud = torch.zeros_like(fd)
    info = P.solve(fd, ud, tol=w.tol, k=w.k, maxit=400)
    assert info["converged"] == 1
    A = dz.operator_A(dz.Helmholtz(w.c, w.h, w.omega, w.gamma, w.pml_C, w.alpha))
    assert true_residual(A, w, f, ud.cpu().numpy()) < w.tol
