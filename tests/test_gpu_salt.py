"""The largest single-GPU workload (salt body in a depth gradient, 32 shots, GMRES(30)), through the C ABI.

At 256^3 the oracle cannot apply the preconditioner, so the checks there hold at any size: the
application is complex symmetric (Alg. 1.5 applies L^{-T} D^{-1} L^{-1} with H_i = H_i^T) and every
shot's solution has a true relative residual below 1e-5, measured on the host with the oracle's own
sparse operator.  The same generator at 128^3 checks, element by element, every front of one
interior panel against the oracle's factorisation (complex64 fronts, tolerance below), and the
complex64 application against the complex128 GPU one.
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

# complex64 fronts (3M products of split TF32 operands, FP32 accumulation) against the complex128
# oracle: relative Frobenius error of each front's G = [inv(L_TL) with D; L_BL inv(L_TL)]
FRONT_TOL_C64 = 1e-3
APPLY_TOL_C64 = 1e-4       # one complex64 application against the complex128 one (lens100: 1.9e-6)


def handle(w, precision):
    c = torch.from_numpy(w.c).cuda()
    return psp.SweepingPreconditioner(c, w.h, w.omega, w.gamma, w.panel_depth, pad=w.pad, leaf=w.leaf,
                                      pml_C=w.pml_C, alpha=w.alpha, precision=precision)


def apply_one(P, x):
    xd = torch.from_numpy(x).cuda()
    out = torch.empty_like(xd)
    P.apply(xd, out)
    torch.cuda.synchronize()
    return out


def test_salt256_complex64_symmetric_and_all_32_shots_to_tolerance():
    w = wl.cube_salt(256)
    assert w.k == 30 and len(w.sources) == 32
    P = handle(w, "c64")
    x = wl.random_vector(w.N, 1, seed=71)
    y = wl.random_vector(w.N, 1, seed=72)
    Mx = apply_one(P, x)
    My = apply_one(P, y)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    a = (yd * Mx).sum().item()
    b = (xd * My).sum().item()
    del Mx, My, xd, yd
    assert abs(a - b) / abs(a) < 1e-4
    f = w.rhs()
    fd = torch.from_numpy(f).cuda()
    ud = torch.zeros_like(fd)
    info = P.solve(fd, ud, tol=w.tol, k=w.k, maxit=400)
    P.close()
    assert info["converged"] == 1 and info["relres_max"] < w.tol
    u = ud.cpu().numpy()
    del fd, ud
    torch.cuda.empty_cache()
    p = dz.Helmholtz(w.c, w.h, w.omega, w.gamma, w.pml_C, w.alpha)
    A = dz.operator_A(p)
    scale = dz.rhs_scale(p)
    worst = 0.0
    for j in range(f.shape[0]):
        bj = scale * f[j]
        worst = max(worst, np.linalg.norm(bj - A @ u[j]) / np.linalg.norm(bj))
    assert worst < w.tol, worst


def test_salt128_fronts_of_one_panel_match_oracle_and_complex64_apply():
    w = wl.cube_salt(128)
    P64 = handle(w, "c64")
    p = dz.Helmholtz(w.c, w.h, w.omega, w.gamma, w.pml_C, w.alpha)
    plan = opn.panel_plan(p.nz, p.gamma, w.panel_depth)
    i = len(plan) // 2                       # an interior panel crossing the salt body
    z0, z1 = plan[i]
    ap = opn.aux_problem(p, z0, z1, w.pad)
    sym = osy.nested_dissection(ap.nx, ap.ny, ap.depth, w.leaf)
    fronts = omf.factor(ap.H, sym)
    worst = 0.0
    for f, fr in enumerate(fronts):
        G, s, u = P64.export_front(i, f)
        Linv = sla.solve_triangular(fr.L_TL, np.eye(s), lower=True, unit_diagonal=True)
        exp = np.vstack([np.tril(Linv, -1) + np.diag(fr.d), fr.L_BL @ Linv])
        got = G.copy()
        got[:s] = np.tril(got[:s])
        worst = max(worst, np.linalg.norm(got - exp) / np.linalg.norm(exp))
    assert worst < FRONT_TOL_C64, worst
    x = wl.random_vector(w.N, 2, seed=81)
    got = apply_one(P64, x).cpu().numpy()
    P64.close()
    P128 = handle(w, "c128")
    ref = apply_one(P128, x).cpu().numpy()
    P128.close()
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < APPLY_TOL_C64, err
