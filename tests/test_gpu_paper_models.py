"""The paper's four analytic velocity models and four forcing functions (§3) through the C ABI.

Each model with the paper's settings (gamma 5, four planes per panel, damping 7, its tabulated PML
amplitude, ten points per shortest wavelength) on 24^3: GMRES(20) iteration counts of the GPU
path equal the oracle's within one for the single shot and the Gaussian beam, and all four
forcing functions solved as one block reach a true relative residual of 1e-5 (complex128 and
complex64 fronts).
"""
import numpy as np
import pytest

from oracle import discretize as dz
from oracle import gmres as ogm
from oracle import sweep as osw
from paper_1204_0111_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1204_0111_gb300 import psp  # noqa: E402

N_SIDE = 24


@pytest.mark.parametrize("model", list(wl.PAPER_MODELS))
def test_paper_model_iterations_and_four_forcings(model):
    w = wl.cube_paper(model, N_SIDE)
    p = dz.Helmholtz(w.c, w.h, w.omega, w.gamma, w.pml_C, w.alpha)
    A = dz.operator_A(p)
    scale = dz.rhs_scale(p)
    F = w.rhs()
    O = osw.SweepingPreconditioner(p, w.panel_depth, w.pad, w.leaf)
    c = torch.from_numpy(w.c).cuda()
    P = psp.SweepingPreconditioner(c, w.h, w.omega, w.gamma, w.panel_depth, pad=w.pad, leaf=w.leaf,
                                   pml_C=w.pml_C, alpha=w.alpha)
    for j in (0, 2):   # one shot; Gaussian beam (complex forcing)
        _, it_oracle, _ = ogm.gmres(lambda v: A @ v, O.apply, scale * F[j], tol=1e-5, k=20, maxit=300)
        f = F[j:j + 1].copy()
        u = np.zeros_like(f)
        info = P.solve(f, u, tol=1e-5, k=20, maxit=300)
        assert abs(info["iterations"] - it_oracle) <= 1, (model, j, info["iterations"], it_oracle)
    for precision in ("c128", "c64"):
        Q = P if precision == "c128" else psp.SweepingPreconditioner(
            c, w.h, w.omega, w.gamma, w.panel_depth, pad=w.pad, leaf=w.leaf, pml_C=w.pml_C, alpha=w.alpha,
            precision="c64")
        u = np.zeros_like(F)
        info = Q.solve(F.copy(), u, tol=1e-5, k=20, maxit=300)
        assert info["converged"] == 1
        for j in range(4):
            b = scale * F[j]
            assert np.linalg.norm(b - A @ u[j]) / np.linalg.norm(b) < 1e-5, (model, precision, j)
