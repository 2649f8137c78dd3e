"""Panels with identical auxiliary problems share one factorisation (§3: a velocity model invariant
along the sweep direction needs only O(1) distinct panel factorisations), through the C ABI.

The waveguide model of §3 does not vary along x3, so every interior panel away from the top and
bottom PML has the same H_i.  Sharing must not change a single bit of the preconditioner: the
applications of a sharing handle equal those of a handle that factors every panel, and both match
the oracle (which factors every panel itself).
"""
import numpy as np
import pytest

from oracle import discretize as dz
from oracle import sweep as osw
from paper_1204_0111_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1204_0111_gb300 import psp  # noqa: E402


def handle(w, **kw):
    c = torch.from_numpy(w.c).cuda()
    return psp.SweepingPreconditioner(c, w.h, w.omega, w.gamma, w.panel_depth, pad=w.pad, leaf=w.leaf,
                                      pml_C=w.pml_C, alpha=w.alpha, **kw)


def apply(P, x):
    xd = torch.from_numpy(x).cuda()
    out = torch.empty_like(xd)
    P.apply(xd, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("precision", ["c128", "c64"])
def test_invariant_model_factors_distinct_panels_once(precision):
    w = wl.cube_paper("waveguide", 40)
    S = handle(w, precision=precision)
    E = handle(w, precision=precision, factor_every_panel=True)
    si, ei = S.info(), E.info()
    assert si["panels"] == ei["panels"] == 9
    # panel 0 (bottom PML), the last two (top PML) and one interior panel for the six identical ones
    assert si["factor_bytes"] < ei["factor_bytes"] and si["fronts"] < ei["fronts"]
    interior = [1, 2, 3, 4, 5, 6]
    for f in (0, 5, 17):
        g0 = S.export_front(interior[0], f)[0]
        for i in interior[1:]:
            assert np.array_equal(S.export_front(i, f)[0], g0)
            assert np.array_equal(E.export_front(i, f)[0], g0)
    x = wl.random_vector(w.N, 2, seed=3)
    assert np.array_equal(apply(S, x), apply(E, x))
    S.close()
    E.close()


def test_shared_factorisations_match_the_oracle():
    w = wl.cube_paper("waveguide", 24)
    S = handle(w)
    E = handle(w, factor_every_panel=True)
    assert S.info()["fronts"] < E.info()["fronts"]
    E.close()
    p = dz.Helmholtz(w.c, w.h, w.omega, w.gamma, w.pml_C, w.alpha)
    O = osw.SweepingPreconditioner(p, w.panel_depth, w.pad, w.leaf)
    x = wl.random_vector(w.N, 1, seed=11)
    got = apply(S, x)
    ref = O.apply(x)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-10
    S.close()


def test_varying_model_shares_nothing():
    w = wl.cube_lens(24, gamma=3, panel_depth=3)
    S = handle(w)
    E = handle(w, factor_every_panel=True)
    assert S.info() == E.info()
    S.close()
    E.close()
