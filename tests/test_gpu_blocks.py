"""Blocks of panels (one GPU's share of a multi-GPU sweep) through the C ABI, on one GPU.

Each block handle factors only its panels (§2: the panel factorisations are independent).  Running
the blocks' forward halves in order and then their backward halves in reverse order (psp_sweep_part)
on one vector block must reproduce psp_apply of a handle holding every panel: on one GPU the blocks
share the vectors, so the planes the ranks would hand over are already in place.  The blocks run
one after another; no kernel waits for another block's kernel.
"""
import numpy as np
import pytest

from paper_1204_0111_gb300 import parallel as par
from paper_1204_0111_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1204_0111_gb300 import psp  # noqa: E402


def make(w, precision, panels=None):
    c = torch.from_numpy(w.c).cuda()
    return psp.SweepingPreconditioner(c, w.h, w.omega, w.gamma, w.panel_depth, pad=w.pad, leaf=w.leaf,
                                      pml_C=w.pml_C, alpha=w.alpha, precision=precision, panels=panels)


@pytest.mark.parametrize("precision,world,nrhs", [("c128", 2, 1), ("c128", 3, 2), ("c64", 3, 3)])
def test_blocks_compose_to_the_full_application(precision, world, nrhs):
    w = wl.cube_lens(40, gamma=4, panel_depth=3)
    plan, cost = psp.plan_panels(w.n, w.n, w.n, w.h, w.gamma, w.panel_depth, pad=w.pad, leaf=w.leaf)
    blocks = par.partition(cost, world)
    full = make(w, precision)
    x = torch.from_numpy(wl.random_vector(w.N, nrhs, seed=13)).cuda()
    ref = torch.empty_like(x)
    full.apply(x, ref)
    parts = [make(w, precision, panels=b) for b in blocks]
    assert sum(P.info()["factor_bytes"] for P in parts) == full.info()["factor_bytes"]
    u = x.clone()
    for P in parts:                      # forward halves, block by block
        P.sweep_part(u, 0)
    for P in reversed(parts):            # backward halves, in reverse order
        P.sweep_part(u, 1)
    torch.cuda.synchronize()
    for P in parts:
        P.check_status()
    err = float(torch.linalg.norm(u - ref) / torch.linalg.norm(ref))
    assert err < 1e-13, err
    # a block handle does not run the whole application, and holds only its own panels' fronts
    with pytest.raises(psp.PSPError) as e:
        parts[1].apply(x, torch.empty_like(x))
    assert e.value.name == "PSP_ERR_STATE"
    with pytest.raises(psp.PSPError) as e:
        parts[1].export_front(blocks[0][0], 0)
    assert e.value.name == "PSP_ERR_ARG"
    G1, _, _ = parts[1].export_front(blocks[1][0], 3)
    G0, _, _ = full.export_front(blocks[1][0], 3)
    assert np.array_equal(G1, G0)
    for P in parts:
        P.close()
    full.close()


def test_block_range_is_checked():
    w = wl.cube_lens(20, gamma=3, panel_depth=3)
    plan, _ = psp.plan_panels(w.n, w.n, w.n, w.h, w.gamma, w.panel_depth, pad=w.pad, leaf=w.leaf)
    with pytest.raises(psp.PSPError) as e:
        make(w, "c128", panels=(len(plan) - 1, 2))
    assert e.value.name == "PSP_ERR_ARG"
