"""Panels spread over ranks (the multi-GPU design), on the CPU: the cost-balanced partition, the
library's host-only panel plan, and the pipelined sweep with gloo ranks.

Each rank's block is factored and solved by the oracle (test side), and the ranks exchange only the
one plane per block boundary and direction that paper_1204_0111_gb300.parallel hands over; the
vectors the ranks hold at the end must equal the single-process oracle application of Alg. 1.5.
"""
import itertools
import os
import socket

import numpy as np
import pytest

from paper_1204_0111_gb300 import parallel as par
from paper_1204_0111_gb300 import workloads as wl

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def test_partition_is_contiguous_and_minimises_the_largest_block():
    rng = np.random.default_rng(0)
    for m, world in ((7, 3), (9, 2), (6, 6), (12, 4)):
        costs = list(rng.uniform(1.0, 5.0, m))
        blocks = par.partition(costs, world)
        assert [b for b, _ in blocks] == [sum(n for _, n in blocks[:r]) for r in range(world)]
        assert sum(n for _, n in blocks) == m and all(n >= 1 for _, n in blocks)
        worst = max(sum(costs[b:b + n]) for b, n in blocks)
        # brute force over every set of cut points
        best = min(max(sum(costs[a:b]) for a, b in zip((0,) + cuts, cuts + (m,)))
                   for cuts in itertools.combinations(range(1, m), world - 1))
        assert worst == pytest.approx(best)
    assert par.partition([1, 1, 1, 1], 2) == [(0, 2), (2, 2)]
    with pytest.raises(ValueError):
        par.partition([1.0, 2.0], 3)


def test_library_panel_plan_matches_the_oracle_on_the_host():
    from oracle import panels as opn
    from paper_1204_0111_gb300 import build as B
    from paper_1204_0111_gb300 import psp
    if not os.path.exists(B.LIB):
        B.build()
    for n, nz, gamma, depth in ((100, 100, 8, 4), (20, 20, 5, 4), (16, 23, 3, 3), (12, 9, 2, 8)):
        plan, cost = psp.plan_panels(n, n, nz, 1.0 / (n + 1), gamma, depth)
        assert plan == opn.panel_plan(nz, gamma, depth)
        assert all(c > 0 for c in cost)
    # deeper auxiliary boxes cost more to factor: panel 0 (gamma + d planes, no pad) vs pad + d
    plan, cost = psp.plan_panels(20, 20, 30, 1 / 21, 6, 3, pad=2)
    assert cost[0] > cost[1] and cost[1] == cost[2]


class OraclePart:
    """One block [b, e) of panels on the oracle (test side): the forward and backward halves of Alg. 1.5."""

    def __init__(self, O, b, e):
        self.O, self.b, self.e = O, b, e

    def forward(self, u):
        a = u.numpy().T                    # (N, nrhs) view of the rank's (nrhs, N) block
        O = self.O
        for i in range(self.b, self.e):
            si = O.panel_slice(i)
            if i > 0:
                a[si] -= O.coupling(i - 1) @ a[O.panel_slice(i - 1)]
            a[si] = O.T(i, a[si])

    def backward(self, u):
        a = u.numpy().T
        O = self.O
        for i in range(min(self.e, O.m - 1) - 1, self.b - 1, -1):
            si, sn = O.panel_slice(i), O.panel_slice(i + 1)
            a[si] -= O.T(i, O.coupling(i).T @ a[sn])


def _case():
    w = wl.cube_lens(14, gamma=2, panel_depth=2)
    return w


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, nrhs, groups, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import discretize as dz
        from oracle import panels as opn
        from oracle import sweep as osw
        w = _case()
        p = dz.Helmholtz(w.c, w.h, w.omega, w.gamma, w.pml_C, w.alpha)
        plan = opn.panel_plan(p.nz, p.gamma, w.panel_depth)
        costs = [(w.pad if z0 > 0 else 0) + z1 - z0 for z0, z1 in plan]   # box depth as the cost proxy
        blocks = par.partition(costs, world)
        b, n = blocks[rank]
        O = osw.SweepingPreconditioner(p, w.panel_depth, w.pad, w.leaf, panels=range(b, b + n))   # own block only
        r = wl.random_vector(w.N, nrhs, seed=5)
        u = torch.zeros((nrhs, w.N), dtype=torch.complex128)
        own = slice(plan[b][0] * w.n * w.n, plan[b + n - 1][1] * w.n * w.n)
        u[:, own] = torch.from_numpy(r[:, own])            # each rank holds only its block's right-hand side
        sweep = par.PipelinedSweep(plan, blocks, rank, OraclePart(O, b, b + n), w.n * w.n)
        sweep.apply(u, groups=groups)
        mine = torch.zeros_like(u)
        mine[:, own] = u[:, own]
        full = torch.view_as_real(mine).contiguous()
        dist.all_reduce(full)                               # gather the blocks (test side)
        out[rank] = (torch.view_as_complex(full).numpy().copy(), blocks)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,nrhs,groups", [(2, 1, 1), (2, 3, 2), (3, 2, 2)])
def test_gloo_ranks_pipelined_sweep_equals_one_process(world, nrhs, groups):
    from oracle import discretize as dz
    from oracle import sweep as osw
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), nrhs, groups, out), nprocs=world, join=True)
        res = dict(out)
    w = _case()
    p = dz.Helmholtz(w.c, w.h, w.omega, w.gamma, w.pml_C, w.alpha)
    ref = osw.SweepingPreconditioner(p, w.panel_depth, w.pad, w.leaf).apply(wl.random_vector(w.N, nrhs, seed=5))
    blocks = res[0][1]
    assert len(blocks) == world and all(n >= 1 for _, n in blocks)
    for rank in range(world):
        got = res[rank][0]
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12, rank
