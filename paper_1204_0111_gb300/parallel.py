"""Panels spread over several GPUs: a cost-balanced partition and the pipelined sweep.

The panel factorisations of Alg. 1.4 are independent (§2), so each rank factors one contiguous
block of panels with no exchange (a handle made with ``panels=(begin, count)``).  The application,
Alg. 1.5, is a chain of panel solves (§2: the subdomain solves run in sequence): rank r runs the
forward half over its block, hands the block's last plane to rank r + 1, and later, in the backward
half, hands its block's first plane to rank r - 1.  One plane of nx * ny * nrhs values crosses each
block boundary in each direction; nothing else is exchanged.  With many right-hand sides the
columns are cut into groups so that the ranks work on different groups at the same time.

This module only orders the calls and moves the planes (``torch.distributed`` point-to-point:
NCCL between GPUs, gloo on the CPU); the arithmetic runs in each rank's ``part``.
"""
from __future__ import annotations


def partition(costs, world):
    """Split panels 0..m-1 into ``world`` contiguous non-empty blocks minimising the largest block
    cost (the slowest rank's setup).  Returns [(begin, count), ...] in rank order."""
    m = len(costs)
    if world < 1 or m < world:
        raise ValueError(f"cannot split {m} panels over {world} ranks")
    pre = [0.0]
    for c in costs:
        if c < 0:
            raise ValueError("negative panel cost")
        pre.append(pre[-1] + float(c))
    inf = float("inf")
    # best[k][i]: smallest possible largest cost of splitting panels [0, i) into k blocks
    best = [[inf] * (m + 1) for _ in range(world + 1)]
    cut = [[0] * (m + 1) for _ in range(world + 1)]
    best[0][0] = 0.0
    for k in range(1, world + 1):
        for i in range(k, m - (world - k) + 1):
            for j in range(k - 1, i):
                v = max(best[k - 1][j], pre[i] - pre[j])
                if v < best[k][i]:
                    best[k][i] = v
                    cut[k][i] = j
    bounds, i = [], m
    for k in range(world, 0, -1):
        j = cut[k][i]
        bounds.append((j, i - j))
        i = j
    return bounds[::-1]


class PipelinedSweep:
    """Alg. 1.5 over panel blocks on ``world`` ranks.

    plan     [(z0, z1), ...] of all m panels (psp_plan_panels)
    blocks   [(begin, count), ...] of every rank (partition)
    part     this rank's block: forward(u) and backward(u) in place on a (nrhs, N) block of global
             vectors (psp_sweep_part on a handle made with panels=blocks[rank])
    plane    nx * ny
    comm     object with send(tensor, dst) and recv(tensor, src) (default: torch.distributed)
    """

    def __init__(self, plan, blocks, rank, part, plane, comm=None):
        self.plan, self.blocks, self.rank, self.part, self.plane = plan, blocks, rank, part, plane
        self.world = len(blocks)
        b, n = blocks[rank]
        self.begin, self.end = b, b + n
        if comm is None:
            import torch.distributed as dist
            comm = dist
        self.comm = comm

    def _planes(self, z):
        return slice(z * self.plane, (z + 1) * self.plane)

    def apply(self, u, groups=1):
        """u: (nrhs, N) contiguous; on entry it holds the right-hand sides on this block's planes, on
        return the preconditioned vectors there (other planes: hand-off values or untouched)."""
        nrhs = u.shape[0]
        groups = max(1, min(groups, nrhs))
        edges = [nrhs * g // groups for g in range(groups + 1)]
        first = self.plan[self.begin][0]
        last = self.plan[self.end - 1][1]
        # forward half, block by block in rank order; groups pipeline through the ranks
        for g in range(groups):
            ug = u[edges[g]:edges[g + 1]]
            if self.rank > 0:
                buf = ug[:, self._planes(first - 1)].contiguous()
                self.comm.recv(buf, self.rank - 1)
                ug[:, self._planes(first - 1)] = buf
            self.part.forward(ug)
            if self.rank < self.world - 1:
                self.comm.send(ug[:, self._planes(last - 1)].contiguous(), self.rank + 1)
        # backward half, in reverse rank order
        for g in range(groups):
            ug = u[edges[g]:edges[g + 1]]
            if self.rank < self.world - 1:
                buf = ug[:, self._planes(last)].contiguous()
                self.comm.recv(buf, self.rank + 1)
                ug[:, self._planes(last)] = buf
            self.part.backward(ug)
            if self.rank > 0:
                self.comm.send(ug[:, self._planes(first)].contiguous(), self.rank - 1)
        return u


class LibraryPart:
    """A rank's block as a library handle: psp_sweep_part in place (forward 0, backward 1)."""

    def __init__(self, handle):
        self.h = handle

    def forward(self, u):
        self.h.sweep_part(u, 0)

    def backward(self, u):
        self.h.sweep_part(u, 1)
