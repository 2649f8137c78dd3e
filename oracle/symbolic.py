"""Supernodal nested-dissection elimination tree of a quasi-2D box.

Oracle module (test infrastructure only).  Follows §2.1 and its
separator-tree figure (Fig. 3): separators are cut across x1 and x2 only,
never across the shallow x3 direction; supernodes are numbered in postorder.

Reading of the dissection rule (the paper gives only the figure):

* A box [x0, x1) x [y0, y1) x (all planes) with wx * wy * depth <= leaf is a
  leaf supernode.
* Otherwise the longer side is cut (a tie cuts x) at mid = x0 + wx // 2
  (resp. y0 + wy // 2); the separator is that whole-depth plane; the children
  are the two remaining boxes, empty ones skipped.
* Postorder: lower-coordinate child subtree, higher-coordinate child subtree,
  separator.  Inside a supernode nodes run x fastest, then y, then z.
* struct(S) is every node outside the subtree of S that is a stencil
  neighbour of a node inside it, sorted by elimination index; the front's row
  order is S followed by struct(S).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Supernode:
    box: tuple            # (x0, x1, y0, y1) of the subtree's region
    nodes: np.ndarray     # local node ids, internal order
    children: list
    parent: int = -1
    struct: np.ndarray = field(default_factory=lambda: np.zeros(0, dtype=np.int64))
    first: int = 0        # elimination index of nodes[0]
    subtree_first: int = 0  # first elimination index of the subtree


@dataclass
class Symbolic:
    nx: int
    ny: int
    nz: int
    leaf: int
    supernodes: list      # postorder
    elim: np.ndarray      # node id -> elimination index
    order: np.ndarray     # elimination index -> node id

    @property
    def N(self):
        return self.nx * self.ny * self.nz


def _box_nodes(nx, ny, nz, x0, x1, y0, y1):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(y0, y1), np.arange(x0, x1), indexing="ij")
    return (x + nx * y + nx * ny * z).ravel().astype(np.int64)


def nested_dissection(nx: int, ny: int, nz: int, leaf: int) -> Symbolic:
    sns: list = []

    def rec(x0, x1, y0, y1):
        wx, wy = x1 - x0, y1 - y0
        if wx <= 0 or wy <= 0:
            return None
        if wx * wy * nz <= leaf:
            sns.append(Supernode((x0, x1, y0, y1), _box_nodes(nx, ny, nz, x0, x1, y0, y1), []))
            return len(sns) - 1
        if wx >= wy:
            mid = x0 + wx // 2
            kids = [rec(x0, mid, y0, y1), rec(mid + 1, x1, y0, y1)]
            sep = _box_nodes(nx, ny, nz, mid, mid + 1, y0, y1)
        else:
            mid = y0 + wy // 2
            kids = [rec(x0, x1, y0, mid), rec(x0, x1, mid + 1, y1)]
            sep = _box_nodes(nx, ny, nz, x0, x1, mid, mid + 1)
        kids = [k for k in kids if k is not None]
        sns.append(Supernode((x0, x1, y0, y1), sep, kids))
        me = len(sns) - 1
        for k in kids:
            sns[k].parent = me
        return me

    rec(0, nx, 0, ny)

    order = np.concatenate([sn.nodes for sn in sns])
    N = nx * ny * nz
    elim = np.empty(N, dtype=np.int64)
    elim[order] = np.arange(N)
    pos = 0
    for sn in sns:
        sn.first = pos
        pos += len(sn.nodes)
    # subtree ranges: postorder makes every subtree contiguous in elimination order
    for f, sn in enumerate(sns):
        lo = sn.first
        stack = list(sn.children)
        while stack:
            c = stack.pop()
            lo = min(lo, sns[c].first)
            stack.extend(sns[c].children)
        sn.subtree_first = lo

    # struct(S) = stencil neighbours of the subtree that lie outside it
    for sn in sns:
        lo, hi = sn.subtree_first, sn.first + len(sn.nodes)   # subtree = elim range [lo, hi)
        sub = order[lo:hi]
        x = sub % nx
        y = (sub // nx) % ny
        z = sub // (nx * ny)
        nbrs = []
        for dx, dy, dz in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
            xx, yy, zz = x + dx, y + dy, z + dz
            ok = (xx >= 0) & (xx < nx) & (yy >= 0) & (yy < ny) & (zz >= 0) & (zz < nz)
            nbrs.append((xx + nx * yy + nx * ny * zz)[ok])
        nb = np.unique(np.concatenate(nbrs))
        e = elim[nb]
        outside = (e < lo) | (e >= hi)
        e = np.sort(e[outside])
        sn.struct = order[e]
    return Symbolic(nx, ny, nz, leaf, sns, elim, order)
