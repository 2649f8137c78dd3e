"""Pins of the oracle's nested dissection (§2.1 and its separator-tree figure)."""
import os

import numpy as np
import pytest

from oracle import symbolic as sy

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig3_separator_tree.txt")


def _load_fig3():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            i, par, kind, cx, cy = line.split()
            rows.append((int(i), int(par), kind, float(cx), float(cy)))
    return rows


def test_reproduces_separator_tree_figure():
    # a square quasi-2D box dissected four times gives the paper's 31-supernode tree, same numbers
    W = 31
    sym = sy.nested_dissection(W, W, 1, leaf=60)
    fig = _load_fig3()
    assert len(sym.supernodes) == len(fig) == 31
    for (i, par, kind, cx, cy), sn in zip(fig, sym.supernodes):
        assert sn.parent == par, i
        x0, x1, y0, y1 = sn.box
        if kind == "L":
            assert not sn.children
            bx, by = (x0 + x1) / 2 / W, (y0 + y1) / 2 / W
        else:
            xs = sn.nodes % W
            ys = sn.nodes // W
            assert (len(np.unique(xs)) == 1) == (kind == "V"), i
            assert (len(np.unique(ys)) == 1) == (kind == "H"), i
            bx, by = (xs.mean() + 0.5) / W, (ys.mean() + 0.5) / W
        assert abs(bx - cx) < 0.03 and abs(by - cy) < 0.03, (i, bx, by, cx, cy)


@pytest.mark.parametrize("nx,ny,nz,leaf", [(9, 7, 3, 12), (12, 12, 4, 64), (5, 11, 2, 8), (1, 1, 5, 2)])
def test_bijection_postorder_and_sizes(nx, ny, nz, leaf):
    sym = sy.nested_dissection(nx, ny, nz, leaf)
    N = nx * ny * nz
    assert sorted(sym.order.tolist()) == list(range(N))
    assert sum(len(sn.nodes) for sn in sym.supernodes) == N
    for f, sn in enumerate(sym.supernodes):
        for c in sn.children:
            assert c < f and sym.supernodes[c].parent == f
    assert sum(1 for sn in sym.supernodes if sn.parent < 0) == 1


def _brute_force_structs(nx, ny, nz, order):
    """Symbolic Gaussian elimination of the 7-point graph in the given order."""
    N = nx * ny * nz
    adj = [set() for _ in range(N)]
    for v in range(N):
        x, y, z = v % nx, (v // nx) % ny, v // (nx * ny)
        for dx, dy, dz in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
            xx, yy, zz = x + dx, y + dy, z + dz
            if xx < nx and yy < ny and zz < nz:
                w = xx + nx * yy + nx * ny * zz
                adj[v].add(w)
                adj[w].add(v)
    done = np.zeros(N, dtype=bool)
    col = {}
    for v in order:
        nb = {w for w in adj[v] if not done[w]}
        col[v] = nb
        for a in nb:
            adj[a] |= nb - {a}
        done[v] = True
    return col


@pytest.mark.parametrize("nx,ny,nz,leaf", [(12, 12, 3, 20), (10, 7, 4, 30), (6, 12, 2, 6)])
def test_struct_matches_symbolic_elimination(nx, ny, nz, leaf):
    sym = sy.nested_dissection(nx, ny, nz, leaf)
    col = _brute_force_structs(nx, ny, nz, sym.order)
    for sn in sym.supernodes:
        S = set(sn.nodes.tolist())
        fill = set()
        for v in sn.nodes:
            fill |= col[int(v)]
        fill -= S
        expect = sorted(fill, key=lambda v: sym.elim[v])
        assert sn.struct.tolist() == expect
        # supernodal: every column of S below the diagonal block has the same structure
        for v in sn.nodes:
            assert col[int(v)] - S <= fill


def test_no_cut_across_the_shallow_direction():
    # §2.1: separators span every plane of the quasi-2D box
    nz = 5
    sym = sy.nested_dissection(16, 16, nz, 40)
    for sn in sym.supernodes:
        if sn.children:
            z = sn.nodes // 256
            assert len(np.unique(z)) == nz
