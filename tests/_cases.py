"""Shared small problem cases for parity tests (inputs only; no method arithmetic)."""
import math

import numpy as np

from paper_1204_0111_gb300 import workloads as wl


def random_velocity(nx, ny, nz, seed, lo=1.0, hi=1.6):
    rng = np.random.default_rng(seed)
    return lo + (hi - lo) * rng.random((nz, ny, nx))


class Case:
    """A problem given by (c, h, omega, gamma, depth, pad, leaf, C, alpha, faces)."""

    def __init__(self, c, h, omega, gamma, depth, pad=None, leaf=64, C=4.0, alpha=2 * math.pi, faces=63, name=""):
        self.c = np.ascontiguousarray(c, dtype=np.float64)
        self.h, self.omega, self.gamma, self.depth = h, omega, gamma, depth
        self.pad = gamma if pad is None else pad
        self.leaf, self.C, self.alpha, self.faces, self.name = leaf, C, alpha, faces, name
        self.nz, self.ny, self.nx = self.c.shape
        self.N = self.c.size

    def oracle_problem(self):
        from oracle import discretize as dz
        return dz.Helmholtz(self.c, self.h, self.omega, self.gamma, self.C, self.alpha, self.faces)


def small_cases():
    out = []
    # the CPU-seconds workload: 20^3, c = 1, gamma 5, 4-plane panels, pad 5 (ragged last panel: 3 planes)
    w = wl.cube_constant(20)
    out.append(Case(w.c, w.h, w.omega, w.gamma, w.panel_depth, w.pad, w.leaf, name="constant20"))
    # non-cubic, heterogeneous, ragged, small leaf (deep trees, many tiles), PML on four faces only
    nx, ny, nz = 13, 9, 17
    h = 1.0 / 14
    out.append(Case(random_velocity(nx, ny, nz, 1), h, 2 * math.pi / (10 * h), 3, 3, pad=4, leaf=16,
                    faces=1 | 2 | 16 | 32, name="ragged13x9x17"))
    # fronts larger than several 64-wide tiles and 32-wide diagonal blocks: 40 x 40 x 6 panel boxes
    n = 40
    h = 1.0 / (n + 1)
    out.append(Case(random_velocity(n, n, 14, 2, 1.0, 1.4), h, 2 * math.pi / (10 * h), 2, 2, pad=4, leaf=64,
                    name="wide40x40x14"))
    return out
