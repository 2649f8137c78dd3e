"""Panels and PML-padded auxiliary problems H_i.

Oracle module (test infrastructure only).  Follows §1.1 of the paper: panels
of O(gamma) contiguous x3-planes, numbered 0..m-1 (Alg. 1.4); S_0 is the
leading diagonal block J_{0,0}; for i >= 1, H_i is J_{i,i} with an artificial
PML prefixed below it (Fig. 2, right), and T_i of Alg. 1.3 reads the panel's
own planes out of H_i^{-1}.

Readings of what the paper leaves open:

* Panel 0 is the planes [0, gamma + d) of J with no pad; panel i >= 1 is the
  next d planes, the last panel taking whatever remains (it contains the top
  physical PML).
* The pad is p virtual planes below the panel.  In the pad, c is copied from
  the panel's first plane (same x1, x2) and the mass term is J's.  The lateral
  stretches are the domain's.  The x3-stretch of the pad follows the module
  ``discretize`` profile with gamma replaced by p, measured from a virtual
  Dirichlet wall one plane below the pad; it vanishes at the panel's first
  plane.  The panel's planes keep their physical x3-stretch.  The far side of
  the panel is cut with a Dirichlet condition.
* "exact" mode (a test device, Fig. 2 middle): H_i is J on ALL planes below the
  panel's top, so T_i is the exact S_i^{-1} of Alg. 1.1.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from .discretize import (FACE_Z_HI, FACE_Z_LO, AxisStretch, Helmholtz, global_stretches, k2_J,
                         pml_sigma, stencil_operator, stretch_from_sigma)


def panel_plan(nz: int, gamma: int, depth: int):
    """[(z0, z1), ...] half-open plane ranges of the m panels."""
    if depth <= 0:
        raise ValueError("panel depth must be positive")
    first = min(gamma + depth, nz)
    plan = [(0, first)]
    z = first
    while z < nz:
        plan.append((z, min(z + depth, nz)))
        z += depth
    return plan


@dataclass
class AuxProblem:
    """One auxiliary problem: the box nx x ny x D with D = lead + (z1 - z0).

    ``lead`` leading planes (pad, or all earlier planes in exact mode) come
    before the panel's planes; ``H`` is its sparse matrix.
    """

    z0: int
    z1: int
    lead: int
    H: sp.csr_matrix
    nx: int
    ny: int

    @property
    def depth(self) -> int:
        return self.lead + self.z1 - self.z0

    @property
    def n_panel(self) -> int:
        return self.nx * self.ny * (self.z1 - self.z0)


def aux_problem(p: Helmholtz, z0: int, z1: int, pad: int, mode: str = "moving") -> AuxProblem:
    s1, s2, s3g = global_stretches(p)
    k2 = k2_J(p)
    if z0 == 0 or mode == "exact":
        # S_0 := J_{0,0} (Alg. 1.4), or the exact auxiliary problem of Fig. 2 (middle)
        zlo = 0
        s3 = AxisStretch(s3g.node[zlo:z1], s3g.half[zlo:z1 + 1])
        H = stencil_operator(p.h, k2[zlo:z1], s1, s2, s3)
        return AuxProblem(z0, z1, z0 - zlo, H, p.nx, p.ny)

    d = z1 - z0
    D = pad + d
    lo = bool(p.pml_faces & FACE_Z_LO)
    hi = bool(p.pml_faces & FACE_Z_HI)
    # node k of the box: pad planes k < pad, panel plane k >= pad is global plane z0 + k - pad
    xi_node = np.arange(D, dtype=np.float64)
    xi_half = np.arange(D + 1, dtype=np.float64) - 0.5
    sig_pad_node = pml_sigma(xi_node, 10 ** 9, pad, p.pml_C, p.h, low=True, high=False)
    sig_pad_half = pml_sigma(xi_half, 10 ** 9, pad, p.pml_C, p.h, low=True, high=False)
    g_node = z0 + xi_node - pad
    g_half = z0 + xi_half - pad
    sig_phys_node = np.where(xi_node >= pad, pml_sigma(g_node, p.nz, p.gamma, p.pml_C, p.h, lo, hi), 0.0)
    sig_phys_half = np.where(xi_half >= pad - 0.5, pml_sigma(g_half, p.nz, p.gamma, p.pml_C, p.h, lo, hi), 0.0)
    s3 = stretch_from_sigma(sig_pad_node + sig_phys_node, sig_pad_half + sig_phys_half, p.omega)

    k2_box = np.empty((D, p.ny, p.nx), dtype=np.complex128)
    k2_box[:pad] = k2[z0][None, :, :]          # c copied from the panel's first plane
    k2_box[pad:] = k2[z0:z1]
    H = stencil_operator(p.h, k2_box, s1, s2, s3)
    return AuxProblem(z0, z1, pad, H, p.nx, p.ny)
