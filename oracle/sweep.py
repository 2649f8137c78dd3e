"""The moving-PML sweeping preconditioner: Algs. 1.3, 1.4 and 1.5.

Oracle module (test infrastructure only).

* Alg. 1.4 (setup): S_0 := J_{0,0} is factored, then H_i is formed for every
  later panel by prefixing PML to J_{i,i} and factored (multifrontal, §2.2).
* Alg. 1.3 (T_i): extend u_i by zero over the artificial PML, solve with H_i,
  keep the entries of the panel's own planes.
* Alg. 1.5 (apply): for i = 0..m-2:  u_i := T_i u_i ; u_{i+1} -= J_{i+1,i} u_i ;
  then u_{m-1} := T_{m-1} u_{m-1}; then for i = m-2..0: u_i -= T_i (J_{i+1,i}^T u_{i+1}).

Vectors are arrays of shape (N,) or (nrhs, N) in the global ordering.
"""
from __future__ import annotations

import numpy as np

from . import multifrontal as mf
from .discretize import Helmholtz, operator_J
from .panels import aux_problem, panel_plan
from .symbolic import nested_dissection


class SweepingPreconditioner:
    def __init__(self, prob: Helmholtz, panel_depth: int, pad: int | None = None, leaf: int = 64,
                 mode: str = "moving", panels=None):
        """Alg. 1.4.  ``panels`` restricts setup to a subset of panel indices (sampling)."""
        self.p = prob
        self.pad = prob.gamma if pad is None else pad
        self.leaf = leaf
        self.mode = mode
        self.plan = panel_plan(prob.nz, prob.gamma, panel_depth)
        self.m = len(self.plan)
        self.plane = prob.nx * prob.ny
        self.J = operator_J(prob)
        self.aux = {}
        self.sym = {}
        self.fronts = {}
        sym_cache = {}
        for i in (range(self.m) if panels is None else panels):
            z0, z1 = self.plan[i]
            ap = aux_problem(prob, z0, z1, self.pad, mode)
            key = (ap.nx, ap.ny, ap.depth)
            if key not in sym_cache:
                sym_cache[key] = nested_dissection(ap.nx, ap.ny, ap.depth, leaf)
            self.aux[i] = ap
            self.sym[i] = sym_cache[key]
            self.fronts[i] = mf.factor(ap.H, self.sym[i])

    def panel_slice(self, i):
        z0, z1 = self.plan[i]
        return slice(z0 * self.plane, z1 * self.plane)

    def T(self, i, v):
        """Alg. 1.3 on panel i; ``v`` has shape (n_panel,) or (n_panel, nrhs)."""
        ap = self.aux[i]
        v = np.asarray(v, dtype=np.complex128)
        off = ap.lead * self.plane
        hat_u = np.zeros((off + v.shape[0],) + v.shape[1:], dtype=np.complex128)
        hat_u[off:] = v                                      # extension by zero over the pad
        hat_v = mf.solve(self.fronts[i], self.sym[i], hat_u)  # H_i^{-1} hat_u
        return hat_v[off:]                                   # the panel's own planes

    def coupling(self, i):
        """J_{i+1,i}: rows on panel i+1, columns on panel i (sparse block of J)."""
        return self.J[self.panel_slice(i + 1)][:, self.panel_slice(i)]

    def apply(self, r):
        """Alg. 1.5: returns M^{-1} r for r of shape (N,) or (nrhs, N)."""
        r = np.asarray(r, dtype=np.complex128)
        vec = r.ndim == 1
        u = (r[None, :] if vec else r).T.copy()   # (N, nrhs)
        m = self.m
        for i in range(m - 1):
            si, sn = self.panel_slice(i), self.panel_slice(i + 1)
            u[si] = self.T(i, u[si])
            u[sn] -= self.coupling(i) @ u[si]
        sl = self.panel_slice(m - 1)
        u[sl] = self.T(m - 1, u[sl])
        for i in range(m - 2, -1, -1):
            si, sn = self.panel_slice(i), self.panel_slice(i + 1)
            u[si] -= self.T(i, self.coupling(i).T @ u[sn])
        return u[:, 0] if vec else u.T
