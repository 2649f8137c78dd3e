"""Second-order 7-point discretisation of the Helmholtz operators with PML.

Oracle module (test infrastructure only).  Follows the paper's §1 and §1.1:

* Eq. (1.1): the Helmholtz operator  A = -Laplacian - omega^2 / c(x)^2;
* Eq. (1.5): the artificially damped operator J = -Laplacian - (omega + i alpha)^2 / c(x)^2;
* §1.1: n interior points per axis on the unit cube, node (i1, i2, i3) at
  ((i1+1)h, (i2+1)h, (i3+1)h), h = 1/(n+1), global index i1 + i2 n + i3 n^2,
  which makes the matrix block tridiagonal in x3-planes (Eq. (1.2)) and complex
  symmetric, not Hermitian, because of the PML.

Readings of what the paper leaves open (it defers the PML to Engquist and
Ying's PML paper and only names its amplitude "C"):

* Complex stretch s_j(x_j) = 1 + i sigma_j(x_j) / omega with the REAL omega in
  both A and J, so the off-diagonal plane blocks of A and J coincide.
* The operator is used in the divergence form multiplied through by s1 s2 s3:
      -sum_j d_j( a_j d_j u ) - k^2 s1 s2 s3 u,   a_1 = s2 s3 / s1, a_2 = s1 s3 / s2,
      a_3 = s1 s2 / s3,  k^2 = omega^2 / c^2 (A) or (omega + i alpha)^2 / c^2 (J),
  which is symmetric by construction.  The system solved is A_s u = s1 s2 s3 f.
* Finite differences: a_j is evaluated at the half-point between two nodes along
  axis j, with s_j taken at that half-point and the other two stretches at the
  node; every term is divided by h^2.  Nodes outside the grid are zero
  (homogeneous Dirichlet); the wall half-point still enters the diagonal.
* Profile: sigma(xi) = (C / eta) t^2 with eta = gamma h and
  t = max(0, ((gamma + 1) h - dist) / (gamma h)), dist being the distance from
  the point at fractional node coordinate xi to the wall.  The gamma outermost
  nodes get t in [1/gamma, 1]; the half-point next to the wall gets
  (gamma + 1/2) / gamma, which is left unclamped.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

# bit masks of the six faces that carry a PML
FACE_X_LO, FACE_X_HI, FACE_Y_LO, FACE_Y_HI, FACE_Z_LO, FACE_Z_HI = 1, 2, 4, 8, 16, 32
ALL_FACES = 63


@dataclass
class Helmholtz:
    """A heterogeneous Helmholtz problem on an nx x ny x nz interior grid.

    ``c`` has shape (nz, ny, nx) so that its C-order flat index is the
    paper's global index i1 + i2 nx + i3 nx ny.
    """

    c: np.ndarray
    h: float
    omega: float
    gamma: int
    pml_C: float = 4.0
    alpha: float = 2.0 * math.pi
    pml_faces: int = ALL_FACES
    nz: int = field(init=False)
    ny: int = field(init=False)
    nx: int = field(init=False)

    def __post_init__(self):
        self.c = np.asarray(self.c, dtype=np.float64)
        self.nz, self.ny, self.nx = self.c.shape

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz


def pml_sigma(xi, n, gamma, C, h, low=True, high=True):
    """sigma at fractional node coordinates ``xi`` of an axis with n interior nodes.

    Node i sits at xi = i, the walls at xi = -1 and xi = n (§1.1 grid).  The
    distance to the low wall is (xi + 1) h and to the high wall (n - xi) h.
    """
    xi = np.asarray(xi, dtype=np.float64)
    sig = np.zeros_like(xi)
    if gamma <= 0:
        return sig
    eta = gamma * h
    if low:
        dist = (xi + 1.0) * h
        t = np.maximum(0.0, ((gamma + 1) * h - dist) / (gamma * h))
        sig = sig + (C / eta) * t * t
    if high:
        dist = (n - xi) * h
        t = np.maximum(0.0, ((gamma + 1) * h - dist) / (gamma * h))
        sig = sig + (C / eta) * t * t
    return sig


@dataclass
class AxisStretch:
    """Complex stretch of one axis: at its n nodes and its n + 1 half-points.

    ``half[k]`` is the stretch at xi = k - 1/2 (between node k-1 and node k).
    """

    node: np.ndarray
    half: np.ndarray


def stretch_from_sigma(sig_node, sig_half, omega) -> AxisStretch:
    """s = 1 + i sigma / omega (real omega, reading stated in the module header)."""
    return AxisStretch(1.0 + 1j * np.asarray(sig_node) / omega, 1.0 + 1j * np.asarray(sig_half) / omega)


def axis_stretch(n, gamma, C, h, omega, low, high) -> AxisStretch:
    xs = np.arange(n, dtype=np.float64)
    xh = np.arange(n + 1, dtype=np.float64) - 0.5
    return stretch_from_sigma(pml_sigma(xs, n, gamma, C, h, low, high),
                              pml_sigma(xh, n, gamma, C, h, low, high), omega)


def global_stretches(p: Helmholtz):
    f = p.pml_faces
    s1 = axis_stretch(p.nx, p.gamma, p.pml_C, p.h, p.omega, bool(f & FACE_X_LO), bool(f & FACE_X_HI))
    s2 = axis_stretch(p.ny, p.gamma, p.pml_C, p.h, p.omega, bool(f & FACE_Y_LO), bool(f & FACE_Y_HI))
    s3 = axis_stretch(p.nz, p.gamma, p.pml_C, p.h, p.omega, bool(f & FACE_Z_LO), bool(f & FACE_Z_HI))
    return s1, s2, s3


def k2_A(p: Helmholtz) -> np.ndarray:
    """omega^2 / c^2 of Eq. (1.1), as complex."""
    return (p.omega ** 2 / p.c ** 2).astype(np.complex128)


def k2_J(p: Helmholtz) -> np.ndarray:
    """(omega + i alpha)^2 / c^2 of Eq. (1.5)."""
    return ((p.omega + 1j * p.alpha) ** 2) / p.c ** 2


def stencil_operator(h, k2, s1: AxisStretch, s2: AxisStretch, s3: AxisStretch) -> sp.csr_matrix:
    """Symmetric 7-point matrix of -sum_j d_j(a_j d_j .) - k2 s1 s2 s3 on a box.

    ``k2`` has shape (nz, ny, nx); the stretches are the box's own axis tables.
    Unknown (x, y, z) has index x + nx y + nx ny z.
    """
    k2 = np.asarray(k2, dtype=np.complex128)
    nz, ny, nx = k2.shape
    N = nx * ny * nz
    idx = np.arange(N).reshape(nz, ny, nx)
    S1n = s1.node[None, None, :]
    S2n = s2.node[None, :, None]
    S3n = s3.node[:, None, None]
    inv_h2 = 1.0 / (h * h)

    diag = -k2 * (S1n * S2n * S3n)
    rows, cols, vals = [], [], []

    # axis 1: a_1 = s2 s3 / s1(half-point), shape (nz, ny, nx + 1)
    a1 = (S2n * S3n) / s1.half[None, None, :]
    diag = diag + (a1[:, :, :-1] + a1[:, :, 1:]) * inv_h2
    off = -a1[:, :, 1:-1] * inv_h2
    rows.append(idx[:, :, :-1].ravel()); cols.append(idx[:, :, 1:].ravel()); vals.append(off.ravel())

    # axis 2: a_2 = s1 s3 / s2(half-point), shape (nz, ny + 1, nx)
    a2 = (S1n * S3n) / s2.half[None, :, None]
    diag = diag + (a2[:, :-1, :] + a2[:, 1:, :]) * inv_h2
    off = -a2[:, 1:-1, :] * inv_h2
    rows.append(idx[:, :-1, :].ravel()); cols.append(idx[:, 1:, :].ravel()); vals.append(off.ravel())

    # axis 3: a_3 = s1 s2 / s3(half-point), shape (nz + 1, ny, nx)
    a3 = (S1n * S2n) / s3.half[:, None, None]
    diag = diag + (a3[:-1, :, :] + a3[1:, :, :]) * inv_h2
    off = -a3[1:-1, :, :] * inv_h2
    rows.append(idx[:-1, :, :].ravel()); cols.append(idx[1:, :, :].ravel()); vals.append(off.ravel())

    r_off = np.concatenate(rows)
    c_off = np.concatenate(cols)
    v_off = np.concatenate(vals)
    r = np.concatenate([np.arange(N), r_off, c_off])
    c = np.concatenate([np.arange(N), c_off, r_off])
    v = np.concatenate([diag.ravel(), v_off, v_off])
    return sp.coo_matrix((v, (r, c)), shape=(N, N)).tocsr()


def operator_A(p: Helmholtz) -> sp.csr_matrix:
    s1, s2, s3 = global_stretches(p)
    return stencil_operator(p.h, k2_A(p), s1, s2, s3)


def operator_J(p: Helmholtz) -> sp.csr_matrix:
    s1, s2, s3 = global_stretches(p)
    return stencil_operator(p.h, k2_J(p), s1, s2, s3)


def rhs_scale(p: Helmholtz) -> np.ndarray:
    """s1 s2 s3 at every node (flat): the symmetrised system is A_s u = s1 s2 s3 f."""
    s1, s2, s3 = global_stretches(p)
    return (s3.node[:, None, None] * s2.node[None, :, None] * s1.node[None, None, :]).ravel()
