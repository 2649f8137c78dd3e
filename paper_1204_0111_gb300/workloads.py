"""Seeded synthetic workloads: velocity models, sources and frequencies.

Inputs only: this module holds none of the method's arithmetic and is shared
by the GPU binding's callers, the tests and the CPU oracle runs.  The paper
measures on analytic models and on the SEG/EAGE Overthrust model (§3); the
generators below stand in for that family (constant, lens-shaped, layered
and faulted, smooth random, salt body), all seeded.

Grid convention (§1.1): n interior points per axis, h = 1/(n+1), node
(i1, i2, i3) at ((i1+1)h, (i2+1)h, (i3+1)h); arrays are (nz, ny, nx).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def coords(nx, ny, nz, h):
    z, y, x = np.meshgrid((np.arange(nz) + 1) * h, (np.arange(ny) + 1) * h, (np.arange(nx) + 1) * h,
                          indexing="ij")
    return x, y, z


def omega_for_ppw(c_min: float, ppw: float, h: float) -> float:
    """omega giving ``ppw`` points per minimum wavelength 2 pi c_min / omega (§1)."""
    return 2.0 * math.pi * c_min / (ppw * h)


def velocity_constant(nx, ny, nz, h, value=1.0):
    return np.full((nz, ny, nx), float(value))


def velocity_lens(nx, ny, nz, h):
    """Converging lens c = 1 - 0.4 exp(-32 |x - 0.5|^2)."""
    x, y, z = coords(nx, ny, nz, h)
    return 1.0 - 0.4 * np.exp(-32.0 * ((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2))


def velocity_layered_faulted(nx, ny, nz, h, seed=3, n_interfaces=12, n_faults=2):
    """Dipping piecewise-constant layers, c ~ U(1.5, 6), offset by planar faults."""
    rng = np.random.default_rng(seed)
    zbar = np.sort(rng.uniform(0.0, 1.0, n_interfaces))
    dip_a = rng.uniform(-0.15, 0.15, n_interfaces)
    dip_b = rng.uniform(-0.15, 0.15, n_interfaces)
    layer_c = rng.uniform(1.5, 6.0, n_interfaces + 1)
    faults = []
    for _ in range(n_faults):
        nrm = rng.normal(size=3)
        nrm /= np.linalg.norm(nrm)
        pt = rng.uniform(0.2, 0.8, 3)
        shift = rng.uniform(1.0, 10.0) * h
        faults.append((nrm, pt, shift))
    x, y, z = coords(nx, ny, nz, h)
    zz = z.copy()
    for nrm, pt, shift in faults:
        side = (x - pt[0]) * nrm[0] + (y - pt[1]) * nrm[1] + (z - pt[2]) * nrm[2] > 0
        zz = np.where(side, zz - shift, zz)
    layer = np.zeros(x.shape, dtype=np.int64)
    for k in range(n_interfaces):
        layer += (zz > zbar[k] + dip_a[k] * (x - 0.5) + dip_b[k] * (y - 0.5)).astype(np.int64)
    return layer_c[layer]


def velocity_smooth_random(nx, ny, nz, h, seed, corr_len=0.1):
    """c = 2 + 0.5 tanh(g), g an N(0,1) field Gaussian-filtered to ``corr_len``, unit variance."""
    from scipy.ndimage import gaussian_filter
    rng = np.random.default_rng(seed)
    g = gaussian_filter(rng.normal(size=(nz, ny, nx)), sigma=corr_len / h, mode="reflect")
    g = (g - g.mean()) / g.std()
    return 2.0 + 0.5 * np.tanh(g)


def velocity_salt(nx, ny, nz, h):
    """Linear gradient 1.5 -> 4.5 with depth plus a smooth ellipsoidal body at 4.5."""
    x, y, z = coords(nx, ny, nz, h)
    bg = 1.5 + 3.0 * z
    r = np.sqrt(((x - 0.5) / 0.3) ** 2 + ((y - 0.5) / 0.3) ** 2 + ((z - 0.55) / 0.2125) ** 2)
    w = 2.0 * h / 0.2125
    blend = 0.5 * (1.0 + np.tanh(-(r - 1.0) / w))
    return bg + (4.5 - bg) * blend


def gaussian_source(nx, ny, nz, h, center, sigma=None):
    """f = exp(-|x - x0|^2 / (2 sigma^2)), sigma = 2h by default; flat (N,) complex.  Built as the
    outer product of its three 1-D factors (the Gaussian is separable)."""
    sigma = 2.0 * h if sigma is None else sigma
    g = [np.exp(-((np.arange(n) + 1) * h - x0) ** 2 / (2.0 * sigma * sigma)) for n, x0 in zip((nx, ny, nz), center)]
    return (g[2][:, None, None] * (g[1][:, None] * g[0][None, :])[None, :, :]).ravel().astype(np.complex128)


def random_vector(N, nrhs=1, seed=0):
    """Seeded complex Gaussian test vectors, shape (nrhs, N)."""
    rng = np.random.default_rng(seed)
    return (rng.normal(size=(nrhs, N)) + 1j * rng.normal(size=(nrhs, N))).astype(np.complex128)


@dataclass
class Workload:
    name: str
    n: int
    c: np.ndarray
    h: float
    omega: float
    gamma: int
    panel_depth: int
    pad: int
    leaf: int = 64
    pml_C: float = 4.0
    alpha: float = 2.0 * math.pi
    sources: list = field(default_factory=list)
    k: int = 20
    tol: float = 1e-5

    @property
    def N(self):
        return self.n ** 3

    forcing: np.ndarray | None = None

    def rhs(self) -> np.ndarray:
        """(nrhs, N) right-hand sides: the explicit forcing if set, else Gaussian shots."""
        if self.forcing is not None:
            return self.forcing
        return np.stack([gaussian_source(self.n, self.n, self.n, self.h, s) for s in self.sources])


def cube_constant(n=20, gamma=5, panel_depth=4, pad=None, ppw=10.0, leaf=64):
    """Constant c = 1 on n^3, Gaussian shot at the centre (the CPU-seconds case at n = 20)."""
    h = 1.0 / (n + 1)
    c = velocity_constant(n, n, n, h)
    return Workload(f"constant{n}", n, c, h, omega_for_ppw(1.0, ppw, h), gamma, panel_depth,
                    gamma if pad is None else pad, leaf, sources=[(0.5, 0.5, 0.5)])


def cube_lens(n=100, gamma=8, panel_depth=4, pad=None, ppw=10.0, leaf=64):
    """Converging lens on n^3, shot at (0.5, 0.5, 0.1) (the plain-complex128 GPU case at n = 100)."""
    h = 1.0 / (n + 1)
    c = velocity_lens(n, n, n, h)
    return Workload(f"lens{n}", n, c, h, omega_for_ppw(float(c.min()), ppw, h), gamma, panel_depth,
                    gamma if pad is None else pad, leaf, sources=[(0.5, 0.5, 0.1)])


def cube_layered(n=200, gamma=10, panel_depth=4, pad=None, ppw=10.0, leaf=64, seed=3, pml_C=None, alpha=2.0 * math.pi):
    """Layered and faulted model on n^3, shot at (0.5, 0.5, 0.1).  PML amplitude 4 relative to the
    fastest wave speed: pml_C = 4 c_max (see pml_amplitude)."""
    h = 1.0 / (n + 1)
    c = velocity_layered_faulted(n, n, n, h, seed=seed)
    omega = omega_for_ppw(float(c.min()), ppw, h)
    C = pml_amplitude(4.0, float(c.max())) if pml_C is None else pml_C
    return Workload(f"layered{n}", n, c, h, omega, gamma, panel_depth, gamma if pad is None else pad, leaf,
                    pml_C=C, alpha=alpha, sources=[(0.5, 0.5, 0.1)])


def pml_amplitude(C_rel, c_ref):
    """The stretch's amplitude for a PML amplitude C_rel given relative to the wave speed c_ref.

    With s = 1 + i sigma / omega and sigma = (C / eta) t^2, a wave of speed c crossing the layer
    decays by exp(-C / (3 c)): the same C absorbs less where waves are faster.  The amplitudes the
    paper reports (2-4, sec. 3) behave, on its models, like amplitudes relative to the fastest
    propagating speed, so a workload passes C = C_rel * c_ref."""
    return C_rel * c_ref


def top_shots(n, h, gamma, nx_shots, ny_shots, lo=0.2, hi=0.8):
    """Shot positions on an nx_shots x ny_shots grid of (x, y) in [lo, hi]^2, in the first plane
    below the top PML (plane n - gamma - 1, at z = (n - gamma) h)."""
    xs = np.linspace(lo, hi, nx_shots)
    ys = np.linspace(lo, hi, ny_shots)
    z = (n - gamma) * h
    return [(float(x), float(y), z) for y in ys for x in xs]


def cube_smooth(k, gamma=8, panel_depth=4, pad=None, ppw=10.0, leaf=64, base_seed=400):
    """Problem k of the batch of independent problems: n_k = 40 + 8 (k mod 11), smooth random
    velocity (seed base_seed + k), 8 shots on a 4 x 2 grid below the top PML."""
    n = 40 + 8 * (k % 11)
    h = 1.0 / (n + 1)
    c = velocity_smooth_random(n, n, n, h, seed=base_seed + k)
    return Workload(f"smooth{n}_k{k}", n, c, h, omega_for_ppw(float(c.min()), ppw, h), gamma, panel_depth,
                    gamma if pad is None else pad, leaf, pml_C=pml_amplitude(4.0, 2.5),   # c < 2.5
                    sources=top_shots(n, h, gamma, 4, 2))


def cube_salt(n=256, gamma=12, panel_depth=8, pad=8, ppw=8.0, leaf=64, shots=(8, 4)):
    """Salt body in a depth gradient on n^3, 8 points per wavelength, shots on a grid below the top
    PML, GMRES(30)."""
    h = 1.0 / (n + 1)
    c = velocity_salt(n, n, n, h)
    return Workload(f"salt{n}", n, c, h, omega_for_ppw(float(c.min()), ppw, h), gamma, panel_depth,
                    gamma if pad is None else pad, leaf, pml_C=pml_amplitude(4.0, float(c.max())),
                    sources=top_shots(n, h, gamma, *shots), k=30)


# ---------------------------------------------------------------------------------------------
# The paper's analytic models and forcing functions (§3), on the unit cube, any n
# ---------------------------------------------------------------------------------------------
def velocity_barrier(nx, ny, nz, h, high=1e10):
    """c = 1 with a slab x1 in [0, 1], x2 in [0.25, 0.3], x3 in [0, 0.75] at c = 1e10."""
    x, y, z = coords(nx, ny, nz, h)
    slab = (y >= 0.25) & (y <= 0.3) & (z <= 0.75)
    return np.where(slab, high, 1.0)


def velocity_wedge(nx, ny, nz, h):
    """c = 2 below x3 = 0.4 + 0.1 x2, else 1.5 below x3 = 0.8 - 0.2 x2, else 3."""
    x, y, z = coords(nx, ny, nz, h)
    return np.where(z <= 0.4 + 0.1 * y, 2.0, np.where(z <= 0.8 - 0.2 * y, 1.5, 3.0))


def velocity_two_layer(nx, ny, nz, h):
    """c = 4 for x2 < 0.5, else 1."""
    x, y, z = coords(nx, ny, nz, h)
    return np.where(y < 0.5, 4.0, 1.0)


def velocity_waveguide(nx, ny, nz, h):
    """c = 1.25 (1 - 0.4 exp(-32 ((x1 - 0.5)^2 + (x2 - 0.5)^2)))."""
    x, y, z = coords(nx, ny, nz, h)
    return 1.25 * (1.0 - 0.4 * np.exp(-32.0 * ((x - 0.5) ** 2 + (y - 0.5) ** 2)))


PAPER_SHOTS = ((0.5, 0.5, 0.1), (0.25, 0.25, 0.1), (0.75, 0.75, 0.5))   # x0, x1, x2 of §3
PAPER_DIRECTION = (1.0 / math.sqrt(3.0), 1.0 / math.sqrt(3.0), -1.0 / math.sqrt(3.0))


def paper_forcing(n, h, omega):
    """The four right-hand sides of §3 on an n^3 grid, shape (4, N) complex:
    f0 one shot n exp(-10 n |x - x0|^2); f1 the shots at x0, x1, x2 summed; f2 a Gaussian beam
    exp(i omega x.d) exp(-4 omega |x - x2|^2); f3 a plane wave exp(i omega x.d)."""
    x, y, z = coords(n, n, n, h)
    shot = [n * np.exp(-10.0 * n * ((x - p[0]) ** 2 + (y - p[1]) ** 2 + (z - p[2]) ** 2)) for p in PAPER_SHOTS]
    d = PAPER_DIRECTION
    phase = np.exp(1j * omega * (x * d[0] + y * d[1] + z * d[2]))
    x2 = PAPER_SHOTS[2]
    beam = phase * np.exp(-4.0 * omega * ((x - x2[0]) ** 2 + (y - x2[1]) ** 2 + (z - x2[2]) ** 2))
    f = [shot[0], shot[0] + shot[1] + shot[2], beam, phase]
    return np.stack([np.asarray(v, dtype=np.complex128).ravel() for v in f])


# model -> (velocity, PML amplitude of the paper's table, fastest propagating wave speed; the
# barrier's slab at c = 1e10 is an obstacle, not a propagating medium)
PAPER_MODELS = {"barrier": (velocity_barrier, 3.0, 1.0), "wedge": (velocity_wedge, 4.0, 3.0),
                "two_layer": (velocity_two_layer, 4.0, 4.0), "waveguide": (velocity_waveguide, 2.0, 1.25)}


def cube_paper(model, n, gamma=5, panel_depth=4, pad=None, ppw=10.0, leaf=64, alpha=7.0):
    """One of the paper's analytic models on n^3 with its settings (§3): gamma = 5 PML points,
    4 planes per panel, damping 7, the tabulated PML amplitude (relative to the fastest propagating
    speed, see pml_amplitude), 10 points per shortest wavelength; rhs() gives its four forcing
    functions."""
    vel, C, c_ref = PAPER_MODELS[model]
    h = 1.0 / (n + 1)
    c = vel(n, n, n, h)
    omega = omega_for_ppw(float(c.min()), ppw, h)
    w = Workload(f"{model}{n}", n, c, h, omega, gamma, panel_depth, gamma if pad is None else pad, leaf,
                 pml_C=pml_amplitude(C, c_ref), alpha=alpha)
    w.forcing = paper_forcing(n, h, omega)
    return w
