"""The seeded workload generators against the definitions they follow (inputs only; no method
arithmetic): the paper's analytic models and forcing functions (§3) at sample points, the batch
sizes, and the PML amplitude convention."""
import math

import numpy as np

from paper_1204_0111_gb300 import workloads as wl


def _at(field, n, x, y, z):
    """Value of an (nz, ny, nx) field at the grid node nearest to (x, y, z), h = 1/(n+1)."""
    i = [int(round(v * (n + 1))) - 1 for v in (x, y, z)]
    return field[i[2], i[1], i[0]]


def test_paper_velocity_models_at_sample_points():
    n = 39
    h = 1.0 / (n + 1)
    w = wl.velocity_wedge(n, n, n, h)
    assert _at(w, n, 0.5, 0.0 + h, 0.2) == 2.0     # below x3 = 0.4 + 0.1 x2
    assert _at(w, n, 0.5, 0.5, 0.6) == 1.5         # above it, below x3 = 0.8 - 0.2 x2
    assert _at(w, n, 0.5, 0.5, 0.9) == 3.0
    t = wl.velocity_two_layer(n, n, n, h)
    assert _at(t, n, 0.5, 0.25, 0.5) == 4.0 and _at(t, n, 0.5, 0.75, 0.5) == 1.0
    b = wl.velocity_barrier(n, n, n, h)
    assert _at(b, n, 0.5, 0.275, 0.5) == 1e10 and _at(b, n, 0.5, 0.275, 0.9) == 1.0
    assert _at(b, n, 0.5, 0.6, 0.5) == 1.0
    g = wl.velocity_waveguide(n, n, n, h)
    assert abs(_at(g, n, 0.5, 0.5, 0.3) - 1.25 * 0.6) < 1e-12           # the axis
    x, y = 0.5 + 8 * h, 0.5
    assert abs(_at(g, n, x, y, 0.7) - 1.25 * (1 - 0.4 * math.exp(-32 * (8 * h) ** 2))) < 1e-12
    assert np.allclose(g[0], g[-1])                                        # invariant along x3


def test_paper_forcing_functions():
    n = 23
    h = 1.0 / (n + 1)
    omega = 10.0
    F = wl.paper_forcing(n, h, omega)
    assert F.shape == (4, n ** 3)
    f0, f1, f2, f3 = F
    assert np.allclose(np.abs(f3), 1.0)                                    # a plane wave
    x, y, z = (a.ravel() for a in wl.coords(n, n, n, h))
    d = wl.PAPER_DIRECTION
    assert np.allclose(f3, np.exp(1j * omega * (d[0] * x + d[1] * y + d[2] * z)))
    assert abs(np.linalg.norm(d) - 1.0) < 1e-15 and d[2] < 0
    k0 = np.argmax(np.abs(f0))                                             # the shot peaks at x0
    assert np.allclose((x[k0], y[k0], z[k0]), wl.PAPER_SHOTS[0], atol=h)
    assert np.all(np.abs(f1) >= np.abs(f0) - 1e-12)                        # three shots contain it
    k2 = np.argmax(np.abs(f2))                                             # the beam peaks at x2
    assert np.allclose((x[k2], y[k2], z[k2]), wl.PAPER_SHOTS[2], atol=h)


def test_paper_model_settings_and_amplitude_convention():
    w = wl.cube_paper("wedge", 24)
    assert (w.gamma, w.panel_depth, w.pad, w.alpha) == (5, 4, 5, 7.0)
    assert w.pml_C == 4.0 * 3.0                     # the table's amplitude times the fastest speed
    assert abs(w.omega - 2 * math.pi * 1.5 / (10 * w.h)) < 1e-12     # ten points per shortest wavelength
    assert wl.cube_paper("barrier", 24).pml_C == 3.0
    assert wl.pml_amplitude(4.0, 2.5) == 10.0


def test_batch_sizes_and_shots():
    sizes = [wl.cube_smooth(k).n for k in range(16)]
    assert sizes == [40 + 8 * (k % 11) for k in range(16)]
    w = wl.cube_smooth(0)
    assert len(w.sources) == 8 and all(abs(s[2] - (w.n - w.gamma) * w.h) < 1e-15 for s in w.sources)
    assert 1.5 < w.c.min() and w.c.max() < 2.5
