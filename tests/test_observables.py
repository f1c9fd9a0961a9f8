"""Host-side observables of the drop impact (Sec. 4.5): cavity depth and crown
inner diameter on the phi = 1/2 contour of the central cross-section,
checked on hand-built fill-level fields with known answers."""
import numpy as np

from paper_2207_14496_gb300.experiments import drop_observables


def _pool(n=96, pool=60):
    z = np.arange(n)[:, None, None] + 0.5
    return z, np.where(z < pool, 1.0, 0.0) * np.ones((n, n, n))


def test_flat_pool_has_no_cavity_and_no_crown():
    _, phi = _pool()
    assert drop_observables(phi, 60.0, 20.0) == (0.0, 0.0)


def test_cylindrical_cavity():
    z, phi = _pool()
    y = np.arange(96)[None, :, None] + 0.5
    # gas cylinder along x, radius 7 around y = 48, from z = 45 up to the surface
    cav = (np.abs(y - 48.0) < 7.0) & (z > 45) & (z < 60)
    h, d = drop_observables(np.where(cav, 0.0, phi), 60.0, 20.0)
    assert abs(h - 15.0 / 20.0) < 1e-12   # bottom crossing halfway between cells 44 and 45
    assert abs(d - 14.0 / 20.0) < 1e-12   # gas cells 41..54, walls halfway to 40 and 55


def test_partial_fill_levels_interpolate():
    z, phi = _pool()
    # the centre column's cell 50 holds 0.25 liquid above full cells: the
    # contour lies a quarter of the way from centre 49.5 to centre 50.5
    phi[50:60, :, :] = 0.0
    phi[50, :, :] = 0.25
    h, _ = drop_observables(phi, 60.0, 20.0)
    assert abs(h - (60.0 - (49.5 + 0.5 / 0.75)) / 20.0) < 1e-12
