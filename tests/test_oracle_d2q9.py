"""The paper runs its two-dimensional cases on D2Q9 (Sec. 2.1).  Here they
run on D3Q19 (or D3Q27) with one periodic layer in z: the populations that
differ only in c_z stream to the same cell, their weights add up to the
D2Q9 weights (1/3 + 2/18 = 4/9, 1/18 + 2/36 = 1/9, 1/36), and with u_z = 0
and no z-gradients their equilibria, Guo force terms and SRT relaxation add
up to the D2Q9 ones.  So the layer's populations summed over c_z follow
D2Q9 exactly.  Pinned against a plain D2Q9 BGK scheme with Guo forcing
written out in numpy (the textbook scheme, Krueger et al. Ch. 3 and 6) on a
decaying shear wave under a body force."""
import numpy as np
import pytest

import oracle
from paper_2207_14496_gb300 import inputs

C9 = np.array([(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1), (1, -1), (-1, 1)])
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def _feq(rho, ux, uy):
    cu = 3.0 * (C9[:, 0, None, None] * ux + C9[:, 1, None, None] * uy)
    usq = 1.5 * (ux * ux + uy * uy)
    return W9[:, None, None] * rho * (1.0 + cu + 0.5 * cu * cu - usq)


def _d2q9_run(ux0, omega, g, steps):
    """Post-collision populations after `steps` pull steps of BGK with Guo
    forcing F = rho g on a periodic grid; starts from f* = f^eq(1, u0)."""
    ny, nx = ux0.shape
    f = _feq(np.ones((ny, nx)), ux0, np.zeros((ny, nx)))
    for _ in range(steps):
        fin = np.empty_like(f)
        for i, (cx, cy) in enumerate(C9):
            fin[i] = np.roll(np.roll(f[i], cy, axis=0), cx, axis=1)
        rho = fin.sum(axis=0)
        Fx, Fy = rho * g[0], rho * g[1]
        ux = ((fin * C9[:, 0, None, None]).sum(axis=0) + 0.5 * Fx) / rho
        uy = ((fin * C9[:, 1, None, None]).sum(axis=0) + 0.5 * Fy) / rho
        feq = _feq(rho, ux, uy)
        cx = C9[:, 0, None, None]
        cy = C9[:, 1, None, None]
        cu = cx * ux + cy * uy
        force = W9[:, None, None] * (1.0 - 0.5 * omega) * (
            3.0 * ((cx - ux) * Fx + (cy - uy) * Fy) + 9.0 * cu * (cx * Fx + cy * Fy))
        f = fin - omega * (fin - feq) + force
    return f


@pytest.mark.parametrize("q", [19, 27])
def test_one_periodic_layer_is_d2q9(q):
    nx, ny, steps = 12, 10, 60
    nu = 0.02
    omega = 1.0 / (3.0 * nu + 0.5)
    g = (2e-5, -1e-5, 0.0)
    params = inputs._base(q=q, collision="srt", refill="eq", shape=(nx, ny, 1),
                          periodic=(True, True, True), nu=nu, g=g)
    y = np.arange(ny) + 0.5
    ux0 = np.broadcast_to((0.01 * np.sin(2 * np.pi * y / ny))[:, None], (ny, nx)).copy()
    o = oracle.Oracle(params)
    u0 = np.zeros((1, ny, nx, 3))
    u0[0, :, :, 0] = ux0
    o.init_fill(np.ones((1, ny, nx)), u0=u0)
    o.step(steps)
    f3 = o.pdfs()[:, 0]
    cx, cy = o.lattice()[0][:, 0], o.lattice()[0][:, 1]
    proj = np.zeros((9, ny, nx))
    for i in range(q):
        k = [j for j, c in enumerate(C9) if c[0] == cx[i] and c[1] == cy[i]][0]
        proj[k] += f3[i]
    ref = _d2q9_run(ux0, omega, g, steps)
    assert np.abs(proj - ref).max() < 1e-14
    # the wave decays and the force accelerates the fluid: the check is not trivial
    assert np.abs(ref - _feq(np.ones((ny, nx)), ux0, np.zeros((ny, nx)))).max() > 1e-4
