"""Seeded synthetic inputs: initial fill levels, velocities and parameter sets.

This module holds geometry and parameter recipes only -- none of the method's
arithmetic.  Both the CUDA library (through its Python binding) and the CPU
oracle consume what it returns, so each workload is defined exactly once.

Geometry conventions (reading R13):
  * arrays are (nz, ny, nx), x fastest;
  * for the wave, cell i covers x in [i - 1/2, i + 1/2) so that column 0 is
    centred on x = 0, and cell j covers y in [j, j + 1) above the bottom wall;
  * elsewhere cell (i, j, k) covers [i, i+1) x [j, j+1) x [k, k+1);
  * walls are a virtual obstacle layer outside the stated domain size.

The workloads restate the paper's experiments in shape (standing gravity wave,
Sec. 4.1; rectangular dam break, Sec. 4.2; Taylor bubble, Sec. 4.4; drop
impact, Sec. 4.5; bubbly plane Poiseuille flow, Sec. 4.6) at the sizes used
for parity and measurement.
"""
from __future__ import annotations

import math

import numpy as np

REFILL_SCHEMES = ("eq", "eq_neq", "geq", "ext", "avg")


# ----------------------------------------------------------------- geometry
def wave_fill(nx: int, ny: int, nz: int, depth: float, amp: float, wavelength: float,
              perturb=None) -> np.ndarray:
    """Fill level of h(x) = depth + amp cos(2 pi x / wavelength) (+ perturb[i]).

    phi(i, j) is the cell average over x of clamp(h(x) - j, 0, 1), taken with
    64-point Gauss-Legendre quadrature; perturb (length nx, cells) shifts the
    surface of column i uniformly.
    """
    xg, wg = np.polynomial.legendre.leggauss(64)
    k = 2.0 * math.pi / wavelength
    i = np.arange(nx, dtype=np.float64)
    xs = i[:, None] + 0.5 * xg[None, :]                      # (nx, 64)
    h = depth + amp * np.cos(k * xs)
    if perturb is not None:
        h = h + np.asarray(perturb, dtype=np.float64)[:, None]
    j = np.arange(ny, dtype=np.float64)
    frac = np.clip(h[None, :, :] - j[:, None, None], 0.0, 1.0)  # (ny, nx, 64)
    phi2 = 0.5 * np.tensordot(frac, wg, axes=([2], [0]))        # (ny, nx)
    phi2 = np.where(phi2 > 1.0 - 1e-15, 1.0, phi2)
    phi2 = np.where(phi2 < 1e-15, 0.0, phi2)
    return np.ascontiguousarray(np.broadcast_to(phi2, (nz, ny, nx)))


def wave_fill_dperturb(nx: int, ny: int, depth: float, amp: float, wavelength: float,
                       perturb=None) -> np.ndarray:
    """d phi(i, j) / d perturb[i] of wave_fill, shape (ny, nx): the fraction of
    the cell's width (same quadrature) where 0 < h(x) - j < 1."""
    xg, wg = np.polynomial.legendre.leggauss(64)
    k = 2.0 * math.pi / wavelength
    i = np.arange(nx, dtype=np.float64)
    xs = i[:, None] + 0.5 * xg[None, :]
    h = depth + amp * np.cos(k * xs)
    if perturb is not None:
        h = h + np.asarray(perturb, dtype=np.float64)[:, None]
    j = np.arange(ny, dtype=np.float64)
    r = h[None, :, :] - j[:, None, None]
    inside = ((r > 0.0) & (r < 1.0)).astype(np.float64)
    return 0.5 * np.tensordot(inside, wg, axes=([2], [0]))


def box_fill(nx: int, ny: int, nz: int, width: int, height: int) -> np.ndarray:
    """Liquid column occupying cells i < width, j < height (all k)."""
    phi = np.zeros((nz, ny, nx))
    phi[:, :height, :width] = 1.0
    return phi


def sphere_fraction(nx: int, ny: int, nz: int, centre, radius: float, sub: int = 8):
    """Volume fraction of a sphere in each cell, sub^3 samples per cut cell."""
    cx, cy, cz = centre
    frac = np.zeros((nz, ny, nx))
    lo = [max(0, int(math.floor(c - radius)) - 1) for c in (cx, cy, cz)]
    hi = [min(n, int(math.ceil(c + radius)) + 2) for c, n in zip((cx, cy, cz), (nx, ny, nz))]
    ks = np.arange(lo[2], hi[2])
    js = np.arange(lo[1], hi[1])
    is_ = np.arange(lo[0], hi[0])
    K, J, I = np.meshgrid(ks, js, is_, indexing="ij")
    # distance from the cell centre: classify cells entirely in or out
    d = np.sqrt((I + 0.5 - cx) ** 2 + (J + 0.5 - cy) ** 2 + (K + 0.5 - cz) ** 2)
    half_diag = math.sqrt(3.0) / 2.0
    inside = d <= radius - half_diag
    cut = (~inside) & (d < radius + half_diag)
    block = np.where(inside, 1.0, 0.0)
    off = (np.arange(sub) + 0.5) / sub
    ox, oy, oz = np.meshgrid(off, off, off, indexing="ij")
    ox, oy, oz = ox.ravel(), oy.ravel(), oz.ravel()
    kk, jj, ii = np.nonzero(cut)
    for t in range(0, kk.size, 4096):
        k_ = K[kk[t:t + 4096], jj[t:t + 4096], ii[t:t + 4096]][:, None]
        j_ = J[kk[t:t + 4096], jj[t:t + 4096], ii[t:t + 4096]][:, None]
        i_ = I[kk[t:t + 4096], jj[t:t + 4096], ii[t:t + 4096]][:, None]
        r2 = (i_ + ox - cx) ** 2 + (j_ + oy - cy) ** 2 + (k_ + oz - cz) ** 2
        block[kk[t:t + 4096], jj[t:t + 4096], ii[t:t + 4096]] = (r2 <= radius * radius).mean(axis=1)
    frac[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = block
    return frac


def cylinder_fraction(nx: int, ny: int, centre, radius: float, sub: int = 16):
    """Area fraction of a disc in each cell of an nx x ny layer (nz = 1)."""
    cx, cy = centre
    off = (np.arange(sub) + 0.5) / sub
    J, I = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    acc = np.zeros((ny, nx))
    for oy in off:
        for ox in off:
            acc += ((I + ox - cx) ** 2 + (J + oy - cy) ** 2 <= radius * radius)
    return (acc / (sub * sub))[None, :, :]


# ----------------------------------------------------------------- workloads
def _base(**kw):
    p = dict(q=19, collision="srt", magic=3.0 / 16.0, refill="eq", periodic=(True, False, True),
             nu=0.01, g=(0.0, 0.0, 0.0), sigma=0.0, p_v=1.0 / 3.0, eps=1e-2, options=0)
    p.update(kw)
    return p


def standing_wave(L: int = 64, nz: int = 1, depth=None, amp=None, nu: float = 0.01,
                  g: float = 1e-5, refill: str = "eq", q: int = 19, collision: str = "srt",
                  perturb=None, ny=None):
    """Standing gravity wave (Sec. 4.1): L x L x nz, periodic x and z, no-slip y
    walls, depth L/2, amplitude 0.01 L, wavelength L, gravity -y."""
    depth = L / 2 if depth is None else depth
    amp = 0.01 * L if amp is None else amp
    ny = L if ny is None else ny
    params = _base(q=q, collision=collision, refill=refill, shape=(L, ny, nz),
                   periodic=(True, False, True), nu=nu, g=(0.0, -g, 0.0))
    phi = wave_fill(L, ny, nz, depth, amp, L, perturb)
    return dict(name=f"standing_wave_{L}x{ny}x{nz}", params=params, phi=phi, u0=None,
                obstacle=None, h_ref=float(depth), depth=float(depth), amp=float(amp),
                wavelength=float(L))


def dam_break(nx=512, ny=256, nz=16, width=128, height=128, g=2e-5, nu=5e-4,
              refill="eq", q=19, collision="trt"):
    """Rectangular dam break (Sec. 4.2 in shape): column width x height at the
    left wall, no-slip walls on all faces, gravity -y, TRT with Lambda = 3/16."""
    params = _base(q=q, collision=collision, refill=refill, shape=(nx, ny, nz),
                   periodic=(False, False, False), nu=nu, g=(0.0, -g, 0.0))
    phi = box_fill(nx, ny, nz, width, height)
    return dict(name=f"dam_break_{nx}x{ny}x{nz}", params=params, phi=phi, u0=None,
                obstacle=None, h_ref=float(height), width=width, height=height)


def paper_dam_break(W: int = 50, refill: str = "eq", collision: str = "srt", les_cs: float = 0.1,
                    omega: float = 1.9995, ga: float = 1.83e9, bo: float = 445.0):
    """The paper's rectangular dam break (Sec. 4.2): column W x 2W at the left
    wall of a 15W x 4W x 1 domain, free-slip walls, relaxation rate 1.9995,
    Smagorinsky C_S = 0.1, gravity from the Galilei number Ga = g W^3 / nu^2,
    surface tension from the Bond number Bo = g W^2 / sigma (rho = 1),
    hydrostatic pressure with p = p0 at the column top."""
    nu = (1.0 / 3.0) * (1.0 / omega - 0.5)
    g = ga * nu * nu / float(W) ** 3
    sigma = g * float(W) ** 2 / bo
    H = 2 * W
    params = _base(q=19, collision=collision, refill=refill, shape=(15 * W, 2 * H, 1),
                   periodic=(False, False, True), nu=nu, g=(0.0, -g, 0.0), sigma=sigma)
    params["free_slip"] = (True, True, False)
    params["les_cs"] = les_cs
    phi = box_fill(15 * W, 2 * H, 1, W, H)
    return dict(name=f"paper_dam_break_W{W}", params=params, phi=phi, u0=None, obstacle=None,
                h_ref=float(H), width=W, height=H, g=g)


# Ohnesorge number of the paper's drop impact (Sec. 4.5): Oh = mu / sqrt(sigma rho D)
DROP_OH = 0.0384


def drop_nu(diameter=40.0, sigma=1e-4, oh=DROP_OH):
    """Kinematic viscosity that gives the paper's Ohnesorge number at this
    drop diameter and surface tension (rho = 1)."""
    return oh * math.sqrt(sigma * diameter)


DROP_NU = drop_nu()


def drop_impact(n=256, pool=96, diameter=40.0, gap=30.0, speed=0.05, sigma=1e-4, g=1e-6,
                nu=DROP_NU, refill="eq", q=27, collision="trt", nxy=None):
    """Drop impact into a pool (Sec. 4.5 in shape): n^3 (or nxy x nxy x n),
    periodic x and y, no-slip z walls, pool depth `pool`, drop of the given
    diameter centred `gap` cells above the surface, moving at -speed in z
    (Weber number rho U^2 D / sigma = 1000 at the defaults); viscosity from the
    paper's Ohnesorge number Oh = 0.0384 (2.43e-3 at the defaults)."""
    nxy = n if nxy is None else nxy
    params = _base(q=q, collision=collision, refill=refill, shape=(nxy, nxy, n),
                   periodic=(True, True, False), nu=nu, g=(0.0, 0.0, -g), sigma=sigma)
    phi = np.zeros((n, nxy, nxy))
    phi[:pool] = 1.0
    centre = (nxy / 2.0, nxy / 2.0, pool + gap)
    drop = sphere_fraction(nxy, nxy, n, centre, diameter / 2.0)
    phi = np.maximum(phi, drop)
    u0 = np.zeros((n, nxy, nxy, 3))
    u0[..., 2] = np.where(drop > 0.0, -speed, 0.0)
    return dict(name=f"drop_impact_{nxy}x{nxy}x{n}", params=params, phi=phi, u0=u0,
                obstacle=None, h_ref=float(pool))


def bubbles_in_pool(nx=48, ny=40, depth=32, bubbles=((12.0, 9.0, 4.5), (30.0, 13.0, 5.5),
                                                      (21.0, 21.0, 4.0)), g=2e-4, nu=5e-3,
                    q=19, collision="trt", refill="eq"):
    """Enclosed gas bubbles (discs (x, y, radius)) in a pool of depth `depth`
    under a gas layer, nx x ny x 1, periodic x and z, walls in y, gravity -y,
    with the bubble model on (each bubble keeps its own volume pressure)."""
    phi = np.zeros((1, ny, nx))
    phi[0, :depth, :] = 1.0
    if depth < ny:
        phi[0, depth, :] = 0.0
    for cx, cy, r in bubbles:
        phi -= cylinder_fraction(nx, ny, (cx, cy), r)
    phi = np.clip(phi, 0.0, 1.0)
    params = _base(q=q, collision=collision, refill=refill, shape=(nx, ny, 1),
                   periodic=(True, False, True), nu=nu, g=(0.0, -g, 0.0), options=16)
    return dict(name=f"bubbles_in_pool_{nx}x{ny}", params=params, phi=phi, u0=None,
                obstacle=None, h_ref=float(depth))


def taylor_bubble(D: int = 32, refill: str = "eq", omega: float = 1.8, mo: float = 0.015,
                  bo: float = 100.0, collision: str = "srt"):
    """The paper's Taylor bubble (Sec. 4.4): a tube of diameter D along z
    (cells whose centre lies more than D/2 from the axis are obstacles) in a
    D x D x 10D domain, no-slip everywhere, filled with liquid except for a
    cylindrical gas bubble of diameter 0.75 D and length 3 D whose bottom is
    D above the floor; D3Q19 SRT at relaxation rate `omega`, gravity -z and
    surface tension from the Morton number Mo = g mu^4 / (rho sigma^3) and the
    Bond number Bo = g D^2 / sigma (rho = 1, so mu = nu); hydrostatic density
    with rho = 1 at z = 5D; the bubble model keeps the bubble's volume
    pressure, p_V(0) = 1/3."""
    nu = (1.0 / 3.0) * (1.0 / omega - 0.5)
    # Mo = nu^4 Bo^3 / (g^2 D^6)  ->  g = nu^2 Bo^1.5 / (sqrt(Mo) D^3)
    g = nu * nu * bo ** 1.5 / (math.sqrt(mo) * float(D) ** 3)
    sigma = g * float(D) ** 2 / bo
    nx = ny = D
    nz = 10 * D
    c = D / 2.0
    J, I = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    outside = (I + 0.5 - c) ** 2 + (J + 0.5 - c) ** 2 > c * c
    obstacle = np.zeros((nz, ny, nx), dtype=np.uint8)
    obstacle[:, outside] = 1
    phi = np.ones((nz, ny, nx))
    disc = cylinder_fraction(nx, ny, (c, c), 0.375 * D)[0]
    phi[D:4 * D] = 1.0 - disc
    phi[:, outside] = 0.0
    params = _base(q=19, collision=collision, refill=refill, shape=(nx, ny, nz),
                   periodic=(False, False, False), nu=nu, g=(0.0, 0.0, -g), sigma=sigma,
                   options=16)
    return dict(name=f"taylor_bubble_D{D}", params=params, phi=phi, u0=None, obstacle=obstacle,
                h_ref=5.0 * D, D=D, g=g, sigma=sigma, nu=nu)


def bubbly_poiseuille(L: int = 100, n_bubbles: int = 381, refill: str = "eq", seed: int = 2577,
                      omega: float = 1.989, re: float = 1e4, mo: float = 1e-5,
                      collision: str = "srt"):
    """The paper's bubbly plane Poiseuille flow (Sec. 4.6): a 2L x L x L
    channel, periodic in x and y, no-slip walls in z, driven by a force along
    x; `n_bubbles` spheres of diameter 0.1 L at seeded random positions (centres
    at least 0.05 L from the walls, at least three cells between the
    spheres' surfaces), gas fraction about 0.1; the liquid starts on the parabola
    u(z) = F z (L - z) / (2 mu); Re = L u_max / nu with u_max = u(L/2),
    Mo = F mu^4 / (rho sigma^3) with the driving acceleration in the place of
    g (rho = 1, so mu = nu); no hydrostatic gradient (the force is along the
    periodic axis); the bubble model is on."""
    nu = (1.0 / 3.0) * (1.0 / omega - 0.5)
    u_max = re * nu / L
    F = 8.0 * nu * u_max / float(L) ** 2
    sigma = (F * nu ** 4 / mo) ** (1.0 / 3.0)
    nx, ny, nz = 2 * L, L, L
    R = 0.05 * L
    rng = np.random.default_rng(seed)
    centres = []
    tries = 0
    while len(centres) < n_bubbles:
        tries += 1
        if tries > 1000000:
            raise RuntimeError("could not place the bubbles")
        c = np.array([rng.uniform(0, nx), rng.uniform(0, ny), rng.uniform(0.05 * L, 0.95 * L)])
        ok = True
        for q in centres:
            d = np.abs(c - q)
            d[0] = min(d[0], nx - d[0])
            d[1] = min(d[1], ny - d[1])
            if float(np.sqrt((d * d).sum())) < 2.0 * R + 3.0:
                ok = False
                break
        if ok:
            centres.append(c)
    gas = np.zeros((nz, ny, nx))
    n = int(math.ceil(2 * R)) + 4
    for c in centres:
        o = [int(math.floor(c[a] - R)) - 1 for a in range(3)]
        loc = sphere_fraction(n, n, n, tuple(c[a] - o[a] for a in range(3)), R)
        zi = np.arange(o[2], o[2] + n)
        keep = (zi >= 0) & (zi < nz)
        yi = np.mod(np.arange(o[1], o[1] + n), ny)
        xi = np.mod(np.arange(o[0], o[0] + n), nx)
        gas[np.ix_(zi[keep], yi, xi)] += loc[keep]
    phi = 1.0 - np.clip(gas, 0.0, 1.0)
    z = np.arange(nz) + 0.5
    ux = F / (2.0 * nu) * z * (L - z)
    u0 = np.zeros((nz, ny, nx, 3))
    u0[..., 0] = ux[:, None, None]
    params = _base(q=19, collision=collision, refill=refill, shape=(nx, ny, nz),
                   periodic=(True, True, False), nu=nu, g=(F, 0.0, 0.0), sigma=sigma,
                   options=16)
    return dict(name=f"bubbly_poiseuille_L{L}", params=params, phi=phi, u0=u0, obstacle=None,
                h_ref=float("nan"), L=L, u_max=u_max, F=F, sigma=sigma, nu=nu,
                centres=np.array(centres))


def static_drop(n=32, radius=8.0, sigma=1e-3, nu=0.1, q=19, two_d=False):
    """Resting drop in a fully periodic box without gravity (Young-Laplace)."""
    if two_d:
        params = _base(q=q, shape=(n, n, 1), periodic=(True, True, True), nu=nu, sigma=sigma)
        phi = cylinder_fraction(n, n, (n / 2.0, n / 2.0), radius)
    else:
        params = _base(q=q, shape=(n, n, n), periodic=(True, True, True), nu=nu, sigma=sigma)
        phi = sphere_fraction(n, n, n, (n / 2.0, n / 2.0, n / 2.0), radius)
    return dict(name=f"static_drop_{n}", params=params, phi=phi, u0=None, obstacle=None,
                h_ref=float("nan"), radius=radius)


def poiseuille(ny=16, nx=4, g=1e-6, nu=0.1, collision="trt", q=19):
    """Fully liquid channel between no-slip walls at y = 0 and y = ny, driven by
    a body force along x (no interface)."""
    params = _base(q=q, collision=collision, shape=(nx, ny, 1), periodic=(True, False, True),
                   nu=nu, g=(g, 0.0, 0.0))
    phi = np.ones((1, ny, nx))
    return dict(name=f"poiseuille_{ny}", params=params, phi=phi, u0=None, obstacle=None,
                h_ref=float("nan"))


def batched_waves(seed: int = 2207, n_geom: int = 64):
    """Geometries of the batched standing-wave set: wavelength U[32, 256],
    width U{1..8}, depth = wavelength/2, amplitude 1% of the wavelength,
    viscosity U[1e-3, 1e-2], gravity 1e-5; each geometry times five schemes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for gi in range(n_geom):
        lam = int(round(rng.uniform(32.0, 256.0)))
        width = int(rng.integers(1, 9))
        nu = float(rng.uniform(1e-3, 1e-2))
        for scheme in REFILL_SCHEMES:
            out.append(dict(lam=lam, width=width, nu=nu, refill=scheme, geom=gi))
    return out


def workload(name: str, **kw):
    """Named workloads at the sizes quoted for them."""
    if name == "standing_wave_64":
        return standing_wave(64, **kw)
    if name == "dam_break_512":
        return dam_break(**kw)
    if name == "drop_impact_256":
        return drop_impact(**kw)
    raise KeyError(name)
