"""Pins of the oracle's interface mass flux, conversions, excess-mass
redistribution, refilling means, obstacle-narrowed normals, observables and
input geometry (Sec. 2.2, 3.1, 3.2 and the readings R3, R5, R6, R7, R11,
R13, R14): each expected value is computed here from the paper's
definitions on a hand-built state, in code that shares nothing with the
oracle but the lattice table (itself pinned by test_oracle_pins)."""
import numpy as np
import pytest

import oracle
from paper_2207_14496_gb300 import inputs

STD, NF, NE = 0, 1, 2


def _lattice(q):
    o = oracle.Oracle(dict(q=q, shape=(4, 4, 4), periodic=(True, True, True), nu=0.1))
    c, w, opp = o.lattice()
    return c, w, opp


def _neighbour(idx, cvec, shape, periodic):
    """(k, j, i) of cell idx + c, or None beyond a non-periodic wall."""
    nz, ny, nx = shape
    k, j, i = idx
    out = []
    for v, d, n, per in ((i, cvec[0], nx, periodic[0]), (j, cvec[1], ny, periodic[1]),
                         (k, cvec[2], nz, periodic[2])):
        u = v + d
        if u < 0 or u >= n:
            if not per:
                return None
            u %= n
        out.append(u)
    return (out[2], out[1], out[0])


def _classes(types, c, periodic):
    """Thuerey's class of every interface cell (Sec. 2.2): no liquid
    neighbour -> NF, no gas neighbour -> NE, both or neither -> standard;
    walls count as neither."""
    cls = np.zeros(types.shape, dtype=int)
    for idx in zip(*np.nonzero(types == oracle.IFACE)):
        liq = gas = False
        for cv in c[1:]:
            n = _neighbour(idx, cv, types.shape, periodic)
            if n is None:
                continue
            liq |= types[n] == oracle.LIQUID
            gas |= types[n] == oracle.GAS
        cls[idx] = NF if gas and not liq else NE if liq and not gas else STD
    return cls


def _expected_mass(types, phi, mass, f, c, opp, periodic, thurey):
    """m + sum_i dm_i for every interface cell: dm_i = f_in - f_out with a
    liquid neighbour, (phi_x + phi_n)/2 times the bracket of the class table
    with an interface neighbour (Thuerey: a standard cell takes only f_in
    from an NF neighbour and only -f_out towards an NE neighbour; an NF cell
    only loses, an NE cell only gains; equal classes use the full bracket),
    nothing with gas or a wall; f_in = f*_{opp i}(x + c_i), f_out = f*_i(x)."""
    cls = _classes(types, c, periodic)
    out = mass.copy()
    for idx in zip(*np.nonzero(types == oracle.IFACE)):
        dm = 0.0
        for i in range(1, len(c)):
            n = _neighbour(idx, c[i], types.shape, periodic)
            if n is None or types[n] not in (oracle.LIQUID, oracle.IFACE):
                continue
            f_in, f_out = f[(opp[i],) + n], f[(i,) + idx]
            both = f_in - f_out
            if types[n] == oracle.LIQUID:
                dm += both
                continue
            cx, cn = cls[idx], cls[n]
            if not thurey or cx == cn:
                br = both
            elif cx == STD:
                br = f_in if cn == NF else -f_out if cn == NE else both
            elif cx == NF:
                br = -f_out
            else:
                br = f_in
            dm += 0.5 * (phi[idx] + phi[n]) * br
        out[idx] = mass[idx] + dm
    return out


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("thurey", [True, False])
def test_mass_flux_of_every_class_pair(q, thurey):
    """Eq. nm-fslbm-mass-flux with Thuerey's table (R5): on a periodic chain
    of liquid, interface and gas cells laid out so that every ordered pair of
    classes meets (one cell across, walls above and below, the chain its own
    neighbour across the periodic z), with non-equilibrium stored PDFs, one
    step changes each interface cell's mass by exactly the flux computed
    here (no cell converts: fill levels stay inside (0.2, 0.8))."""
    c, w, opp = _lattice(q)
    L, I, G = oracle.LIQUID, oracle.IFACE, oracle.GAS
    chain = [L, I, I, G, G, I, I, G, L, I, I, L, L, I, I, I, I, G]
    nx, ny, nz = len(chain), 1, 1
    periodic = (True, False, True)
    rng = np.random.default_rng(2207 + q)
    types = np.array(chain, dtype=np.uint8).reshape(nz, ny, nx)
    f = w[:, None, None, None] * (1.0 + 0.02 * rng.standard_normal((q, nz, ny, nx)))
    rho = f.sum(0)
    phi = np.where(types == oracle.LIQUID, 1.0, 0.0)
    iface = types == oracle.IFACE
    phi[iface] = rng.uniform(0.3, 0.7, iface.sum())
    mass = np.where(types == oracle.LIQUID, rho, phi * rho)
    cls = _classes(types, c, periodic)
    pairs = set()
    for idx in zip(*np.nonzero(iface)):
        for cv in c[1:]:
            n = _neighbour(idx, cv, types.shape, periodic)
            if n is not None and types[n] == oracle.IFACE:
                pairs.add((cls[idx], cls[n]))
    assert len(pairs) == 9, pairs
    o = oracle.Oracle(dict(q=q, shape=(nx, ny, nz), periodic=periodic, nu=0.05,
                           options=0 if thurey else oracle.OPT_SIMPLE_FLUX))
    o.set_state(types, phi, f, mass)
    want = _expected_mass(types, phi, mass, f, c, opp, periodic, thurey)
    o.step(1)
    assert np.array_equal(o.types(), types), "a cell converted"
    got = o.mass()
    assert np.allclose(got[iface], want[iface], rtol=0.0, atol=1e-15)


# ------------------------------------------------------------------ conversions
def _flat_layer(q, nx=7, ny=8):
    """Liquid rows y < 3, an interface row y = 3 (phi = 1/2), gas above; one
    cell across z (periodic), walls at y = 0 and y = ny - 1; every stored PDF
    is the rest equilibrium w_i, so no mass flows in one step and the only
    mass changes come from conversions."""
    c, w, opp = _lattice(q)
    types = np.full((1, ny, nx), oracle.GAS, dtype=np.uint8)
    types[0, :3, :] = oracle.LIQUID
    types[0, 3, :] = oracle.IFACE
    phi = np.where(types == oracle.LIQUID, 1.0, 0.0)
    phi[0, 3, :] = 0.5
    f = np.broadcast_to(w[:, None, None, None], (q,) + types.shape).copy()
    mass = phi * f.sum(0)
    o = oracle.Oracle(dict(q=q, shape=(nx, ny, 1), periodic=(True, False, True), nu=0.05))
    return o, types, phi, f, mass, c


@pytest.mark.parametrize("q", [19, 27])
def test_excess_mass_shared_per_direction_among_interface_neighbours(q):
    """Eq. nm-fslbm-excess-mass with R3: a filled interface cell's excess
    m - rho goes in equal shares to the stencil neighbours that are interface
    cells after the conversions (its gas neighbours, new interface cells now,
    included), one share per direction (a neighbour reached along several
    directions, here across the periodic z, takes several)."""
    o, types, phi, f, mass, c = _flat_layer(q)
    a = (0, 3, 3)
    mass[a] = 1.3
    phi[a] = 1.3
    o.set_state(types, phi, f, mass)
    o.step(1)
    got_t, got_m = o.types(), o.mass()
    assert got_t[a] == oracle.LIQUID
    rho_a = got_m[a]                      # a filled cell keeps m = rho
    mex = mass[a] - rho_a
    shares = {}
    for cv in c[1:]:
        n = _neighbour(a, cv, types.shape, (True, False, True))
        if n is None or n == a:
            continue
        if types[n] in (oracle.IFACE, oracle.GAS):   # gas neighbours become interface
            shares[n] = shares.get(n, 0) + 1
    nr = sum(shares.values())
    for n, k in shares.items():
        assert got_t[n] == oracle.IFACE
        start = mass[n] if types[n] == oracle.IFACE else 0.0
        assert abs(got_m[n] - (start + k * mex / nr)) < 1e-14, (n, k, nr)
    untouched = (types == oracle.IFACE)
    for n in shares:
        untouched[n] = False
    untouched[a] = False
    assert np.array_equal(got_m[untouched], mass[untouched])
    assert o.lost_mass() == 0.0


@pytest.mark.parametrize("q", [19, 27])
def test_excess_mass_without_receiver_is_kept_as_lost_mass(q):
    """R3: a filled cell with no interface neighbour after the conversions
    hands its excess to the per-cell lost-mass accumulator, which the total
    mass includes (Sec. 3.2: mass is conserved)."""
    o, types, phi, f, mass, c = _flat_layer(q)
    types[0, 1, 3] = oracle.IFACE     # an interface cell inside the liquid
    phi[0, 1, 3] = 1.25
    mass[0, 1, 3] = 1.25
    o.set_state(types, phi, f, mass)
    m0 = o.total_mass()
    o.step(1)
    assert o.types()[0, 1, 3] == oracle.LIQUID
    rho = o.mass()[0, 1, 3]
    assert abs(o.lost_mass() - (1.25 - rho)) < 1e-15
    assert abs(o.total_mass() - m0) < 1e-13


@pytest.mark.parametrize("q", [19, 27])
def test_filling_wins_over_an_emptying_neighbour(q):
    """R6 (Sec. 2.2, separation prioritised): an interface cell whose fill
    level falls below -eps stays interface when a neighbour fills in the same
    step; without the filling neighbour it empties and its liquid neighbours
    become interface (R18: with their density of the step as mass)."""
    for filling in (True, False):
        o, types, phi, f, mass, c = _flat_layer(q)
        a, b = (0, 3, 3), (0, 3, 4)
        mass[a] = phi[a] = 1.3 if filling else 0.5
        mass[b] = phi[b] = -0.3
        o.set_state(types, phi, f, mass)
        o.step(1)
        t = o.types()
        if filling:
            assert t[a] == oracle.LIQUID and t[b] == oracle.IFACE
        else:
            assert t[a] == oracle.IFACE and t[b] == oracle.GAS
            assert t[0, 2, 4] == oracle.IFACE          # liquid below b
            assert t[0, 2, 1] == oracle.LIQUID          # away from b
            # R18: a liquid cell turned interface starts from m = its density
            # of the step (the rest equilibrium's, sum w_i = 1), then receives
            # its shares of b's (negative) excess m_b = -0.3 (R3)
            shares = {}
            for cv in c[1:]:
                n = _neighbour(b, cv, types.shape, (True, False, True))
                if n is not None and n != b and types[n] in (oracle.IFACE, oracle.LIQUID):
                    shares[n] = shares.get(n, 0) + 1
            nr = sum(shares.values())
            want = 1.0 + shares[(0, 2, 4)] * (-0.3) / nr
            assert abs(o.mass()[0, 2, 4] - want) < 1e-14


# ------------------------------------------------------------------ refilling means
@pytest.mark.parametrize("q", [19, 27])
def test_refill_eq_takes_plain_means_of_the_valid_neighbours(q):
    """R7 (Sec. 3.1, EQ): a new interface cell gets f^eq(rho_bar, u_bar) with
    rho_bar and u_bar the plain means, over its stencil neighbours that are
    fluid and not new themselves, of each neighbour's density and velocity
    (stored PDFs, no forcing), whatever their spread."""
    c, w, opp = _lattice(q)
    nx, ny, nz = 9, 7, 7
    rng = np.random.default_rng(14496 + q)
    o = oracle.Oracle(dict(q=q, shape=(nx, ny, nz), periodic=(False, True, True), nu=0.02,
                           refill="eq"))
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    types = np.where(x >= 4, oracle.LIQUID, oracle.GAS).astype(np.uint8)
    types[(x == 5) & (y == 2)] = oracle.IFACE       # interface neighbours count too
    centre = (3, 3, 4)                              # (k, j, i)
    types[centre] = oracle.IFACE
    other_new = (3, 4, 4)                           # a second new cell: not a source
    types[other_new] = oracle.IFACE
    fluid = (types == oracle.LIQUID) | (types == oracle.IFACE)
    rho = 1.0 + 0.05 * rng.standard_normal(x.shape)
    u = 0.03 * rng.standard_normal((3,) + x.shape)
    f = np.zeros((q,) + x.shape)
    for i in range(q):
        cu = c[i, 0] * u[0] + c[i, 1] * u[1] + c[i, 2] * u[2]
        usq = (u ** 2).sum(0)
        f[i] = np.where(fluid, w[i] * rho * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * usq), 0.0)
    f = f * (1.0 + 0.01 * rng.standard_normal(f.shape)) * fluid
    phi = np.where(types == oracle.LIQUID, 1.0, np.where(types == oracle.IFACE, 0.5, 0.0))
    phi[centre] = phi[other_new] = 0.0
    o.set_state(types, phi, f)
    new = np.zeros(x.shape, dtype=np.uint8)
    new[centre] = new[other_new] = 1
    idx = centre[2] + nx * (centre[1] + ny * centre[0])
    out = o.refill_probe(idx, new)
    rs, us, count = 0.0, np.zeros(3), 0
    for cv in c[1:]:
        n = _neighbour(centre, cv, x.shape, (False, True, True))
        if n is None or not fluid[n] or new[n]:
            continue
        fn = f[(slice(None),) + n]
        r = fn.sum()
        rs += r
        us += (fn @ c) / r
        count += 1
    assert count >= 8
    rb, ub = rs / count, us / count
    cu = c @ ub
    want = w * rb * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * ub @ ub)
    assert np.allclose(out, want, rtol=1e-13, atol=1e-16)


# ------------------------------------------------------------------ normals next to obstacles
@pytest.mark.parametrize("blocked", [[(1, 0, 0)], [(0, -1, 0), (1, 1, 1)], [(-1, 1, 0), (0, 0, 1)],
                                     [(1, 0, 0), (-1, 0, 0)]])
def test_normal_next_to_obstacles_is_exact_for_linear_fill(blocked):
    """R11: the Parker-Youngs gradient of a linear fill level stays exact
    when obstacle cells (fill level 0 here, so that using them would show)
    sit in the stencil: an axis whose 3x3 block touches one falls back to the
    central or one-sided difference over the other cells; an axis blocked on
    both sides has no difference (zero)."""
    n = 9
    o = oracle.Oracle(dict(q=19, shape=(n, n, n), periodic=(False, False, False), nu=0.1))
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    grad = np.array([0.03, -0.02, 0.05])
    phi = 0.4 + grad[0] * x + grad[1] * y + grad[2] * z
    types = np.full(phi.shape, oracle.IFACE, dtype=np.uint8)
    for dx, dy, dz in blocked:
        types[4 + dz, 4 + dy, 4 + dx] = oracle.OBST
        phi[4 + dz, 4 + dy, 4 + dx] = 0.0
    o.set_state(types, phi, np.ones((19,) + phi.shape) / 19.0)
    got = o.normal_at(4 + n * (4 + n * 4))
    want = grad.copy()
    if (1, 0, 0) in blocked and (-1, 0, 0) in blocked:
        want[0] = 0.0
    assert np.allclose(got, want, rtol=0.0, atol=1e-15)


# ------------------------------------------------------------------ observables and geometry
def test_trace_observables_follow_their_definitions():
    """R14: column height at x = 0 = sum over y of phi(0, y, z), averaged over
    z; front = 1 + the largest x of an interface cell in the y = 0 layer;
    height = 1 + the largest y of an interface cell at x = 0 (any z)."""
    nx, ny, nz = 12, 9, 3
    rng = np.random.default_rng(9)
    types = rng.choice([oracle.GAS, oracle.IFACE, oracle.LIQUID], size=(nz, ny, nx),
                       p=[0.4, 0.3, 0.3]).astype(np.uint8)
    phi = np.where(types == oracle.LIQUID, 1.0, np.where(types == oracle.IFACE,
                                                         rng.uniform(0.1, 0.9, types.shape), 0.0))
    o = oracle.Oracle(dict(q=19, shape=(nx, ny, nz), periodic=(False, False, True), nu=0.1))
    o.set_state(types, phi, np.ones((19,) + types.shape) / 19.0)
    assert o.column_height(0) == pytest.approx(phi[:, :, 0].sum(axis=1).mean(), rel=1e-15)
    xs = np.nonzero((types[:, 0, :] == oracle.IFACE).any(axis=0))[0]
    ys = np.nonzero((types[:, :, 0] == oracle.IFACE).any(axis=0))[0]
    assert o.front() == 1.0 + xs.max()
    assert o.height() == 1.0 + ys.max()


def test_wave_fill_cell_convention():
    """R13: in the standing wave, cell i covers x in [i - 1/2, i + 1/2) and
    cell j covers y in [j, j + 1); phi(i, j) is the cell average of the
    clamped height h(x) - j (here by a fine midpoint rule, independent of
    the generator's Gauss-Legendre quadrature, whose error at the kinks of
    the clamp is a few 1e-6; a half-cell shift of either convention would
    change phi by about 0.1)."""
    nx, ny, depth, amp, lam = 16, 12, 6.3, 0.8, 16.0
    phi = inputs.wave_fill(nx, ny, 1, depth, amp, lam)[0]
    m = 20000
    for i in range(nx):
        xs = i - 0.5 + (np.arange(m) + 0.5) / m
        h = depth + amp * np.cos(2.0 * np.pi * xs / lam)
        for j in range(ny):
            want = np.clip(h - j, 0.0, 1.0).mean()
            assert abs(phi[j, i] - want) < 1e-4, (i, j)
