"""Pins of the oracle's bubble model (Sec. 2.2, Eq. nm-fslbm-pressure-volume:
p_V(t) = p_V(0) V(0) / V(t) per enclosed gas volume, bubbles merging and
splitting).  Checked against a library labelling, brute force on small
grids, and the invariants the bookkeeping must keep: p V per bubble without
topology change, the sum of p V through a merge, one pressure for the parts
of a split bubble, and mass conservation with the model on.  Both
connectivity readings are pinned: gas and interface cells together (the
default) and gas cells alone with interface cells attached (option 32)."""
import numpy as np
import pytest

import oracle
from paper_2207_14496_gb300 import inputs

ndimage = pytest.importorskip("scipy.ndimage")

GAS, IFACE, LIQ = 0, 1, 2


MODES = {"gas_iface": oracle.OPT_BUBBLES,
         "gas_only": oracle.OPT_BUBBLES | oracle.OPT_BUBBLE_GAS_ONLY}


def _orc(shape, periodic=(False, False, False), p_v=1.0 / 3.0, q=19, mode="gas_iface"):
    params = inputs._base(q=q, collision="srt", refill="eq", shape=shape, periodic=periodic,
                          nu=0.05, g=(0.0, 0.0, 0.0))
    params["options"] = MODES[mode]
    params["p_v"] = p_v
    return oracle.Oracle(params)


def _blobs(shape, seed, frac=0.55):
    """Random gas blobs in liquid with interface cells around them."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    # 55% before the opening leaves several components of a few cells each
    gas = rng.random((nz, ny, nx)) < frac
    gas = ndimage.binary_opening(gas)
    types = np.full((nz, ny, nx), LIQ, dtype=np.uint8)
    types[gas] = GAS
    near = ndimage.binary_dilation(gas, structure=np.ones((3, 3, 3))) & ~gas
    types[near] = IFACE
    phi = np.where(types == LIQ, 1.0, np.where(types == GAS, 0.0, rng.uniform(0.05, 0.95,
                                                                            types.shape)))
    return types, phi


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_gas_components_match_library_labelling(seed, mode):
    # large and sparse enough that the interface layers leave several
    # gas + interface components
    shape = (24, 20, 16)
    types, phi = _blobs(shape, seed, frac=0.45)
    o = _orc(shape, mode=mode)
    lab, p = o.bubble_probe(types, phi, first=True)
    member = (types == GAS) if mode == "gas_only" else (types == GAS) | (types == IFACE)
    ref, n = ndimage.label(member, structure=ndimage.generate_binary_structure(3, 1))
    assert n >= 3
    gas = member
    # same partition, labels = smallest flat index of the component
    flat = np.arange(types.size).reshape(types.shape)
    for k in range(1, n + 1):
        cells = ref == k
        labels = np.unique(lab[cells])
        assert labels.size == 1
        assert labels[0] == flat[cells].min()
    assert (lab[types == LIQ] == -1).all()
    # every bubble starts at the volume pressure
    assert np.allclose(p[gas], 1.0 / 3.0, rtol=0, atol=1e-15)


def test_interface_cells_take_smallest_gas_neighbour_label():
    """Gas-only reading: an interface cell joins the bubble with the smallest
    label among its gas stencil neighbours."""
    shape = (12, 10, 8)
    types, phi = _blobs(shape, 7)
    o = _orc(shape, q=27, mode="gas_only")
    lab, _ = o.bubble_probe(types, phi, first=True)
    nz, ny, nx = types.shape
    for z, y, x in zip(*np.nonzero(types == IFACE)):
        best = -1
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    zz, yy, xx = z + dz, y + dy, x + dx
                    if (dz, dy, dx) == (0, 0, 0) or not (0 <= zz < nz and 0 <= yy < ny and 0 <= xx < nx):
                        continue
                    if types[zz, yy, xx] == GAS and (best < 0 or lab[zz, yy, xx] < best):
                        best = lab[zz, yy, xx]
        assert lab[z, y, x] == best


def _volume(types, phi, lab, root):
    cells = lab == root
    return float(np.sum(np.where(types[cells] == GAS, 1.0, 1.0 - phi[cells])))


@pytest.mark.parametrize("mode", list(MODES))
def test_compression_keeps_pv_and_merge_adds_pv(mode):
    """Two bubbles, then the first compressed (its interface cells fuller),
    then both joined by a gas bridge."""
    shape = (16, 6, 1)
    nz, ny, nx = 1, 6, 16
    types = np.full((nz, ny, nx), LIQ, dtype=np.uint8)
    phi = np.ones((nz, ny, nx))
    types[0, 1:5, 1:5] = IFACE
    types[0, 2:4, 2:4] = GAS
    types[0, 1:5, 9:14] = IFACE
    types[0, 2:4, 10:13] = GAS
    phi[types == IFACE] = 0.5
    phi[types == GAS] = 0.0
    o = _orc(shape, p_v=0.3, mode=mode)
    lab, p = o.bubble_probe(types, phi, first=True)
    ra, rb = lab[0, 2, 2], lab[0, 2, 10]
    assert ra != rb
    Va, Vb = _volume(types, phi, lab, ra), _volume(types, phi, lab, rb)
    Ka, Kb = 0.3 * Va, 0.3 * Vb
    # compress bubble a: its interface cells fill to 0.8
    phi2 = phi.copy()
    phi2[0, 1:5, 1:5][types[0, 1:5, 1:5] == IFACE] = 0.8
    lab2, p2 = o.bubble_probe(types, phi2, first=False)
    Va2 = _volume(types, phi2, lab2, ra)
    assert p2[0, 2, 2] * Va2 == pytest.approx(Ka, rel=1e-13)
    assert p2[0, 2, 2] > 0.3
    assert p2[0, 2, 10] == pytest.approx(0.3, rel=1e-13)
    # bridge: gas cells join the two bubbles
    types3 = types.copy()
    types3[0, 2:4, 4:10] = GAS
    types3[0, 1, 4:10] = IFACE
    types3[0, 4, 4:10] = IFACE
    phi3 = phi2.copy()
    phi3[types3 == GAS] = 0.0
    phi3[0, 1, 4:10] = 0.5
    phi3[0, 4, 4:10] = 0.5
    lab3, p3 = o.bubble_probe(types3, phi3, first=False)
    r = lab3[0, 2, 2]
    assert lab3[0, 2, 10] == r
    V3 = _volume(types3, phi3, lab3, r)
    # the new gas cells carry no old K: the merged bubble holds Ka + Kb
    assert p3[0, 2, 2] * V3 == pytest.approx(Ka + Kb, rel=1e-13)


@pytest.mark.parametrize("mode", list(MODES))
def test_split_bubble_keeps_its_pressure_in_every_part(mode):
    shape = (14, 5, 1)
    nz, ny, nx = 1, 5, 14
    types = np.full((nz, ny, nx), LIQ, dtype=np.uint8)
    types[0, 1:4, 1:13] = IFACE
    types[0, 2, 2:12] = GAS
    phi = np.where(types == IFACE, 0.4, np.where(types == GAS, 0.0, 1.0))
    o = _orc(shape, p_v=0.25, mode=mode)
    lab, p = o.bubble_probe(types, phi, first=True)
    # compress, then cut the bubble in two with a liquid plug
    phi2 = np.where(types == IFACE, 0.7, phi)
    lab2, p2 = o.bubble_probe(types, phi2, first=False)
    p_before = p2[0, 2, 2]
    types3 = types.copy()
    types3[0, 1:4, 7] = LIQ
    phi3 = np.where(types3 == LIQ, 1.0, phi2)
    lab3, p3 = o.bubble_probe(types3, phi3, first=False)
    assert lab3[0, 2, 2] != lab3[0, 2, 10]
    # each part keeps K in proportion to its volume: same pressure, up to the
    # volume the plug removed (the parts' total volume is what K is spread over)
    assert p3[0, 2, 2] == pytest.approx(p3[0, 2, 10], rel=1e-13)
    V_all2 = _volume(types, phi2, lab2, lab2[0, 2, 2])
    V_parts = _volume(types3, phi3, lab3, lab3[0, 2, 2]) + _volume(types3, phi3, lab3, lab3[0, 2, 10])
    assert p3[0, 2, 2] == pytest.approx(p_before * V_all2 / V_parts, rel=1e-13)


def test_periodic_wrap_joins_components():
    shape = (10, 6, 1)
    types = np.full((1, 6, 10), LIQ, dtype=np.uint8)
    types[0, 2:4, 0:2] = GAS
    types[0, 2:4, 8:10] = GAS
    phi = np.where(types == GAS, 0.0, 1.0)
    lab_open, _ = _orc(shape).bubble_probe(types, phi, first=True)
    assert lab_open[0, 2, 0] != lab_open[0, 2, 9]
    lab_per, _ = _orc(shape, periodic=(True, False, False)).bubble_probe(types, phi, first=True)
    assert lab_per[0, 2, 0] == lab_per[0, 2, 9] == 20


def test_mass_conserved_with_bubbles_through_conversions():
    """A closed box: the gas above a sloshing column is one bubble whose
    volume pressure follows its volume; mass stays conserved."""
    w = inputs.dam_break(nx=40, ny=30, nz=1, width=12, height=20, g=2e-4, nu=5e-3)
    w["params"]["periodic"] = (False, False, True)
    w["params"]["options"] = oracle.OPT_BUBBLES
    o = oracle.Oracle(w["params"])
    o.init_fill(w["phi"], h_ref=w["h_ref"])
    m0 = o.total_mass()
    t0, phi0 = o.types(), o.phi()
    lab0, _ = o.bubbles()
    r0 = lab0[t0 == GAS][0]
    K0 = (1.0 / 3.0) * _volume(t0, phi0, lab0, r0)
    o.step(300)
    assert abs(o.total_mass() - m0) <= 4 * 300 * np.finfo(float).eps * m0
    lab, p = o.bubbles()
    t, phi = o.types(), o.phi()
    gas = t == GAS
    assert len(np.unique(lab[gas])) == 1
    r = lab[gas][0]
    # one bubble through 300 steps of conversions: p V keeps its initial value
    assert p[gas][0] * _volume(t, phi, lab, r) == pytest.approx(K0, rel=1e-12)
    assert p[gas][0] != 1.0 / 3.0


@pytest.mark.parametrize("mode", list(MODES))
def test_pressures_do_not_depend_on_cell_order(mode):
    """The volume and K sums run in cell order: relabelling the grid by a
    mirror (which reverses the summation order) changes the pressures only by
    FP64 rounding, and every bubble's K = p V still equals its old K."""
    shape = (14, 11, 9)
    types, phi = _blobs(shape, 5)
    # interface cells next to two components would change bubble with the
    # labels under the mirror: make them liquid
    ref, n = ndimage.label(types == GAS, structure=ndimage.generate_binary_structure(3, 1))
    assert n >= 3
    big = np.where(ref > 0, ref, n + 1)
    two = ndimage.maximum_filter(ref, size=3, mode="constant") != ndimage.minimum_filter(
        big, size=3, mode="constant", cval=n + 1)
    cut = (types == IFACE) & two & (ndimage.maximum_filter(ref, size=3, mode="constant") > 0)
    types[cut] = LIQ
    phi[cut] = 1.0
    o = _orc(shape, mode=mode)
    o.bubble_probe(types, phi, first=True)
    phi2 = np.where(types == IFACE, np.clip(phi + 0.1, 0, 1), phi)
    _, p = o.bubble_probe(types, phi2, first=False)
    m = _orc(shape, mode=mode)
    m.bubble_probe(types[::-1, ::-1, ::-1], phi[::-1, ::-1, ::-1], first=True)
    _, pm = m.bubble_probe(types[::-1, ::-1, ::-1], phi2[::-1, ::-1, ::-1], first=False)
    np.testing.assert_allclose(p, pm[::-1, ::-1, ::-1], rtol=1e-14, atol=0)
    # a pure volume change (same labels): p V of every bubble is unchanged
    lab, _ = o.bubbles()
    for r in np.unique(lab[lab >= 0]):
        cells = lab == r
        v0 = _volume(types, phi, lab, r)
        v1 = _volume(types, phi2, lab, r)
        assert p[cells][0] * v1 == pytest.approx(v0 / 3.0, rel=1e-14)


@pytest.mark.parametrize("D", [16, 32])
def test_taylor_bubble_setup_matches_paper_numbers(D):
    """Sec. 4.4 setup: Mo = g nu^4 / sigma^3 = 0.015 and Bo = g D^2 / sigma =
    100 at relaxation rate 1.8, a bubble of diameter 0.75 D and length 3 D
    starting D above the floor, in a D x D x 10 D box with a tube of
    diameter D."""
    w = inputs.taylor_bubble(D)
    nu, g, sigma = w["nu"], w["g"], w["sigma"]
    assert 1.0 / (3.0 * nu + 0.5) == pytest.approx(1.8, rel=1e-14)
    assert g * nu ** 4 / sigma ** 3 == pytest.approx(0.015, rel=1e-12)
    assert g * D * D / sigma == pytest.approx(100.0, rel=1e-12)
    phi, ob = w["phi"], w["obstacle"]
    assert phi.shape == (10 * D, D, D)
    open_area = float((ob[0] == 0).sum())
    assert open_area == pytest.approx(np.pi * D * D / 4, rel=0.05)
    gas = (1.0 - phi) * (ob == 0)
    assert gas.sum() == pytest.approx(np.pi * (0.375 * D) ** 2 * 3 * D, rel=1e-3)
    zs = np.nonzero(gas.sum(axis=(1, 2)))[0]
    assert zs.min() == D and zs.max() == 4 * D - 1
    o = oracle.Oracle(w["params"])
    o.init_fill(phi, obstacle=ob, h_ref=w["h_ref"])
    lab, p = o.bubbles()
    t = o.types()
    assert np.unique(lab[t == GAS]).size == 1
    assert np.allclose(p[t == IFACE], 1.0 / 3.0, rtol=1e-14)


def test_touching_interface_layers_merge_and_a_liquid_layer_separates():
    """Default reading: two bubbles whose interface cells are face
    neighbours are one bubble; one liquid cell between the interface layers
    keeps them apart; the gas-only reading keeps them apart in both cases."""
    def two(gap):
        nx = 12 + gap
        types = np.full((1, 5, nx), LIQ, dtype=np.uint8)
        types[0, 1:4, 1:5] = IFACE
        types[0, 2, 2:4] = GAS
        types[0, 1:4, 5 + gap:9 + gap] = IFACE
        types[0, 2, 6 + gap:8 + gap] = GAS
        phi = np.where(types == IFACE, 0.5, np.where(types == GAS, 0.0, 1.0))
        return types, phi
    for gap, merged in ((0, True), (1, False)):
        types, phi = two(gap)
        shape = (types.shape[2], 5, 1)
        lab, _ = _orc(shape).bubble_probe(types, phi, first=True)
        assert (lab[0, 2, 2] == lab[0, 2, 6 + gap]) == merged
        lab, _ = _orc(shape, mode="gas_only").bubble_probe(types, phi, first=True)
        assert lab[0, 2, 2] != lab[0, 2, 6 + gap]


def test_bubbly_poiseuille_setup_matches_paper_numbers():
    """Sec. 4.6 setup: 2L x L x L, 381 spheres of diameter 0.1 L, gas
    fraction about 0.1, centres at least 0.05 L from the walls, Re = 1e4 and
    Mo = 1e-5 at relaxation rate 1.989, the liquid on the Poiseuille
    parabola with its maximum u_max at mid-channel."""
    w = inputs.bubbly_poiseuille()
    L, nu, F, sigma = w["L"], w["nu"], w["F"], w["sigma"]
    assert 1.0 / (3.0 * nu + 0.5) == pytest.approx(1.989, rel=1e-14)
    assert L * w["u_max"] / nu == pytest.approx(1e4, rel=1e-12)
    assert F * nu ** 4 / sigma ** 3 == pytest.approx(1e-5, rel=1e-12)
    assert w["phi"].shape == (L, L, 2 * L)
    assert 1.0 - w["phi"].mean() == pytest.approx(0.1, abs=0.005)
    c = w["centres"]
    assert len(c) == 381
    assert c[:, 2].min() >= 0.05 * L and c[:, 2].max() <= 0.95 * L
    d = np.abs(c[:, None, :] - c[None, :, :])
    d[..., 0] = np.minimum(d[..., 0], 2 * L - d[..., 0])
    d[..., 1] = np.minimum(d[..., 1], L - d[..., 1])
    r = np.sqrt((d * d).sum(axis=-1)) + np.eye(len(c)) * 1e9
    assert r.min() >= 0.1 * L + 3.0
    ux = w["u0"][:, 0, 0, 0]
    assert ux.max() == pytest.approx(w["u_max"], rel=1e-3)
    assert ux[0] == pytest.approx(ux[-1], rel=1e-12)


def test_largest_bubble_centroid_of_the_taylor_start():
    """The experiments' centre of mass of the largest bubble, on the initial
    Taylor-bubble state: the bubble spans z in [D, 4D), so its centre is at
    z = 2.5 D, and its volume is the gas volume of the setup."""
    from paper_2207_14496_gb300 import experiments
    w = inputs.taylor_bubble(12)
    o = oracle.Oracle(w["params"])
    o.init_fill(w["phi"], obstacle=w["obstacle"], h_ref=w["h_ref"])

    class View:
        def types(self):
            return o.types()

        def phi(self):
            return o.phi()

        def bubbles(self):
            return o.bubbles()[0]

    z, V, n = experiments.gas_centroid(View())
    gas = ((1.0 - w["phi"]) * (w["obstacle"] == 0)).sum()
    assert z == pytest.approx(2.5 * 12, rel=1e-12)
    assert V == pytest.approx(gas, rel=1e-12)
    assert n == 1
