"""The bulk stream-collide variants of the 16/32-bit path are interchangeable:
same arithmetic (collide_v, explicitly rounded), same inputs, so every
variant must give the same bits as every other after many steps, including
conversions, refilling and the near-wall / periodic-wrap special cases."""
import numpy as np
import pytest

from paper_2207_14496_gb300 import inputs

pytestmark = pytest.mark.gpu

VARIANTS = ["pair", "pair_r128", "pair_r96", "pair_r80", "tma", "quad64", "warp_tma", "pair_pipe",
            "cpa", "cpa_deep", "cpa_r96", "seg", "seg_r128", "cell", "cell_r80", "tma_r96"]
HALF_ONLY = ("quad64", "pair_pipe", "cpa_r96", "tma_r96")


def _cases():
    # ragged x (nx not a multiple of the tile), walls on every face
    dam = inputs.dam_break(nx=300, ny=40, nz=3, width=90, height=26, g=2e-4, nu=5e-3,
                           refill="geq")
    # periodic x and y (wrap-around pulls at both ends of a row), D3Q27, LES
    drop = inputs.drop_impact(n=32, pool=10, diameter=10.0, gap=8.0, speed=0.05, sigma=1e-3,
                              g=1e-5, nu=5e-3, nxy=30)
    drop["params"]["les_cs"] = 0.1
    # odd periodic width: a cell pair straddles the wrap
    wave = inputs.standing_wave(33, nz=2)
    # interior obstacle: the per-direction near-wall path inside a tile
    obst = inputs.dam_break(nx=70, ny=40, nz=3, width=20, height=26, g=2e-4, nu=5e-3,
                            refill="ext")
    o = np.zeros_like(obst["phi"], dtype=np.uint8)
    o[:, 0:6, 34:40] = 1
    obst["obstacle"] = o
    # free-slip walls (mirrored sources)
    fs = inputs.dam_break(nx=90, ny=50, nz=1, width=20, height=30, g=2e-4, nu=2e-3,
                          refill="avg")
    fs["params"]["periodic"] = (False, False, True)
    fs["params"]["free_slip"] = (True, True, False)
    return {"dam300": (dam, 150), "drop_les": (drop, 100), "wave33": (wave, 200),
            "obstacle": (obst, 120), "freeslip": (fs, 150)}


CASES = _cases()


def _state(sim):
    t = sim.types()
    fl = (t == 1) | (t == 2)
    return t, sim.pdfs()[:, fl], sim.phi(), sim.mass()[t == 1], sim.status()


@pytest.mark.parametrize("prec", ["fp16", "bf16", "fp32"])
@pytest.mark.parametrize("case", list(CASES))
def test_variants_bitwise_identical(fsl, prec, case):
    w, steps = CASES[case]
    ref = None
    for v in VARIANTS:
        if v in HALF_ONLY and prec == "fp32":
            continue
        sim = fsl.Sim(w["params"], prec)
        sim.set_variant(v)
        assert sim.variant() == fsl.VARIANTS[v]
        sim.init_workload(w)
        sim.step(steps)
        st = _state(sim)
        sim.close()
        if ref is None:
            ref = (v, st)
            continue
        for name, a, b in zip(("types", "pdfs", "phi", "mass", "status"), ref[1], st):
            assert np.array_equal(np.asarray(a), np.asarray(b)), (
                f"{case}/{prec}: variant {v} differs from {ref[0]} in {name}")


@pytest.mark.parametrize("v", HALF_ONLY)
def test_half_only_variants_rejected_for_fp32(fsl, v):
    w = inputs.standing_wave(32)
    sim = fsl.Sim(w["params"], "fp32")
    with pytest.raises(fsl.FslError):
        sim.set_variant(v)


@pytest.mark.parametrize("prec", ["fp16", "fp32"])
def test_kernel_stats_every_variant(fsl, prec):
    """The timed bulk kernel reports the same algorithmic bytes and liquid
    count whatever the variant, and a positive duration."""
    w = inputs.drop_impact(n=64, pool=20, diameter=16.0, gap=10.0, speed=0.05, sigma=1e-3,
                           g=1e-5, nu=5e-3, nxy=64)
    seen = None
    for v in VARIANTS:
        if v in HALF_ONLY and prec == "fp32":
            continue
        sim = fsl.Sim(w["params"], prec)
        sim.set_variant(v)
        sim.init_workload(w)
        sim.step(4)
        ks = sim.kernel_stats(reps=3)
        sim.close()
        assert ks["ms"] > 0
        key = (ks["bytes"], ks["n_liquid"])
        assert seen is None or key == seen, f"{v}: {key} vs {seen}"
        seen = key
