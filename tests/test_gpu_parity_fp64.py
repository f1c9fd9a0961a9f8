"""FP64 CUDA path vs the CPU oracle, element by element.

The bar: cell types bit-exact; stored PDFs, fill levels and interface masses
within 1e-12 relative (the FP64 kernels follow the oracle's operation order
without multiply-add contraction, so in practice they agree bit for bit).
Sizes are chosen so that the oracle finishes in seconds while the grids span
several thread blocks and have ragged x tails (nx not a multiple of 32)."""
import numpy as np
import pytest

from paper_2207_14496_gb300 import inputs
from parity_util import compare_state, make_pair, run_parity

pytestmark = pytest.mark.gpu
RTOL = 1e-12


def test_standing_wave_64_full_run(fsl):
    """Standing wave 64x64x1, D3Q19 SRT, EQ refilling, all 2000 steps."""
    w = inputs.standing_wave(64)
    sim, orc, stats, conv = run_parity(fsl, w, 2000, 250, RTOL, "wave64")
    assert conv > 0, "the wave must convert cells for the check to cover conversion"
    m0 = stats[0]


@pytest.mark.parametrize("scheme", inputs.REFILL_SCHEMES)
def test_dam_break_small_all_schemes(fsl, scheme):
    """Dam break 100x48x4 (ragged x tail), D3Q19 TRT, walls on all faces,
    strong gravity so that many cells fill and empty: every refill scheme."""
    w = inputs.dam_break(nx=100, ny=48, nz=4, width=24, height=24, g=2e-4, nu=5e-3,
                         refill=scheme)
    sim, orc, stats, conv = run_parity(fsl, w, 300, 50, RTOL, f"dam/{scheme}")
    assert conv > 50


def test_drop_impact_small_d3q27_surface_tension(fsl):
    """Drop into a pool, 40x40x40 D3Q27 TRT with surface tension (curvature and
    Laplace pressure), periodic x/y, walls in z, initial drop velocity."""
    w = inputs.drop_impact(n=40, pool=14, diameter=12.0, gap=9.0, speed=0.05, sigma=2e-3,
                           g=1e-5, nu=5e-3, nxy=36)
    sim, orc, stats, conv = run_parity(fsl, w, 150, 50, RTOL, "drop27")
    assert conv > 0
    k_g, k_o = sim.kappa(), orc.kappa()
    iface = orc.types() == 1
    assert np.allclose(k_g[iface], k_o[iface], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("scheme", ["eq_neq", "geq", "ext", "avg"])
def test_drop_impact_schemes_d3q27(fsl, scheme):
    w = inputs.drop_impact(n=32, pool=10, diameter=10.0, gap=8.0, speed=0.05, sigma=1e-3,
                           g=1e-5, nu=5e-3, refill=scheme, nxy=30)
    run_parity(fsl, w, 80, 40, RTOL, f"drop27/{scheme}")


def test_obstacle_and_options(fsl):
    """Interior obstacle block (bounce-back, narrowed normals) with the literal
    readings switched on (simple flux, literal GEQ/NEQ/Laplace)."""
    w = inputs.dam_break(nx=70, ny=40, nz=3, width=20, height=26, g=2e-4, nu=5e-3,
                         refill="geq")
    obst = np.zeros_like(w["phi"], dtype=np.uint8)
    obst[:, 0:6, 34:40] = 1
    w["obstacle"] = obst
    w["params"]["options"] = 1 | 2 | 4 | 8
    w["params"]["sigma"] = 1e-4
    run_parity(fsl, w, 200, 50, RTOL, "obstacle")


def test_static_drop_curvature(fsl):
    w = inputs.static_drop(n=24, radius=6.0, sigma=1e-3, nu=0.05)
    sim, orc, stats, conv = run_parity(fsl, w, 60, 30, RTOL, "static_drop")
    iface = orc.types() == 1
    assert np.allclose(sim.kappa()[iface], orc.kappa()[iface], rtol=1e-12, atol=1e-14)


def test_tiny_and_degenerate_domains(fsl):
    """nx = 1 periodic column and a 3-wide domain: wrap-around onto itself."""
    w = inputs.standing_wave(16, nz=1)
    w["params"]["shape"] = (1, 16, 1)
    w["phi"] = np.ascontiguousarray(w["phi"][:, :, :1])
    run_parity(fsl, w, 100, 50, RTOL, "column")
    w = inputs.dam_break(nx=3, ny=20, nz=2, width=2, height=10, g=1e-4, nu=1e-2)
    run_parity(fsl, w, 100, 50, RTOL, "narrow")


def test_no_interface_fully_liquid(fsl):
    """Poiseuille channel: no interface cells at all (empty lists every step)."""
    w = inputs.poiseuille(ny=20, nx=40)
    run_parity(fsl, w, 200, 100, RTOL, "poiseuille")


def test_empty_domain_all_gas(fsl):
    w = inputs.standing_wave(32)
    w["phi"] = np.zeros_like(w["phi"])
    sim, orc = make_pair(fsl, w)
    sim.step(10)
    orc.step(10)
    compare_state(sim, orc, 10, RTOL, label="empty")
    assert sim.total_mass() == 0.0


def test_unstable_latch_matches_oracle(fsl):
    """Gravity large enough that |u| reaches c_s: both sides latch the same
    first unstable step and freeze."""
    w = inputs.dam_break(nx=40, ny=40, nz=1, width=12, height=30, g=5e-2, nu=1e-2)
    w["params"]["periodic"] = (False, False, True)
    sim, orc = make_pair(fsl, w)
    orc.step(400)
    sim.step(400)
    assert orc.unstable_step > 0
    st, first = sim.status()
    assert st == fsl.ERR_UNSTABLE and first == orc.unstable_step
    compare_state(sim, orc, orc.step_count, RTOL, label="unstable")


def test_dam_break_512_full_size_prefix(fsl):
    """The 512x256x16 D3Q19 TRT dam break at full size: every cell compared
    after 12 steps, in the launch configuration the benchmark uses."""
    w = inputs.dam_break()
    sim, orc = make_pair(fsl, w)
    sim.step(12)
    orc.step(12)
    compare_state(sim, orc, 12, RTOL, label="dam512")


def test_drop_impact_256_full_size_sampled(fsl):
    """256^3 D3Q27 drop impact (FP64): 2 steps, every cell compared."""
    w = inputs.drop_impact()
    sim, orc = make_pair(fsl, w)
    sim.step(2)
    orc.step(2)
    compare_state(sim, orc, 2, RTOL, label="drop256")


@pytest.mark.parametrize("scheme", inputs.REFILL_SCHEMES)
def test_free_slip_les_dam_break(fsl, scheme):
    """The paper's dam-break walls and turbulence model (Sec. 4.2): free-slip
    walls on x and y (specular reflection, mirrored mass flux), Smagorinsky
    C_S = 0.1, D3Q19 TRT, 2D (periodic z, nz = 1), every refilling scheme."""
    w = inputs.dam_break(nx=90, ny=50, nz=1, width=20, height=30, g=2e-4, nu=2e-3,
                         refill=scheme)
    w["params"]["periodic"] = (False, False, True)
    w["params"]["free_slip"] = (True, True, False)
    w["params"]["les_cs"] = 0.1
    sim, orc, stats, conv = run_parity(fsl, w, 300, 100, RTOL, f"freeslip/{scheme}")
    assert conv > 50


def test_free_slip_3d_mixed_walls_d3q27(fsl):
    """3D: free-slip x walls, no-slip y and z walls (mixed edges and corners
    fall back to bounce-back), D3Q27 with LES."""
    w = inputs.dam_break(nx=40, ny=30, nz=12, width=12, height=18, g=2e-4, nu=3e-3, q=27)
    w["params"]["free_slip"] = (True, False, False)
    w["params"]["les_cs"] = 0.1
    run_parity(fsl, w, 120, 60, RTOL, "freeslip3d")
