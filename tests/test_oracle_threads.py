"""The oracle's order-free per-cell loops (classes, stream/collide, refilling,
excess-mass gather, curvature) on several OpenMP threads give the results of
one thread bit for bit: every cell's arithmetic is independent of the order
in which cells are visited, and the loops that sum across cells or write
neighbours stay sequential."""
import numpy as np
import pytest

import oracle
from paper_2207_14496_gb300 import inputs


def _run(w, steps, threads):
    used = oracle.set_threads(threads)
    try:
        o = oracle.Oracle(w["params"])
        o.init_fill(w["phi"], w.get("u0"), w.get("obstacle"), w.get("h_ref", float("nan")))
        conv = 0
        for _ in range(steps):
            o.step(1)
            conv += sum(o.last_counts())
        return used, conv, (o.types(), o.pdfs(), o.phi(), o.mass(), o.kappa(),
                            o.total_mass(), o.unstable_step)
    finally:
        oracle.set_threads(1)


def _same(a, b):
    for x, y in zip(a, b):
        if isinstance(x, np.ndarray):
            assert np.array_equal(x, y)
        else:
            assert x == y


@pytest.mark.parametrize("scheme", inputs.REFILL_SCHEMES)
def test_dam_break_threads_bitwise(scheme):
    w = inputs.dam_break(nx=40, ny=24, nz=3, width=12, height=14, g=2e-4, nu=5e-3, refill=scheme)
    _, conv1, a = _run(w, 60, 1)
    used, conv4, b = _run(w, 60, 4)
    assert conv1 == conv4 and conv1 > 20
    _same(a, b)
    if used == 1:
        pytest.skip("oracle built without OpenMP: both runs were sequential")


def test_drop_impact_with_curvature_threads_bitwise():
    w = inputs.drop_impact(n=28, pool=10, diameter=10.0, gap=6.0, speed=0.05, sigma=1e-3,
                           g=1e-5, nu=5e-3)
    _, conv1, a = _run(w, 50, 1)
    _, conv3, b = _run(w, 50, 3)
    assert conv1 == conv3 and conv1 > 20
    assert np.abs(a[4]).max() > 0.0  # curvature in play
    _same(a, b)
