"""The hand-written discrete adjoint (fsl_adjoint_*): gradients of the
surface-elevation misfit against central finite differences of the GPU
forward run and of the FP64 CPU oracle, on a small standing wave whose
surface moves enough for cells to fill and empty, with checkpoints that cut
the run into several segments."""
import numpy as np
import pytest

import oracle
from paper_2207_14496_gb300 import adjoint, inputs

pytestmark = pytest.mark.gpu

STEPS, EVERY = 240, 70   # four segments, the last one short
NU, G = 0.01, 5e-4


def _setup(prec="fp64"):
    s = adjoint.wave_setup(L=32, ny=20, nz=2, depth=10.0, amp=0.64, steps=STEPS, every=EVERY,
                           precision=prec)
    rng = np.random.default_rng(14496)
    # target: a forward run with other parameters and a perturbed surface
    s["target"] = adjoint.elevation(s, NU * 1.1, G * 0.9, rng.normal(0.0, 0.1, 32))
    return s


def _J(s, nu, g, delta):
    a = adjoint.elevation(s, nu, g, delta)
    r = a - s["target"]
    return float(np.sum(r * r))


def _J_oracle(s, nu, g, delta):
    w = adjoint._workload(s, nu, g, delta)
    o = oracle.Oracle(w["params"])
    o.init_fill(w["phi"], h_ref=w["h_ref"])
    a = np.zeros(s["steps"])
    for t in range(s["steps"]):
        o.step(1)
        a[t] = o.column_height(0) - s["depth"]
    r = a - s["target"]
    return float(np.sum(r * r))


@pytest.fixture(scope="module")
def fp64_case(fsl):
    s = _setup("fp64")
    delta = np.random.default_rng(7).normal(0.0, 0.05, 32)
    res = adjoint.misfit_and_gradients(s, NU, G, delta)
    return s, delta, res


def test_run_converts_cells(fsl, fp64_case):
    """The checked run must exercise conversions, refilling and excess mass."""
    s, delta, res = fp64_case
    w = adjoint._workload(s, NU, G, delta)
    sim = fsl.Sim(w["params"], "fp64")
    sim.init_workload(w)
    total = 0
    for _ in range(s["steps"]):
        sim.step(1)
        c = sim.counts()
        total += c[0] + c[1]
    assert total > 5
    assert res["status"][0] == 0


def test_adjoint_matches_gpu_finite_differences(fsl, fp64_case):
    s, delta, res = fp64_case
    assert abs(res["J"] - _J(s, NU, G, delta)) <= 1e-12 * abs(res["J"])
    h = 1e-6 * NU
    fd_nu = (_J(s, NU + h, G, delta) - _J(s, NU - h, G, delta)) / (2 * h)
    assert res["dnu"] == pytest.approx(fd_nu, rel=1e-4, abs=1e-9 * abs(res["J"]) / NU)
    h = 1e-6 * G
    fd_g = (_J(s, NU, G + h, delta) - _J(s, NU, G - h, delta)) / (2 * h)
    assert res["dg"] == pytest.approx(fd_g, rel=1e-4, abs=1e-9 * abs(res["J"]) / G)
    scale = np.abs(res["ddelta"]).max()
    for i in (0, 5, 16, 27):
        e = np.zeros(32)
        e[i] = 1e-6
        fd = (_J(s, NU, G, delta + e) - _J(s, NU, G, delta - e)) / 2e-6
        assert res["ddelta"][i] == pytest.approx(fd, rel=1e-4, abs=1e-5 * scale), i


def test_adjoint_matches_oracle_reference_gradient(fsl, fp64_case):
    """The FP64 CPU oracle's central differences: the reference gradient."""
    s, delta, res = fp64_case
    h = 1e-6 * NU
    ref_nu = (_J_oracle(s, NU + h, G, delta) - _J_oracle(s, NU - h, G, delta)) / (2 * h)
    assert res["dnu"] == pytest.approx(ref_nu, rel=1e-4)
    h = 1e-6 * G
    ref_g = (_J_oracle(s, NU, G + h, delta) - _J_oracle(s, NU, G - h, delta)) / (2 * h)
    assert res["dg"] == pytest.approx(ref_g, rel=1e-4)


def test_fp32_adjoint_tracks_fp64(fsl, fp64_case):
    s64, delta, r64 = fp64_case
    s = dict(s64, precision="fp32")
    r32 = adjoint.misfit_and_gradients(s, NU, G, delta)
    assert r32["J"] == pytest.approx(r64["J"], rel=1e-3)
    assert r32["dnu"] == pytest.approx(r64["dnu"], rel=2e-2)
    assert r32["dg"] == pytest.approx(r64["dg"], rel=2e-2)
    assert np.allclose(r32["ddelta"], r64["ddelta"], rtol=5e-2,
                       atol=2e-2 * np.abs(r64["ddelta"]).max())


def test_autograd_function(fsl, fp64_case):
    import torch
    s, delta, res = fp64_case
    nu = torch.tensor(NU, dtype=torch.float64, requires_grad=True)
    g = torch.tensor(G, dtype=torch.float64, requires_grad=True)
    d = torch.tensor(delta, dtype=torch.float64, requires_grad=True)
    J = adjoint.WaveMisfit.apply(nu, g, d, s)
    (3.0 * J).backward()
    assert float(J.detach()) == pytest.approx(res["J"], rel=1e-13)
    assert float(nu.grad) == pytest.approx(3.0 * res["dnu"], rel=1e-12)
    assert float(g.grad) == pytest.approx(3.0 * res["dg"], rel=1e-12)
    assert np.allclose(d.grad.numpy(), 3.0 * res["ddelta"], rtol=1e-12)


def test_adjoint_rejects_unsupported_configurations(fsl):
    w = inputs.standing_wave(16, collision="trt")
    sim = fsl.Sim(w["params"], "fp64")
    sim.init_workload(w)
    with pytest.raises(fsl.FslError):
        fsl.Adjoint(sim, 10, 5)
    w = inputs.standing_wave(16)
    sim = fsl.Sim(w["params"], "fp16")
    sim.init_workload(w)
    with pytest.raises(fsl.FslError):
        fsl.Adjoint(sim, 10, 5)
