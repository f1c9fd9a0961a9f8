"""The hand-written adjoint on the full standing-wave gradient case: a wave
128 x 64 x 4 (wavelength 128, depth 32, amplitude 1.28, g = 1e-5,
nu = 0.01), 1500 steps, checkpoints every 100 steps, gradients of the
squared elevation misfit at x = 0 with respect to nu, g and the 128 surface
perturbations, against a target trace from a forward run with seed 14496
(perturbations N(0, 0.1), nu x 1.1, g x 0.9).  Checked against central
differences of the GPU forward run (eps 1e-6, relative for nu and g,
absolute cells for the perturbations) on nu, g and 16 perturbations, against
central differences of the FP64 CPU oracle on nu, g and 3 perturbations,
and FP32 against FP64.

    FSL_LONG_PARITY=1 python -m pytest tests/test_long_adjoint.py -m gpu -q

Skipped unless FSL_LONG_PARITY is set; FSL_LONG_PARITY_OUT=<dir> receives
the record as JSON."""
import json
import os
import time

import numpy as np
import pytest

import oracle
from paper_2207_14496_gb300 import adjoint

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not os.environ.get("FSL_LONG_PARITY"),
                                 reason="long runs: set FSL_LONG_PARITY=1")]

NU, G, L = 0.01, 1e-5, 128
RTOL = 1e-3


def _setup(prec):
    s = adjoint.wave_setup(L=L, ny=64, nz=4, depth=32.0, amp=1.28, steps=1500, every=100,
                           precision=prec)
    rng = np.random.default_rng(14496)
    s["target"] = adjoint.elevation(dict(s, precision="fp64"), NU * 1.1, G * 0.9,
                                    rng.normal(0.0, 0.1, L))
    return s


def _J(s, nu, g, delta):
    r = adjoint.elevation(s, nu, g, delta) - s["target"]
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


def test_adjoint_wave_128_1500_steps(fsl):
    t0 = time.time()
    s = _setup("fp64")
    delta = np.random.default_rng(7).normal(0.0, 0.05, L)
    res = adjoint.misfit_and_gradients(s, NU, G, delta)
    rec = dict(case="adjoint_wave_128x64x4_1500", J=res["J"], status=list(res["status"]),
               checks={})
    assert res["status"][0] == 0
    assert abs(res["J"] - _J(s, NU, G, delta)) <= 1e-12 * abs(res["J"])
    scale = float(np.abs(res["ddelta"]).max())

    def check(name, got, ref, floor):
        # perturbations far from x = 0 do not reach the observed column in
        # 1500 steps: a zero gradient has only an absolute error
        err = abs(got - ref)
        rec["checks"][name] = dict(adjoint=float(got), reference=float(ref), abs_err=float(err),
                                   rel_err=float(err / abs(ref)) if abs(ref) > floor else None)
        return err <= RTOL * abs(ref) + floor

    ok = True
    h = 1e-6 * NU
    ok &= check("gpu_fd_nu", res["dnu"], (_J(s, NU + h, G, delta) - _J(s, NU - h, G, delta)) / (2 * h),
                1e-9 * abs(res["J"]) / NU)
    h = 1e-6 * G
    ok &= check("gpu_fd_g", res["dg"], (_J(s, NU, G + h, delta) - _J(s, NU, G - h, delta)) / (2 * h),
                1e-9 * abs(res["J"]) / G)
    for i in range(0, L, 8):
        e = np.zeros(L)
        e[i] = 1e-6
        fd = (_J(s, NU, G, delta + e) - _J(s, NU, G, delta - e)) / 2e-6
        ok &= check(f"gpu_fd_delta_{i}", res["ddelta"][i], fd, 1e-4 * scale)
    threads = oracle.set_threads(os.cpu_count() or 1)
    try:
        h = 1e-6 * NU
        ok &= check("oracle_fd_nu", res["dnu"],
                    (_J_oracle(s, NU + h, G, delta) - _J_oracle(s, NU - h, G, delta)) / (2 * h),
                    1e-9 * abs(res["J"]) / NU)
        h = 1e-6 * G
        ok &= check("oracle_fd_g", res["dg"],
                    (_J_oracle(s, NU, G + h, delta) - _J_oracle(s, NU, G - h, delta)) / (2 * h),
                    1e-9 * abs(res["J"]) / G)
        for i in (0, 40, 100):
            e = np.zeros(L)
            e[i] = 1e-6
            fd = (_J_oracle(s, NU, G, delta + e) - _J_oracle(s, NU, G, delta - e)) / 2e-6
            ok &= check(f"oracle_fd_delta_{i}", res["ddelta"][i], fd, 1e-4 * scale)
    finally:
        oracle.set_threads(1)
    r32 = adjoint.misfit_and_gradients(dict(s, precision="fp32"), NU, G, delta)
    rec["fp32_vs_fp64"] = dict(
        J_rel=abs(r32["J"] - res["J"]) / abs(res["J"]),
        dnu_rel=abs(r32["dnu"] - res["dnu"]) / abs(res["dnu"]),
        dg_rel=abs(r32["dg"] - res["dg"]) / abs(res["dg"]),
        ddelta_max_rel_to_scale=float(np.abs(r32["ddelta"] - res["ddelta"]).max() / scale))
    rec["oracle_threads"] = threads
    rec["seconds"] = time.time() - t0
    out = os.environ.get("FSL_LONG_PARITY_OUT")
    if out:
        os.makedirs(out, exist_ok=True)
        with open(os.path.join(out, "adjoint_wave_128.json"), "w") as fh:
            json.dump(rec, fh, indent=1)
    assert ok, rec["checks"]
    assert rec["fp32_vs_fp64"]["J_rel"] < 1e-3
    assert rec["fp32_vs_fp64"]["dnu_rel"] < 2e-2 and rec["fp32_vs_fp64"]["dg_rel"] < 2e-2
    assert rec["fp32_vs_fp64"]["ddelta_max_rel_to_scale"] < 5e-2
