"""Failure path of the bounded device waits, made without a fault: a wait at
the conversion phase's grid barrier for an arrival that never comes gives up
after its time bound, the handle reports FSL_ERR_TIMEOUT, the state is
otherwise unchanged, and the CUDA context keeps working for other handles."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TIMEOUT = -5  # FSL_ERR_TIMEOUT


def test_barrier_wait_gives_up_and_is_reported():
    from paper_2207_14496_gb300 import fsl, inputs
    w = inputs.standing_wave(32, nz=2)
    a = fsl.Sim(w["params"], "fp32")
    a.init_workload(w)
    a.step(20)
    assert a.status()[0] == 0
    phi0 = a.phi().copy()
    t0 = time.perf_counter()
    a.selftest_wait()
    waited = time.perf_counter() - t0
    assert 0.15 < waited < 5.0, waited
    assert a.status()[0] == TIMEOUT
    assert np.array_equal(a.phi(), phi0)
    # a fresh handle on the same context steps normally and matches a twin
    b = fsl.Sim(w["params"], "fp32")
    b.init_workload(w)
    b.step(20)
    assert b.status()[0] == 0
    assert np.array_equal(b.phi(), phi0)
