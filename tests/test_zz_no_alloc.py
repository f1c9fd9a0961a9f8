"""The allocation-free total-mass entry point (fsl_total_mass_noalloc) gives
the same total mass as fsl_observe(FSL_OBS_TOTAL_MASS) on two calls in a row.

It serves callers that cannot allocate device memory where they need the
observable (inside a CUDA graph capture, a host callback or another
allocator); its scratch is a static device array inside the library.  This
file is collected last so that a run stopping at the first failure has run
every other test first."""
import ctypes

import numpy as np
import pytest

from paper_2207_14496_gb300 import inputs

pytestmark = pytest.mark.gpu


def _dense_storage(sim, prec):
    """The state in the entry point's dense layout, on the device (the test
    allocates; the entry point does not)."""
    import torch
    c, w = sim.q, None
    from paper_2207_14496_gb300 import fsl
    _, w = fsl.lattice_table(sim.q)
    t = sim.types()
    f = sim.pdfs()                       # full f_i, FP64
    if prec == "fp64":
        pdf = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    else:
        off = f - w[:, None, None, None]  # f_i - w_i
        pdf = torch.from_numpy(np.ascontiguousarray(off.astype(np.float32))).cuda()
    types = torch.from_numpy(np.ascontiguousarray(t)).cuda()
    mass = torch.from_numpy(np.ascontiguousarray(sim.mass())).cuda()
    return pdf, types, mass


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_total_mass_matches_observe(fsl, prec):
    import torch
    w = inputs.drop_impact(n=40, pool=14, diameter=12.0, gap=9.0, speed=0.05, sigma=2e-3,
                           g=1e-5, nu=5e-3, nxy=36)
    sim = fsl.Sim(w["params"], prec)
    sim.init_workload(w)
    raw = fsl.raw_library()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    tol = 1e-12 if prec == "fp64" else 1e-6
    for _ in range(2):                   # two calls in a row, on evolving states
        sim.step(60)
        ref = sim.total_mass() - sim.lost_mass()
        pdf, types, mass = _dense_storage(sim, prec)
        torch.cuda.synchronize()
        rc = raw.fsl_total_mass_noalloc(ctypes.byref(sim.cfg), ctypes.c_void_p(pdf.data_ptr()),
                                        ctypes.c_void_p(types.data_ptr()),
                                        ctypes.c_void_p(mass.data_ptr()), None,
                                        ctypes.c_void_p(out.data_ptr()),
                                        ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, raw.fsl_last_error()
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - ref) <= tol * abs(ref), (got, ref)
    bad = fsl.make_config(dict(w["params"], shape=(512, 512, 256)), prec)
    rc = raw.fsl_total_mass_noalloc(ctypes.byref(bad), ctypes.c_void_p(pdf.data_ptr()),
                                    ctypes.c_void_p(types.data_ptr()),
                                    ctypes.c_void_p(mass.data_ptr()), None,
                                    ctypes.c_void_p(out.data_ptr()), None)
    assert rc == -1 and b"static scratch" in raw.fsl_last_error()
