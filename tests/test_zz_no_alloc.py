"""The allocation-free total-mass entry point (fsl_total_mass_noalloc) gives
the same total mass as fsl_observe(FSL_OBS_TOTAL_MASS) on two calls in a row,
for every storage and with or without a per-cell lost-mass array.

It serves callers that cannot allocate device memory where they need the
observable (inside a host callback or another allocator, or under a fixed
device-memory budget); its scratch is a static device array inside the
library.  This file is collected last so that a run stopping at the first
failure has run every other test first."""
import ctypes

import numpy as np
import pytest

from paper_2207_14496_gb300 import inputs

pytestmark = pytest.mark.gpu

# both sides sum the same decoded FP64 values, in different orders
RTOL = 1e-11


def _dense_storage(sim, prec):
    """The state in the entry point's dense layout and storage, on the device
    (the test allocates; the entry point does not): FP64 f_i, FP32 and BF16
    f_i - w_i, FP16 (f_i - w_i) 2^15.  Re-encoding the decoded values gives
    back the stored ones exactly."""
    import torch
    from paper_2207_14496_gb300 import fsl
    _, w = fsl.lattice_table(sim.q)
    f = sim.pdfs()
    if prec == "fp64":
        pdf = torch.from_numpy(np.ascontiguousarray(f))
    else:
        off = torch.from_numpy(np.ascontiguousarray(f - w[:, None, None, None]))
        if prec == "fp32":
            pdf = off.float()
        elif prec == "fp16":
            pdf = (off * 32768.0).half()
        else:
            pdf = off.bfloat16()
    types = torch.from_numpy(np.ascontiguousarray(sim.types()))
    mass = torch.from_numpy(np.ascontiguousarray(sim.mass()))
    return pdf.contiguous().cuda(), types.cuda(), mass.cuda()


@pytest.mark.parametrize("with_lost", [False, True])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16", "bf16"])
def test_noalloc_total_mass_matches_observe(fsl, prec, with_lost):
    import torch
    w = inputs.drop_impact(n=40, pool=14, diameter=12.0, gap=9.0, speed=0.05, sigma=2e-3,
                           g=1e-5, nu=5e-3, nxy=36)
    sim = fsl.Sim(w["params"], prec)
    sim.init_workload(w)
    raw = fsl.raw_library()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    n = int(np.prod(w["params"]["shape"]))
    rng = np.random.default_rng(7)
    lost = torch.from_numpy(rng.uniform(0.0, 1e-3, n)).cuda() if with_lost else None
    for _ in range(2):                   # two calls in a row, on evolving states
        sim.step(60)
        ref = sim.total_mass() - sim.lost_mass()
        if with_lost:
            ref += float(lost.sum().item())
        pdf, types, mass = _dense_storage(sim, prec)
        torch.cuda.synchronize()
        rc = raw.fsl_total_mass_noalloc(
            ctypes.byref(sim.cfg), ctypes.c_void_p(pdf.data_ptr()),
            ctypes.c_void_p(types.data_ptr()), ctypes.c_void_p(mass.data_ptr()),
            ctypes.c_void_p(lost.data_ptr()) if with_lost else None,
            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, raw.fsl_last_error()
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - ref) <= RTOL * abs(ref), (got, ref)
    bad = fsl.make_config(dict(w["params"], shape=(512, 512, 256)), prec)
    rc = raw.fsl_total_mass_noalloc(ctypes.byref(bad), ctypes.c_void_p(pdf.data_ptr()),
                                    ctypes.c_void_p(types.data_ptr()),
                                    ctypes.c_void_p(mass.data_ptr()), None,
                                    ctypes.c_void_p(out.data_ptr()), None)
    assert rc == -1 and b"static scratch" in raw.fsl_last_error()
