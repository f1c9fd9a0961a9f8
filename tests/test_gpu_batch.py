"""Batched stepping (fsl_batch_*): every member of a batch ends bit-identical
to the same simulation stepped alone, whatever the chunking, with members of
different sizes, schemes and variants, and with per-member work interleaved."""
import numpy as np
import pytest

from paper_2207_14496_gb300 import inputs

pytestmark = pytest.mark.gpu


def _members():
    out = []
    for k, spec in enumerate(inputs.batched_waves(seed=7, n_geom=3)[:9]):
        lam = 24 + 8 * (spec["lam"] % 5)
        w = inputs.standing_wave(lam, nz=spec["width"], nu=spec["nu"], refill=spec["refill"])
        out.append(w)
    return out


def _state(sim):
    t = sim.types()
    fl = (t == 1) | (t == 2)
    return t, sim.pdfs()[:, fl], sim.phi(), sim.mass()[t == 1], sim.step_count


def _same(a, b, label):
    for name, x, y in zip(("types", "pdfs", "phi", "mass", "steps"), a, b):
        assert np.array_equal(np.asarray(x), np.asarray(y)), f"{label}: {name} differs"


@pytest.mark.parametrize("prec", ["fp16", "fp64"])
def test_batch_matches_individual_runs(fsl, prec):
    ws = _members()
    solo = []
    for w in ws:
        s = fsl.Sim(w["params"], prec)
        s.init_workload(w)
        s.step(75)
        solo.append(_state(s))
        s.close()
    sims = []
    for i, w in enumerate(ws):
        s = fsl.Sim(w["params"], prec)
        if prec != "fp64":
            s.set_variant(["pair", "pair_r128", "tma", "quad64", "warp_tma", "pair_pipe"][i % 6])
        s.init_workload(w)
        sims.append(s)
    b = fsl.Batch(sims, chunk=8)
    b.step(75)  # 9 graphs of 8 steps + one of 3
    for i, s in enumerate(sims):
        _same(solo[i], _state(s), f"member {i}")
    b.close()


def test_batch_interleaved_with_member_work_and_reinit(fsl):
    ws = _members()[:4]
    sims = []
    for w in ws:
        s = fsl.Sim(w["params"], "fp16")
        s.init_workload(w)
        sims.append(s)
    b = fsl.Batch(sims, chunk=16)
    b.step(20)
    sims[1].step(7)       # member work between batch steps
    sims[2].init_workload(ws[2])  # re-initialised member: recaptured
    b.step(20)
    expect_steps = [40, 47, 20, 40]
    for i, w in enumerate(ws):
        r = fsl.Sim(w["params"], "fp16")
        r.init_workload(w)
        r.step(expect_steps[i])
        _same(_state(r), _state(sims[i]), f"member {i}")
        r.close()
    b.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batch_with_bubble_model_matches_individual_runs(fsl, prec):
    """Members with the bubble model (both connectivity readings) beside a
    member without it: bubble labels and pressures equal the solo runs bit
    for bit."""
    ws = [inputs.bubbles_in_pool(), inputs.bubbles_in_pool(nx=36, ny=34, depth=28,
                                                          bubbles=((14.0, 9.0, 5.0), (26.0, 9.0, 5.0)),
                                                          g=4e-4),
          _members()[0]]
    ws[1]["params"]["options"] = 48
    solo = []
    for w in ws:
        s = fsl.Sim(w["params"], prec)
        s.init_workload(w)
        s.step(90)
        solo.append(_state(s) + (s.bubbles(), s.pressure()))
        s.close()
    sims = []
    for w in ws:
        s = fsl.Sim(w["params"], prec)
        s.init_workload(w)
        sims.append(s)
    b = fsl.Batch(sims, chunk=16)
    b.step(90)
    for i, s in enumerate(sims):
        st = _state(s) + (s.bubbles(), s.pressure())
        _same(solo[i][:5], st[:5], f"member {i}")
        assert np.array_equal(solo[i][5], st[5]), f"member {i}: bubble labels differ"
        assert np.array_equal(solo[i][6], st[6]), f"member {i}: pressures differ"
    b.close()


def test_batch_fp16_members_track_fp64(fsl):
    """FP16 members of a batch (one launch per kernel for all of them) against
    the FP64 path, PDF by PDF after 20 steps: within 20 half-ulps of FP16
    (2^-11) of the largest offset |f - w|, cell types equal."""
    ws = _members()
    sims = []
    for w in ws:
        s = fsl.Sim(w["params"], "fp16")
        s.init_workload(w)
        sims.append(s)
    b = fsl.Batch(sims, chunk=8)
    b.step(20)
    _, wts = fsl.lattice_table(19)
    for i, w in enumerate(ws):
        r = fsl.Sim(w["params"], "fp64")
        r.init_workload(w)
        r.step(20)
        t = r.types()
        assert np.array_equal(t, sims[i].types()), i
        fl = (t == 1) | (t == 2)
        fa, fb = r.pdfs()[:, fl], sims[i].pdfs()[:, fl]
        off = np.abs(fa - wts[:, None]).max()
        assert np.abs(fa - fb).max() <= 20 * 2.0 ** -11 * off, i
        r.close()
    b.close()


def test_batch_of_many_members_and_two_lattices(fsl):
    """More members than one launch takes (256), of two lattices: every
    member equals its solo run bit for bit."""
    ws = []
    for k in range(300):
        q = 27 if k % 7 == 0 else 19
        ws.append(inputs.standing_wave(16 + 2 * (k % 5), nz=1 + k % 2, q=q,
                                       refill=inputs.REFILL_SCHEMES[k % 5]))
    sims = []
    for w in ws:
        s = fsl.Sim(w["params"], "fp16")
        s.init_workload(w)
        sims.append(s)
    b = fsl.Batch(sims, chunk=16)
    b.step(16)
    for i in range(0, 300, 23):
        r = fsl.Sim(ws[i]["params"], "fp16")
        r.init_workload(ws[i])
        r.step(16)
        _same(_state(r), _state(sims[i]), f"member {i}")
        r.close()
    b.close()
    for s in sims:
        s.close()
