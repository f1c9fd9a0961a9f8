"""Helpers shared by the parity tests: run a workload on the CUDA library and on
the CPU oracle with identical inputs and compare their states."""
from __future__ import annotations

import numpy as np

import oracle

GAS, IFACE, LIQUID, OBST = 0, 1, 2, 3


def make_pair(fsl, w: dict, precision: str = "fp64"):
    sim = fsl.Sim(w["params"], precision)
    sim.init_workload(w)
    orc = oracle.Oracle(w["params"])
    orc.init_fill(w["phi"], w.get("u0"), w.get("obstacle"), w.get("h_ref", float("nan")))
    return sim, orc


def first_mismatch(a: np.ndarray, b: np.ndarray):
    idx = np.argwhere(a != b)
    if idx.size == 0:
        return None
    k = tuple(idx[0])
    return k, a[k], b[k], int(idx.shape[0])


def compare_state(sim, orc, step: int, rtol: float = 1e-12, atol: float = 1e-15,
                  label: str = "", atol_fill: float | None = None) -> dict:
    """Flags bit-exact; PDFs (fluid cells), fill level (all cells) and mass
    (interface cells) within rtol relative (plus atol; atol_fill, when given,
    replaces atol for the fill level and the mass).  Returns error
    statistics."""
    tg, to = sim.types(), orc.types()
    mm = first_mismatch(tg, to)
    assert mm is None, f"{label} step {step}: cell types differ at (z,y,x)={mm[0]}: gpu {mm[1]} oracle {mm[2]} ({mm[3]} cells)"
    fluid = (to == IFACE) | (to == LIQUID)
    iface = to == IFACE
    fg, fo = sim.pdfs()[:, fluid], orc.pdfs()[:, fluid]
    err_f = np.abs(fg - fo)
    bound_f = rtol * np.abs(fo) + atol
    bad = err_f > bound_f
    assert not bad.any(), (f"{label} step {step}: PDFs differ, max rel "
                           f"{float((err_f / (np.abs(fo) + 1e-300)).max()):.3e}")
    af = atol if atol_fill is None else atol_fill
    pg, po = sim.phi(), orc.phi()
    err_p = np.abs(pg - po)
    assert (err_p <= rtol * np.abs(po) + af).all(), (
        f"{label} step {step}: fill level differs, max abs {float(err_p.max()):.3e}")
    mg, mo = sim.mass()[iface], orc.mass()[iface]
    err_m = np.abs(mg - mo)
    assert (err_m <= rtol * np.abs(mo) + af).all(), (
        f"{label} step {step}: interface mass differs, max abs {float(err_m.max()):.3e}")
    return dict(bitwise_pdf=bool((fg == fo).all()), max_pdf_err=float(err_f.max(initial=0.0)),
                max_phi_err=float(err_p.max(initial=0.0)), n_if=int(iface.sum()))


def run_parity(fsl, w: dict, steps: int, every: int, rtol: float = 1e-12, label: str = ""):
    sim, orc = make_pair(fsl, w)
    stats = [compare_state(sim, orc, 0, rtol, label=label)]
    done = 0
    conversions = 0
    while done < steps:
        k = min(every, steps - done)
        for _ in range(k):
            orc.step(1)
            c = orc.last_counts()
            conversions += c[0] + c[1] + c[2]
        sim.step(k)
        done += k
        stats.append(compare_state(sim, orc, done, rtol, label=label))
    assert sim.step_count == orc.step_count
    assert sim.status()[1] == orc.unstable_step
    return sim, orc, stats, conversions
