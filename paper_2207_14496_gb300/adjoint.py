"""Gradients of a surface-elevation misfit of the standing wave (Sec. 4.1)
with respect to the viscosity, the gravity and per-column perturbations of
the initial surface, through the library's hand-written discrete adjoint
(fsl_adjoint_* in include/fsl.h), exposed as a torch.autograd.Function.

    J(nu, g, delta) = sum_{t=1..T} (a(t) - a_target(t))^2,
    a(t) = column height at x = 0 after step t minus the depth d,

for the wave L x ny x nz with surface h(x) = d + a0 cos(2 pi x / L) + delta_x.
The initial fill levels depend on delta through the cell averages of the
geometry builder (inputs.wave_fill); their derivative
(inputs.wave_fill_dperturb) carries the adjoint's d J / d phi0 to d J / d delta.
Gravity points along -y with magnitude g, so d J / d g = -d J / d g_y.
"""
from __future__ import annotations

import numpy as np
import torch

from . import fsl, inputs


def wave_setup(L: int = 128, ny: int = 64, nz: int = 4, depth: float = 32.0, amp=None,
               steps: int = 1500, every: int = 100, precision: str = "fp64",
               target=None) -> dict:
    """The misfit's fixed ingredients: geometry, step count, checkpoint
    interval, precision and target trace (zeros if none)."""
    return dict(L=L, ny=ny, nz=nz, depth=depth, amp=0.01 * L if amp is None else amp,
                steps=steps, every=every, precision=precision,
                target=np.zeros(steps) if target is None else np.asarray(target, float))


def _workload(s: dict, nu: float, g: float, delta):
    return inputs.standing_wave(s["L"], nz=s["nz"], depth=s["depth"], amp=s["amp"], nu=nu, g=g,
                                perturb=delta, ny=s["ny"])


def elevation(s: dict, nu: float, g: float, delta, device: int = 0) -> np.ndarray:
    """a(t), t = 1..T, from a forward run of the library (no adjoint)."""
    w = _workload(s, nu, g, delta)
    sim = fsl.Sim(w["params"], s["precision"], device=device)
    sim.init_workload(w)
    sim.set_trace(1)
    sim.step(s["steps"])
    tr = sim.trace(s["steps"])
    sim.close()
    return tr[:, 0] - s["depth"]


def misfit_and_gradients(s: dict, nu: float, g: float, delta, device: int = 0) -> dict:
    """J and its gradients with respect to nu, g and delta (one forward and one
    adjoint pass on the GPU)."""
    delta = np.zeros(s["L"]) if delta is None else np.asarray(delta, dtype=np.float64)
    w = _workload(s, nu, g, delta)
    sim = fsl.Sim(w["params"], s["precision"], device=device)
    sim.init_workload(w)
    adj = fsl.Adjoint(sim, s["steps"], s["every"])
    a = adj.forward() - s["depth"]
    r = a - s["target"]
    J = float(np.sum(r * r))
    out = adj.backward(2.0 * r)
    dphi = inputs.wave_fill_dperturb(s["L"], s["ny"], s["depth"], s["amp"], s["L"], delta)
    # d J / d delta_x = sum over y, z of d J / d phi0(z, y, x) d phi0(y, x) / d delta_x
    ddelta = np.einsum("zyx,yx->x", out["dphi0"], dphi)
    res = dict(J=J, a=a, dnu=out["nu"], dg=-float(out["g"][1]), ddelta=ddelta,
               status=sim.status())
    adj.close()
    sim.close()
    return res


class WaveMisfit(torch.autograd.Function):
    """J(nu, g, delta) for the setup `s` (wave_setup); nu and g are 0-d float64
    tensors, delta a length-L float64 tensor.  backward runs the adjoint."""

    @staticmethod
    def forward(ctx, nu, g, delta, s):
        r = misfit_and_gradients(s, float(nu), float(g), delta.detach().cpu().numpy())
        ctx.grads = (r["dnu"], r["dg"], r["ddelta"])
        return torch.tensor(r["J"], dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        dnu, dg, dd = ctx.grads
        k = float(gJ)
        return (torch.tensor(k * dnu, dtype=torch.float64),
                torch.tensor(k * dg, dtype=torch.float64),
                torch.from_numpy(k * dd), None)
