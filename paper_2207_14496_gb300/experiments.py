"""Paper-scale experiments run on the CUDA library.

`dam_break` runs the rectangular dam break of Sec. 4.2 (free-slip walls,
Smagorinsky model, W in {50, 100, 200}) and reports the residual height and
front position over time and any instability.

`taylor_bubble` runs the Taylor bubble of Sec. 4.4 (D in {32, 64, 128},
bubble model on) and reports the Reynolds number of the rise velocity taken
from the bubble's centre of mass at t* = 10 and t* = 15, beside the paper's
printed values.

`bubbly_poiseuille` runs the bubbly plane Poiseuille flow of Sec. 4.6 (381
bubbles in a force-driven channel) and reports how the bubbles gather and
coalesce and which schemes go unstable.

`batched_waves` runs the set of 320 small independent wave domains as one
batch and as one launch per domain.

`drop_impact_precision` runs the drop impact of Sec. 4.5 (the benchmark
workload) in FP64, FP32, FP16 and BF16 storage and reports the total-mass
drift, the cavity depth and the crown inner diameter of each against FP64.

`gravity_wave` reproduces the standing gravity wave of Sec. 4.1 at the
paper's resolutions (L in {200, 400, 800}, omega = 1.8, Re = 10, d = L/2,
a0 = 0.01 L, D3Q19 SRT) for the five refilling schemes and evaluates the
half period T*/2 and the logarithmic decrement delta of the surface elevation
at x = 0, as the paper does.  The printed L = 800 values of the paper are
returned beside them as context (a different implementation, waLBerla on CPU).

    python -m paper_2207_14496_gb300.experiments --L 200 400 800
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import inputs

# values printed in Sec. 4.1 (figures of the half period and of the logarithmic
# decrement) for L = 800; EXT has no decrement (irregular amplitudes)
PAPER_L800 = {
    "half_period": {"eq": 3.184, "eq_neq": 3.187, "geq": 3.172, "ext": 3.495, "avg": 3.161},
    "log_decrement": {"eq": 0.404, "eq_neq": 0.429, "geq": 0.405, "avg": 0.336},
    "analytic_half_period": math.pi,
    "analytic_log_decrement": 0.4961,
}


def wave_setting(L: int, omega: float = 1.8, re: float = 10.0):
    nu = (1.0 / 3.0) * (1.0 / omega - 0.5)
    k = 2.0 * math.pi / L
    d = L / 2.0
    a0 = 0.01 * L
    w0 = re * nu / (a0 * L)
    g = w0 * w0 / (k * math.tanh(k * d))
    return dict(nu=nu, k=k, d=d, a0=a0, omega0=w0, g=g)


def _smooth(a, k: int = 5):
    """Centred moving average over k samples (t* = 0.05 at the monitoring
    interval): removes the one-sample jitter that conversions add."""
    if len(a) < k:
        return a
    pad = np.pad(a, (k // 2, k // 2), mode="edge")
    return np.convolve(pad, np.ones(k) / k, mode="valid")


def _crossings(t, a):
    """Times where a changes sign, linearly interpolated."""
    s = np.sign(a)
    idx = np.nonzero(s[1:] * s[:-1] < 0)[0]
    return t[idx] - a[idx] * (t[idx + 1] - t[idx]) / (a[idx + 1] - a[idx])


def gravity_wave(L: int, scheme: str, precision: str = "fp64", periods: float = 1.15,
                 device: int = 0, save_trace: str | None = None):
    """Run one wave and evaluate its first half period and first decrement."""
    from . import fsl
    s = wave_setting(L)
    w = inputs.standing_wave(L, nu=s["nu"], g=s["g"], refill=scheme)
    sim = fsl.Sim(w["params"], precision, device=device)
    sim.init_workload(w)
    a_init = (sim.column_height() - s["d"]) / s["a0"]
    every = max(1, int(round(0.01 / s["omega0"])))  # monitored every t* = 0.01
    sim.set_trace(every)
    steps_total = int(periods * 2 * math.pi / s["omega0"])
    chunk = every * 4096
    done = 0
    trace = []
    t0 = time.perf_counter()
    while done < steps_total:
        k = min(chunk, steps_total - done)
        k -= k % every
        if k <= 0:
            break
        sim.step(k)
        done += k
        n = k // every
        trace.append(sim.trace(n))
        sim.set_trace(every)
    wall = time.perf_counter() - t0
    tr = np.concatenate(trace)
    tstar = (np.arange(len(tr)) + 1) * every * s["omega0"]
    a = _smooth((tr[:, 0] - s["d"]) / s["a0"])
    cr = _crossings(tstar, a)
    half = float(cr[1] - cr[0]) if len(cr) >= 2 else None
    # first positive maxima: the initial elevation at t* = 0 and the largest
    # elevation around one period later
    win = (tstar > 1.5 * math.pi) & (tstar < 2.5 * math.pi)
    dec = None
    if win.any() and a[win].max() > 0:
        dec = float(math.log(a_init / a[win].max()))
    st = sim.status()
    cells = L * L
    if save_trace:
        np.save(save_trace, np.stack([tstar, a]))
    return dict(L=L, scheme=scheme, precision=precision, steps=done,
                half_period=half, log_decrement=dec,
                first_crossing=float(cr[0]) if len(cr) else None,
                unstable_step=st[1], seconds=wall, mlups=cells * done / wall / 1e6)


def dam_break(W: int, scheme: str, precision: str = "fp64", t_end: float = 3.5,
              device: int = 0):
    """The paper's rectangular dam break (Sec. 4.2) with free-slip walls and the
    Smagorinsky model: residual height h* = h/H at x = 0 and front w* = w/W at
    y = 0 over t* = t sqrt(2 g / W), sampled every t* = 0.01; the step at which
    an instability (|u| >= c_s) was latched, if any."""
    from . import fsl
    w = inputs.paper_dam_break(W, refill=scheme)
    sim = fsl.Sim(w["params"], precision, device=device)
    sim.init_workload(w)
    rate = math.sqrt(2.0 * w["g"] / W)          # t* per step
    every = max(1, int(round(0.01 / rate)))
    steps = int(t_end / rate)
    sim.set_trace(every)
    t0 = time.perf_counter()
    trace = []
    done = 0
    while done < steps:
        k = min(every * 4096, steps - done)
        k -= k % every
        if k <= 0:
            break
        sim.step(k)
        done += k
        trace.append(sim.trace(k // every))
        sim.set_trace(every)
    wall = time.perf_counter() - t0
    tr = np.concatenate(trace)
    tstar = (np.arange(len(tr)) + 1) * every * rate
    hstar = tr[:, 2] / w["height"]
    wstar = tr[:, 1] / W
    st = sim.status()
    out = dict(W=W, scheme=scheme, precision=precision, steps=done, seconds=wall,
               unstable_tstar=(st[1] * rate if st[1] >= 0 else None))
    for t in (0.5, 1.0, 1.5, 2.0, 2.5, 3.0):
        i = int(np.searchsorted(tstar, t))
        if i < len(tstar):
            out[f"h*@{t}"] = float(hstar[i])
            out[f"w*@{t}"] = float(wstar[i])
    return out


# Reynolds numbers printed in Sec. 4.4 (table of the Taylor bubble) per D
PAPER_TAYLOR_RE = {
    32: {"eq": 24.12, "eq_neq": 24.14, "geq": 24.16, "ext": 24.12, "avg": 24.09},
    64: {"eq": 25.35, "eq_neq": 25.32, "geq": 25.33, "ext": 25.34, "avg": 25.33},
    128: {"eq": 25.89, "eq_neq": 25.88, "geq": 25.89, "ext": 25.86, "avg": 25.86},
}


def gas_centroid(sim):
    """Centre of mass in z of the largest bubble (its gas cells count 1, its
    interface cells 1 - phi), that bubble's volume, and the number of
    bubbles."""
    t = sim.types()
    phi = sim.phi()
    lab = sim.bubbles()
    w = np.where(t == 0, 1.0, np.where(t == 1, 1.0 - phi, 0.0))
    z = np.broadcast_to((np.arange(t.shape[0]) + 0.5)[:, None, None], t.shape)
    sel = lab >= 0
    roots, inv = np.unique(lab[sel], return_inverse=True)
    vol = np.bincount(inv, weights=w[sel])
    mom = np.bincount(inv, weights=(w * z)[sel])
    k = int(np.argmax(vol))
    return float(mom[k] / vol[k]), float(vol[k]), int(np.unique(lab[t == 0]).size)


def taylor_bubble(D: int, scheme: str, precision: str = "fp32", t_samples=(10.0, 15.0),
                  device: int = 0):
    """Rise of the Taylor bubble: Re = D u / nu with u the velocity of the
    largest bubble's centre of mass between the two sample times
    t* = t sqrt(g / D)."""
    from . import fsl
    w = inputs.taylor_bubble(D, refill=scheme)
    sim = fsl.Sim(w["params"], precision, device=device)
    sim.init_workload(w)
    rate = math.sqrt(w["g"] / D)
    m0 = sim.total_mass()
    zc0, V0, _ = gas_centroid(sim)
    samples = []
    done = 0
    t0 = time.perf_counter()
    for ts in t_samples:
        n = int(round(ts / rate))
        sim.step(n - done)
        done = n
        zc, V, nb = gas_centroid(sim)
        samples.append(dict(tstar=n * rate, step=n, z=zc, volume=V, bubbles=nb))
    wall = time.perf_counter() - t0
    a, b = samples[0], samples[-1]
    u = (b["z"] - a["z"]) / (b["step"] - a["step"])
    st = sim.status()
    lab = sim.bubbles()
    p = sim.pressure()
    t = sim.types()
    pv = p[(t == 1) & (lab >= 0)]
    out = dict(D=D, scheme=scheme, precision=precision, steps=done, seconds=wall,
               Re=D * u / w["nu"], paper_Re=PAPER_TAYLOR_RE.get(D, {}).get(scheme),
               z0=zc0, volume0=V0, samples=samples,
               bubble_pressure=float(pv.mean()) if pv.size else None,
               mass_drift=(sim.total_mass() - m0) / m0,
               unstable_tstar=(st[1] * rate if st[1] >= 0 else None))
    sim.close()
    return out


def bubbly_poiseuille(scheme: str, precision: str = "fp32", L: int = 100, t_end: float = 4.0,
                      every: float = 0.5, options=None, device: int = 0):
    """The bubbly plane Poiseuille flow (Sec. 4.6) to t* = t u_max / L =
    `t_end`: every `every` in t*, the number of bubbles, the gas fraction,
    the gas-weighted mean distance |z - L/2| / (L/2) from the channel's
    centre plane, and max |u| / u_max; the t* of a latched instability.
    `options` replaces the configuration's option bits (0: no bubble model,
    every bubble at the constant volume pressure)."""
    from . import fsl
    w = inputs.bubbly_poiseuille(L=L, refill=scheme)
    if options is not None:
        w["params"]["options"] = options
    sim = fsl.Sim(w["params"], precision, device=device)
    sim.init_workload(w)
    rate = w["u_max"] / L
    zc = (np.arange(L) + 0.5 - L / 2.0) / (L / 2.0)
    m0 = sim.total_mass()

    def sample(step):
        t = sim.types()
        phi = sim.phi()
        lab = sim.bubbles()
        gas = np.where(t == 0, 1.0, np.where(t == 1, 1.0 - phi, 0.0))
        gz = gas.sum(axis=(1, 2))
        return dict(tstar=step * rate, bubbles=int(np.unique(lab[t == 0]).size),
                    gas_fraction=float(gas.sum() / t.size),
                    centre_distance=float((gz * np.abs(zc)).sum() / gz.sum()),
                    umax=sim.max_velocity() / w["u_max"])

    samples = [sample(0)]
    n_every = max(1, int(round(every / rate)))
    total = int(round(t_end / rate))
    done = 0
    t0 = time.perf_counter()
    while done < total:
        k = min(n_every, total - done)
        sim.step(k)
        done += k
        samples.append(sample(done))
        if sim.status()[0] != 0:
            break
    wall = time.perf_counter() - t0
    st = sim.status()
    out = dict(L=L, scheme=scheme, precision=precision, options=w["params"]["options"],
               steps=done, seconds=wall, unstable_tstar=(st[1] * rate if st[1] >= 0 else None),
               mass_drift=(sim.total_mass() - m0) / m0, samples=samples)
    sim.close()
    return out


def batched_waves(steps: int = 4000, n_geom: int = 64, precision: str = "fp16",
                  chunk: int = 16, tune: bool = True, seed: int = 2207, device: int = 0):
    """The batched standing-wave set: n_geom geometries (wavelength U[32, 256],
    width 1..8, depth L/2, amplitude 0.01 L, viscosity U[1e-3, 1e-2],
    g = 1e-5) times the five refilling schemes, FP16 storage.  Runs `steps`
    steps (a) with one fsl_step per domain, one after another on a single
    stream (the per-domain baseline, after the variant autotuner) and (b) as
    one batch (one graph launch per `chunk` steps, each kernel of a step
    launched once for all domains); reports both throughputs (all cells) and
    checks that sampled domains end bit-identical in the two runs."""
    import torch

    from . import autotune, fsl
    specs = inputs.batched_waves(seed=seed, n_geom=n_geom)
    ws = [inputs.standing_wave(sp["lam"], nz=sp["width"], nu=sp["nu"], refill=sp["refill"])
          for sp in specs]
    cells = sum(w["phi"].size for w in ws)

    def build(stream=None):
        sims = []
        for w in ws:
            s = fsl.Sim(w["params"], precision, device=device, stream=stream)
            s.init_workload(w)
            sims.append(s)
        return sims

    def state(s):
        t = s.types()
        fl = (t == 1) | (t == 2)
        return t, s.pdfs()[:, fl], s.mass()[t == 1]

    out = dict(domains=len(ws), cells=cells, steps=steps, precision=precision, chunk=chunk)
    # (a) one launch per domain on one stream
    one = torch.cuda.Stream(device=device)
    sims = build(one)
    picks = autotune.tune_batch(sims) if tune else {}
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(one)
    for s in sims:
        s.step(steps)
    e1.record(one)
    torch.cuda.synchronize()
    ms_a = e0.elapsed_time(e1)
    ref = [state(s) for s in sims[:: max(1, len(sims) // 16)]]
    for s in sims:
        s.close()
    del sims
    torch.cuda.empty_cache()
    # (b) one batch
    sims = build()
    if tune:
        autotune.tune_batch(sims)
    stream = torch.cuda.Stream(device=device)
    b = fsl.Batch(sims, chunk=chunk, stream=stream)
    b.step(chunk)  # capture and warm the graph outside the timed region
    torch.cuda.synchronize()
    e0.record(stream)
    b.step(steps - chunk)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_b = e0.elapsed_time(e1) * steps / (steps - chunk)
    got = [state(s) for s in sims[:: max(1, len(sims) // 16)]]
    same = all(all(np.array_equal(x, y) for x, y in zip(r, g_)) for r, g_ in zip(ref, got))
    status = [s.status() for s in sims]
    b.close()
    for s in sims:
        s.close()
    out.update(per_domain_ms=ms_a, batched_ms=ms_b,
               per_domain_mlups=cells * steps / (ms_a * 1e3),
               batched_mlups=cells * steps / (ms_b * 1e3),
               speedup=ms_a / ms_b, bitwise_equal_sampled=bool(same),
               unstable=[i for i, st in enumerate(status) if st[0] != 0],
               variants=sorted({p["variant"] for p in picks.values()}) if picks else None)
    return out


def _half_crossing(v0, v1, z0):
    """Position between cell centres z0 and z0 + 1 where a linear fill level
    going from v0 to v1 passes 1/2."""
    return z0 + (0.5 - v0) / (v1 - v0)


def drop_observables(phi, pool: float, diameter: float):
    """Cavity depth h_ca* and crown inner diameter d_cr* of the drop impact
    (Sec. 4.5), both in units of the drop diameter, from the fill level phi
    (nz, ny, nx) on the cross-section through the centre with normal x, on
    the phi = 1/2 contour (cell k has its centre at k + 1/2).

    h_ca: from the cavity bottom to the initial surface height `pool`: the
    lowest point of the centre column above which the fill level drops below
    1/2 (0 where the centre column is liquid up to the initial surface).
    d_cr: the crown's inner diameter at the initial surface height: in the row
    of cells just below that height, from the centre outwards along y, the
    first crossing of 1/2 on each side (0 where the centre is liquid)."""
    nz, ny, nx = phi.shape
    sec = phi[:, :, nx // 2]                      # (z, y)
    col = sec[:, ny // 2]
    zc = np.arange(nz) + 0.5
    h = 0.0
    k = int(np.argmax(col < 0.5))                 # first cell from the floor below 1/2
    if col[k] < 0.5 and k > 0:
        bottom = _half_crossing(col[k - 1], col[k], zc[k - 1])
        h = max(pool - bottom, 0.0)
    # the row of cells just below the initial surface height (centre at
    # pool - 1/2): the flat surface of the initial state sits on its top face
    k0 = min(max(int(math.floor(pool - 0.5)), 0), nz - 1)
    row = sec[k0]
    d = 0.0
    yc = ny // 2
    if row[yc] < 0.5:
        right = next((j for j in range(yc + 1, ny) if row[j] >= 0.5), None)
        left = next((j for j in range(yc - 1, -1, -1) if row[j] >= 0.5), None)
        if right is not None and left is not None:
            yr = _half_crossing(row[right - 1], row[right], right - 1 + 0.5)
            yl = _half_crossing(row[left], row[left + 1], left + 0.5)
            d = yr - yl
    return h / diameter, d / diameter


def drop_impact_precision(precisions=("fp64", "fp32", "fp16", "bf16"), steps: int = 2000,
                          every: int = 50, n: int = 256):
    """Error of the 16/32-bit storages against the FP64 path on the drop
    impact (Sec. 4.5 in shape, the benchmark workload): total-mass drift,
    cavity depth h_ca* and crown inner diameter d_cr* every `every` steps
    through the impact and the splash that follows.  Returns the traces and,
    per storage, the largest deviation from FP64 of each observable."""
    from . import fsl
    f = n / 256.0
    w = inputs.drop_impact() if n == 256 else inputs.drop_impact(
        n=n, pool=int(round(96 * f)), diameter=40.0 * f, gap=30.0 * f)
    pool = float(w["h_ref"])
    D = 40.0 * f
    out = dict(workload=w["name"], steps=steps, every=every, diameter=D, pool=pool,
               speed=0.05, traces={})
    for prec in precisions:
        sim = fsl.Sim(w["params"], prec)
        sim.init_workload(w)
        m0 = sim.total_mass()
        tr = dict(step=[], tstar=[], mass_drift=[], h_ca=[], d_cr=[])
        t0 = time.time()
        for k in range(0, steps + 1, every):
            if k:
                sim.step(every)
            h, d = drop_observables(sim.phi(), pool, D)
            tr["step"].append(k)
            tr["tstar"].append(k * 0.05 / D)
            tr["mass_drift"].append((sim.total_mass() - m0) / m0)
            tr["h_ca"].append(h)
            tr["d_cr"].append(d)
        tr["status"] = list(sim.status())
        tr["seconds"] = time.time() - t0
        sim.close()
        out["traces"][prec] = tr
    ref = out["traces"].get("fp64")
    if ref is not None:
        out["error_vs_fp64"] = {}
        for prec, tr in out["traces"].items():
            if prec == "fp64":
                continue
            out["error_vs_fp64"][prec] = dict(
                h_ca_max_abs=float(np.max(np.abs(np.array(tr["h_ca"]) - ref["h_ca"]))),
                d_cr_max_abs=float(np.max(np.abs(np.array(tr["d_cr"]) - ref["d_cr"]))),
                mass_drift_max_abs=float(np.max(np.abs(tr["mass_drift"]))),
                fp64_mass_drift_max_abs=float(np.max(np.abs(ref["mass_drift"]))))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, nargs="*", default=[200, 400, 800])
    ap.add_argument("--schemes", nargs="+", default=list(inputs.REFILL_SCHEMES))
    ap.add_argument("--precision", default="fp64")
    ap.add_argument("--save-dir", default=None, help="write each a*(t*) trace as .npy here")
    ap.add_argument("--dam-break", type=int, nargs="*", default=[],
                    help="also run the Sec. 4.2 dam break at these column widths W")
    ap.add_argument("--taylor", type=int, nargs="*", default=[],
                    help="also run the Sec. 4.4 Taylor bubble at these tube diameters D")
    ap.add_argument("--bubbly", action="store_true",
                    help="also run the Sec. 4.6 bubbly plane Poiseuille flow")
    ap.add_argument("--drop-precision", default=None, metavar="FILE",
                    help="run the drop-impact precision study (FP32/FP16/BF16 against FP64) "
                         "and write its JSON here")
    ap.add_argument("--drop-steps", type=int, default=2000)
    ap.add_argument("--drop-size", type=int, default=256)
    ap.add_argument("--batched", type=int, default=0,
                    help="also run the batched standing-wave set for this many steps")
    args = ap.parse_args()
    if args.drop_precision:
        r = drop_impact_precision(steps=args.drop_steps, n=args.drop_size)
        with open(args.drop_precision, "w") as fh:
            json.dump(r, fh, indent=1)
        print(json.dumps(dict(workload=r["workload"], error_vs_fp64=r.get("error_vs_fp64"))),
              flush=True)
        if not args.L:
            return
    if args.batched:
        print(json.dumps(batched_waves(steps=args.batched)), flush=True)
    if args.bubbly:
        for sc in args.schemes:
            print(json.dumps(bubbly_poiseuille(sc, args.precision)), flush=True)
    for D in args.taylor:
        for sc in args.schemes:
            print(json.dumps(taylor_bubble(D, sc, args.precision)), flush=True)
    for W in args.dam_break:
        for sc in args.schemes:
            print(json.dumps(dam_break(W, sc, args.precision)), flush=True)
    for L in args.L:
        for sc in args.schemes:
            path = None
            if args.save_dir:
                import os
                os.makedirs(args.save_dir, exist_ok=True)
                path = os.path.join(args.save_dir, f"wave_L{L}_{sc}_{args.precision}.npy")
            r = gravity_wave(L, sc, args.precision, save_trace=path)
            r["paper_L800"] = dict(half_period=PAPER_L800["half_period"].get(sc),
                                   log_decrement=PAPER_L800["log_decrement"].get(sc))
            print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
