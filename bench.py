"""Benchmark of the free-surface LBM step on one GB300 (or N replicas).

Workload: the drop impact into a pool, 256^3 cells, D3Q27 TRT (Lambda 3/16),
surface tension 1e-4, gravity 1e-6, EQ refilling (Sec. 4.5 in shape), with
seeded synthetic initial fill levels.  The metric is MLUPS (all lattice cells
per second) of the whole step (stream-collide, interface pass, conversion,
refilling, excess mass, curvature, per-step observables), mixed precision
(FP16 offset storage, FP32 collide) as the headline, with FP32 and FP64 (and
BF16) on the same workload beside it, and the HBM-roofline fraction of the
dominant kernel.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) each rank runs an independent replica of the domain
(the step has no exchange between independent domains); value sums all ranks.
`--impl reference` times the CPU oracle (the only reference implementation of
this method here) on a bounded sample of the workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "drop_impact_256"
METRIC = "FSLBM MLUPS (all cells), mixed FP16 vs FP64, drop impact 256^3 D3Q27"


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return dict(hbm_gbs=float(d["hbm_gbs"]), source="measured")
    return dict(hbm_gbs=6800.0, source="fallback")


# the bulk stream-collide kernel behind each variant of the 16/32-bit path
KERNEL_OF = {"pair": "k_stream_collide_lp", "pair_r128": "k_stream_collide_lp",
             "pair_r96": "k_stream_collide_lp", "pair_r80": "k_stream_collide_lp",
             "tma": "k_stream_collide_bulk", "warp_tma": "k_stream_collide_wtma",
             "quad64": "k_stream_collide_lp4", "pair_pipe": "k_stream_collide_pp",
             "cpa": "k_stream_collide_cpa", "cpa_deep": "k_stream_collide_cpa",
             "cpa_r96": "k_stream_collide_cpa", "seg": "k_stream_collide_seg",
             "seg_r128": "k_stream_collide_seg", "cell": "k_stream_collide_c1",
             "cell_r80": "k_stream_collide_c1", "tma_r96": "k_stream_collide_bulk"}

# FP64 instruction peak for the bit-exact path (built without multiply-add
# contraction): the part's nominal 1.25 TFLOP/s of FP64 counts an FMA as two
# flops, so its FP64 pipes retire 0.625 T FP64 instructions per second.
FP64_PEAK_TINSTR = 1.25 / 2
# nominal HBM3e bandwidth of the part, for the second roofline fraction
NOMINAL_HBM_GBS = 7900.0


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while timing."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = ""

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["unsampled"], samples=0)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return dict(sm_mhz=statistics.median(sm) if sm else None,
                    sm_max_mhz=max(smax) if smax else None, reasons=reasons, samples=len(rows))


def reduce_max(v: float, world: int, device: str) -> float:
    """Maximum of a per-rank value over the ranks of the default process
    group (the slowest replica sets the job's time)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_mlups(cells: int, steps: int, ms_max: float, world: int) -> float:
    """Whole-job throughput of `world` independent replicas of a domain of
    `cells` cells, each advanced `steps` steps, the slowest in ms_max ms."""
    return world * cells * steps / (ms_max * 1e-3) / 1e6


def time_precision(fsl, w, precision, steps, warmup, dev, barrier, start=0, pre_impact=0,
                   variant=None):
    """Device-resident timing: CUDA events on the library's stream around K
    steps (captured CUDA graphs), after W warm-up steps.  The state is first
    advanced `start` steps (untimed) so that the timed window lies in the
    phase after the drop has hit the pool; with pre_impact > 0 that many
    steps are also timed from step W + 3, before the impact (replayed from a
    checkpoint with the tuned variant), and reported beside it."""
    import torch

    from paper_2207_14496_gb300 import autotune

    sim = fsl.Sim(w["params"], precision, device=dev)
    sim.init_workload(w)
    sim.set_trace(1)
    early_state = None
    if pre_impact > 0:
        # the state before the impact, replayed with the tuned variant below
        sim.step(warmup)
        early_state = sim.save()
    done = sim.step_count
    if start > done:
        sim.step(start - done)
    sim.step(warmup)
    torch.cuda.synchronize(dev)
    # bulk-pass variant picked by the autotuner on the warmed-up state (untimed;
    # the measurement leaves the state unchanged)
    if variant and precision != "fp64":
        # a fixed bulk-pass variant (profiling runs, where the timings that
        # the autotuner would compare are distorted)
        sim.set_variant(variant)
        tuned = dict(variant=variant, ms={})
    else:
        tuned = autotune.tune(sim, reps=5)
    # then whole steps with the three fastest bulk passes (the interface pass
    # runs beside the bulk pass and competes with it)
    if tuned["ms"]:
        top = sorted(tuned["ms"], key=tuned["ms"].get)[:3]
        stepwise = autotune.tune_step(sim, top)
        tuned["variant"] = stepwise["variant"]
        tuned["ms_step"] = stepwise["ms_step"]
    sim.step(3)
    torch.cuda.synchronize(dev)
    n_cells = sim.N
    ks0 = sim.kernel_stats(reps=5)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(dev) as clk:
        e0.record(sim.stream)
        sim.step(steps)
        e1.record(sim.stream)
        torch.cuda.synchronize(dev)
    barrier()
    ms = e0.elapsed_time(e1)
    ks1 = sim.kernel_stats(reps=10)
    status = sim.status()
    launches = sim.launches_per_step() * steps
    first = sim.step_count - steps
    early = None
    if early_state is not None:
        sim.load(early_state)
        sim.step(3)  # the step graph is captured again after the load
        torch.cuda.synchronize(dev)
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(sim.stream)
        sim.step(pre_impact)
        a1.record(sim.stream)
        torch.cuda.synchronize(dev)
        t_ms = a0.elapsed_time(a1)
        early = dict(from_step=warmup + 3, steps=pre_impact, ms_per_step=t_ms / pre_impact,
                     mlups=sim.N * pre_impact / (t_ms * 1e-3) / 1e6, variant=tuned["variant"])
    del sim
    torch.cuda.empty_cache()
    return dict(ms=ms, ms_per_step=ms / steps, mlups=n_cells * steps / (ms * 1e-3) / 1e6,
                kernel_ms=0.5 * (ks0["ms"] + ks1["ms"]),
                kernel_bytes=0.5 * (ks0["bytes"] + ks1["bytes"]),
                n_liquid=0.5 * (ks0["n_liquid"] + ks1["n_liquid"]),
                n_interface=0.5 * (ks0["n_interface"] + ks1["n_interface"]),
                clocks=clk.summary(), status=status, launches=launches,
                variant=tuned["variant"], tuning_ms=tuned["ms"],
                tuning_ms_step=tuned.get("ms_step"), first_step=first,
                pre_impact=early)


def e2e_run(fsl, w, precision, steps, dev, variant="default"):
    """End to end through the public API from pinned host memory: initial
    state upload, K steps, per-step observable trace and total mass read back
    (with the bulk-pass variant the device-resident run was tuned to)."""
    import torch

    sim = fsl.Sim(w["params"], precision, device=dev)
    sim.set_variant(variant)
    phi = torch.from_numpy(np.ascontiguousarray(w["phi"], dtype=np.float64)).pin_memory()
    u0 = torch.from_numpy(np.ascontiguousarray(w["u0"], dtype=np.float64)).pin_memory()
    phin, u0n = phi.numpy(), u0.numpy()
    sim.set_trace(1)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    sim.init_fill(phin, u0n, None, w["h_ref"])
    sim.step(steps)
    trace = sim.trace(steps)
    mass = sim.total_mass()
    t1 = time.perf_counter()
    del sim
    torch.cuda.empty_cache()
    n = int(np.prod(w["params"]["shape"]))
    h2d = phin.nbytes + u0n.nbytes
    d2h = trace.nbytes + 8 + 16 * 2  # trace, mass, status/step reads inside observe
    return dict(seconds=t1 - t0, mlups=n * steps / (t1 - t0) / 1e6,
                h2d_per_step=h2d / steps, d2h_per_step=d2h / steps, mass=mass)


def host_cpu():
    """Core count (os.cpu_count, as nproc) and CPU model of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.TimeoutExpired):
        pass
    return os.cpu_count() or 1, model


def time_oracle(w, steps, threads):
    """Wall time of `steps` oracle steps on `threads` OpenMP threads (the
    initial state untimed); returns (seconds, threads in effect)."""
    import oracle
    used = oracle.set_threads(threads)
    try:
        o = oracle.Oracle(w["params"])
        o.init_fill(w["phi"], w.get("u0"), None, w["h_ref"])
        t0 = time.perf_counter()
        o.step(steps)
        return time.perf_counter() - t0, used
    finally:
        oracle.set_threads(1)


def cpu_baseline(w, steps=1):
    """The CPU oracle as it stands on a bounded sample: the full 256^3 workload
    for `steps` time steps, on all host cores (its order-free per-cell loops
    on OpenMP threads) and on one core."""
    cores, model = host_cpu()
    dt_all, used = time_oracle(w, steps, cores)
    dt_one, _ = time_oracle(w, steps, 1)
    n = int(np.prod(w["params"]["shape"]))
    return dict(value=n * steps / dt_all / 1e6, unit="MLUPS", cores=used, kind="oracle",
                cpu_model=model, nproc=cores, single_core=n * steps / dt_one / 1e6,
                sample=f"{steps} step(s) of the full 256^3 D3Q27 drop-impact workload from its "
                       f"initial state, FP64 C oracle: {dt_all:.1f} s on {used} threads, "
                       f"{dt_one:.1f} s on one")


def run_reference(args):
    """Reference arm: the CPU oracle, timed on the machine's host core, one oracle
    time step per bench step on a bounded 64^3 sample of the drop impact
    (same physics scaled down so that the whole run ends within minutes)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2207_14496_gb300 import inputs
    import oracle
    cores, model = host_cpu()
    used = oracle.set_threads(cores)
    w = inputs.drop_impact(n=64, pool=24, diameter=10.0, gap=8.0)
    o = oracle.Oracle(w["params"])
    o.init_fill(w["phi"], w.get("u0"), None, w["h_ref"])
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    oracle.set_threads(1)
    n = int(np.prod(w["params"]["shape"]))
    v = n * args.steps / dt / 1e6
    sample = (f"64^3 D3Q27 TRT drop impact (pool 24, drop D=10), {args.steps} oracle steps "
              f"after {args.warmup}, FP64, {used} OpenMP threads, {dt:.1f} s")
    line = dict(impl="reference", metric=METRIC, value=v, unit="MLUPS", n_gpus=args.gpus,
                steps=args.steps, warmup=args.warmup, ms_per_step=dt * 1e3 / args.steps,
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
                data="synthetic", config=dict(workload=WORKLOAD, sample="64^3 scaled drop impact",
                                              parallelism=f"cpu-{used}"),
                cpu_baseline=dict(value=v, unit="MLUPS", cores=used, kind="oracle", sample=sample,
                                  cpu_model=model, nproc=cores),
                e2e=dict(value=v, unit="MLUPS", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precisions", default="fp16,fp32,fp64,bf16")
    ap.add_argument("--fp64-steps", type=int, default=None,
                    help="steps for the FP64 comparison line (default: steps // 5)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--start", type=int, default=1000,
                    help="untimed steps before the warm-up (the drop reaches the pool near "
                         "step 200; the default window lies in the splash that follows)")
    ap.add_argument("--pre-impact", type=int, default=100,
                    help="steps also timed from step W, before the impact, for the headline "
                         "storage (0: skip)")
    ap.add_argument("--variant", default=None,
                    help="bulk-pass variant of the 16/32-bit storages instead of the autotuner's "
                         "pick (for profiling captures)")
    ap.add_argument("--size", type=int, default=256,
                    help="edge of the drop-impact cube (256 = the benchmark workload; smaller "
                         "sizes scale pool and drop, for profiling captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(v: float) -> float:
        return reduce_max(v, world, f"cuda:{local}")

    from paper_2207_14496_gb300 import build, inputs
    build.build()
    from paper_2207_14496_gb300 import fsl

    if args.size == 256:
        w = inputs.drop_impact()
    else:
        f = args.size / 256.0
        w = inputs.drop_impact(n=args.size, pool=int(round(96 * f)), diameter=40.0 * f,
                               gap=30.0 * f)
    peaks = load_peaks()
    precs = [p for p in args.precisions.split(",") if p]
    res = {}
    for p in precs:
        k = args.steps
        if p == "fp64":
            k = args.fp64_steps or max(10, args.steps // 5)
        res[p] = time_precision(fsl, w, p, k, args.warmup, local, barrier, start=args.start,
                                pre_impact=args.pre_impact if p == precs[0] else 0,
                                variant=args.variant)
        res[p]["steps"] = k
    head = precs[0]
    h = res[head]
    ms_max = max_over_ranks(h["ms"])
    n_cells = int(np.prod(w["params"]["shape"]))
    value = replica_mlups(n_cells, h["steps"], ms_max, world)

    def fluid_mlups(r):
        # liquid + interface cells (mean of the counts before and after the
        # timed steps) per second
        return (r["n_liquid"] + r["n_interface"]) * r["steps"] / (r["ms"] * 1e-3) / 1e6

    def roofline(r, prec):
        if prec == "fp64":
            # FP64 is bound by the FP64 pipe on GB300: FP64 instructions of the
            # stream-collide kernel (D3Q27 TRT with Guo forcing, per liquid
            # cell, counted by ncu) over its launch time
            instr = r["n_liquid"] * FP64_INSTR_PER_LIQUID_CELL_D3Q27_TRT
            ach = instr / (r["kernel_ms"] * 1e-3) / 1e12
            return dict(bound="alu", achieved=ach, peak=FP64_PEAK_TINSTR,
                        unit="T FP64 instructions/s", frac=ach / FP64_PEAK_TINSTR, traffic=None,
                        kernel="k_stream_collide",
                        peak_source="nominal 1.25 TFLOP/s FP64 (an FMA counted as two flops)")
        ach = r["kernel_bytes"] / (r["kernel_ms"] * 1e-3) / 1e9
        return dict(bound="hbm", achieved=ach, peak=peaks["hbm_gbs"], unit="GB/s",
                    frac=ach / peaks["hbm_gbs"], frac_nominal=ach / NOMINAL_HBM_GBS,
                    traffic=traffic_of(prec, r["variant"]) if args.size == 256 else None,
                    kernel=KERNEL_OF.get(r["variant"], "k_stream_collide_lp"),
                    variant=r["variant"], peak_source=peaks["source"])

    by_prec = {}
    for p in precs:
        r = res[p]
        by_prec[p] = dict(mlups=r["mlups"], ms_per_step=r["ms_per_step"], steps=r["steps"],
                          fluid_mlups=fluid_mlups(r),
                          kernel_ms=r["kernel_ms"], kernel_bytes=r["kernel_bytes"],
                          roofline=roofline(r, p), status=list(r["status"]),
                          clocks=r["clocks"], variant=r["variant"], tuning_ms=r["tuning_ms"],
                          tuning_ms_step=r["tuning_ms_step"])
    # a step after a latched instability does no work: such a run is not a
    # measurement of the step
    unstable = {p: res[p]["status"][1] for p in precs if res[p]["status"][0] != 0}
    e2e = None
    if not args.no_e2e:
        e = e2e_run(fsl, w, head, h["steps"], local, variant=h["variant"])
        e2e = dict(value=world * e["mlups"], unit="MLUPS",
                   h2d_bytes_per_step=e["h2d_per_step"], d2h_bytes_per_step=e["d2h_per_step"])
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.size == 256:
        cpu = cpu_baseline(w, steps=1)
    if rank == 0:
        clocks = h["clocks"]
        line = dict(
            metric=METRIC, value=value, unit="MLUPS", n_gpus=world, steps=h["steps"],
            warmup=args.warmup, ms_per_step=ms_max / h["steps"], higher_is_better=True,
            scaling="weak", vs_baseline=None, dtype="f32" if head != "fp64" else "f64",
            storage=head, data="synthetic",
            config=dict(workload=WORKLOAD if args.size == 256 else f"drop_impact_{args.size}",
                        timed_from_step=h["first_step"],
                        shape=[args.size] * 3, lattice="D3Q27",
                        collision="TRT 3/16", refill="eq", sigma=1e-4, gravity=1e-6,
                        nu=round(inputs.DROP_NU, 9), parallelism=f"replicas{world}",
                        l2="inputs larger than L2 (PDF buffers >= 1.8 GB)"),
            roofline=by_prec[head]["roofline"], cpu_baseline=cpu, e2e=e2e,
            gpu_launches=h["launches"],
            fluid_mlups=world * by_prec[head]["fluid_mlups"],
            clocks=dict(sm_mhz=clocks["sm_mhz"], sm_max_mhz=clocks["sm_max_mhz"],
                        reasons=clocks["reasons"], samples=clocks["samples"]),
            by_precision=by_prec,
            speedup_vs_fp64=(h["mlups"] / res["fp64"]["mlups"]) if "fp64" in res else None,
            speedup_vs_fp32=(h["mlups"] / res["fp32"]["mlups"]) if "fp32" in res else None,
            stable=not unstable, unstable_steps=unstable or None,
            pre_impact=h["pre_impact"],
        )
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# FP64 instructions per liquid-cell update of the FP64 stream-collide kernel
# for D3Q27 TRT with Guo forcing: ncu's smsp__sass_thread_inst_executed_op_
# fp64_pred_on.sum (1.3365e9) over the liquid cells (1.526e6) of one launch
# on the 160^3 drop impact.
FP64_INSTR_PER_LIQUID_CELL_D3Q27_TRT = 876
# DRAM bytes (read + write) per launch of the bulk kernel on the 256^3
# workload, from one single-pass ncu capture of the autotuner's launches of
# each variant, with the digest of the kernel sources the capture ran
# (kernel_source_digest); an entry whose digest differs from the sources
# built now is stale and reported as null.
TRAFFIC = {("fp16", "tma"): (673.11e6, "7a0a0cc5ae151d71"),
           ("fp16", "tma_r96"): (686.77e6, "7a0a0cc5ae151d71"),
           ("fp32", "tma"): (1370.97e6, "7a0a0cc5ae151d71")}
KERNEL_SOURCES = ("fsl_kernels.cuh", "fsl_bulk.cuh", "fsl_lattice.cuh", "fsl_internal.h")


def kernel_source_digest() -> str:
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2207_14496_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_of(prec, variant):
    e = TRAFFIC.get((prec, variant))
    if e is None or e[1] != kernel_source_digest():
        return None
    return e[0]

if __name__ == "__main__":
    main()
