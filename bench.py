"""Throughput of the staggered-grid P_N step on GB300, one JSON line on stdout.

Workload (default): P39 (1600 moments) on 200^3 periodic cells, FP32 storage and arithmetic,
sigma_s log-uniform in [0.1, 10] per 8^3 block, sigma_a = 0.01, q = 0, Gaussian u_0 (width 0.1 of
the unit box, unit sum).  A bench "step" is one full time step of Eq. (6) (the merged schedule:
one even and one odd pass per step).  The 51 GB state is far larger than L2, so no flush is needed
between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank advances its own replica (independent instances, no
collective); value = all ranks' updates / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "P_N moment-cell updates/s, % HBM peak; FP32/BF16 vs FP64 at stated error"
UNIT = "MLCUP/s"  # million lattice cell component updates (moment-cell updates) per second


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--N", type=int, default=39)
    p.add_argument("--n", type=int, default=200)
    p.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp64"])
    p.add_argument("--kernel", default="auto", choices=["auto", "generic", "window", "stage", "fused"])
    p.add_argument("--tile", default="0,0,0")
    p.add_argument("--depth", type=int, default=0, help="stage buffers of the staged kernel (0 = default)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-forms", action="store_true",
                   help="skip the BF16 / batched / adjoint form measurements")
    p.add_argument("--forms", default="bf16,fused,reactor,batched,adjoint,scattering",
                   help="which form measurements to run (comma-separated)")
    p.add_argument("--record-traffic", default=None,
                   help="write profiles/stage_traffic.json from an ncu CSV of this workload, then exit")
    return p.parse_args()


def workload_config(args):
    return {"workload": f"P{args.N} {args.n}^3 periodic random-block media, Gaussian u_0",
            "N": args.N, "cells": args.n ** 3, "moments": (args.N + 1) ** 2,
            "storage": args.precision, "kernel": args.kernel,
            "l2_flush": "not needed: state larger than L2 (inputs larger than L2)"}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# DRAM bytes per cell of one launch of the staged kernel, from one ncu capture of a smaller grid
# (dram__bytes_read.sum + dram__bytes_write.sum), keyed by the sha256 of the kernel's sources at
# capture time: once any of them changes, the traffic is reported as null.  `--record-traffic`
# writes the file from the capture's CSV.
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "stage_traffic.json")
KERNEL_SOURCES = ["stage_impl.cuh", "stage.cu", "kernels_stage.cu", "window_impl.cuh"]


def kernel_source_hash() -> str:
    import hashlib

    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2004_02833_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def _traffic_key(N, storage, tile, depth, cls):
    return f"P{N} {storage} tile {tile[0]}x{tile[1]}x{tile[2]} depth {depth} class {cls}"


def traffic_per_launch(kernel, N, storage, tile, depth, cls, cells):
    """(DRAM bytes of one launch, description) scaled from the capture, or (None, why not)."""
    if kernel != "stage" or not os.path.exists(TRAFFIC_FILE):
        return None, "no capture of this kernel"
    rec = json.load(open(TRAFFIC_FILE))
    if rec.get("kernel_sha256") != kernel_source_hash():
        return None, "kernel sources changed since the capture"
    e = rec["entries"].get(_traffic_key(N, storage, tile, depth, cls))
    if e is None:
        return None, "no capture of this configuration"
    return e["bytes_per_cell"] * cells, (f"ncu dram read+write of one launch at {e['grid']}, same kernel "
                                         f"build and configuration, scaled by the cell count")


def record_traffic(args):
    """Write TRAFFIC_FILE entries from an ncu CSV (--metrics dram__bytes_read.sum,dram__bytes_write.sum
    --csv --log-file) of `bench.py --n <n> --tile .. --depth ..` (both classes, one launch each)."""
    import csv

    rows = [r for r in csv.reader(open(args.record_traffic)) if len(r) > 10]
    hdr = rows[0]
    ki, mi, vi, ui, ii = (hdr.index(k) for k in ("Kernel Name", "Metric Name", "Metric Value", "Metric Unit", "ID"))
    launches = {}
    for r in rows[1:]:
        if "k_stage<" not in r[ki] or not r[mi].startswith("dram__bytes_"):
            continue
        scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}[r[ui]]
        d = launches.setdefault(r[ii], {"name": r[ki], "bytes": 0.0})
        d["bytes"] += float(r[vi].replace(",", "")) * scale
    rec = {"kernel_sha256": kernel_source_hash(), "entries": {}}
    if os.path.exists(TRAFFIC_FILE):
        old = json.load(open(TRAFFIC_FILE))
        if old.get("kernel_sha256") == rec["kernel_sha256"]:
            rec["entries"] = old["entries"]
    tile = tuple(int(x) for x in args.tile.split(","))
    cells = args.n ** 3
    for d in launches.values():
        cls = int(d["name"].split("k_stage<")[1].split(",")[0])
        key = _traffic_key(args.N, args.precision, tile, args.depth, cls)
        if key not in rec["entries"]:  # the first launch of each class
            rec["entries"][key] = {"bytes_per_cell": d["bytes"] / cells, "grid": f"{args.n}^3",
                                   "dram_bytes": d["bytes"]}
    json.dump(rec, open(TRAFFIC_FILE, "w"), indent=1, sort_keys=True)
    print(json.dumps(rec, indent=1))


class Clocks:
    """nvidia-smi sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={device_index}",
                                       f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                       "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for name, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform

    return platform.machine()


def _oracle_replica(N, n, steps, warmup, barrier, queue):
    """One serial replica of the FP64 oracle on the n^3 instance with the workload's rules: set-up
    and warm-up steps, then `steps` timed steps started together with the other replicas."""
    from oracle import stepper as st
    from paper_2004_02833_gb300 import synth

    inst = synth.random_blocks(N, n, seed=2)
    P = st.Problem(inst.N, inst.sigma_a, inst.sigma_s, inst.q, inst.h, inst.dt, inst.bc)
    u = inst.full_state()
    for _ in range(warmup):
        u = P.step(u)
    barrier.wait()
    t0 = time.perf_counter()
    for _ in range(steps):
        u = P.step(u)
    queue.put(time.perf_counter() - t0)


def oracle_throughput(N: int, n: int, steps: int, warmup: int, procs: int):
    """(MCU/s, seconds) of `procs` concurrent replicas of the oracle (spawned processes, one core
    each): all replicas' updates over the slowest replica's time."""
    import multiprocessing as mp

    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"  # one thread per replica
    ctx = mp.get_context("spawn")
    barrier, queue = ctx.Barrier(procs), ctx.Queue()
    ps = [ctx.Process(target=_oracle_replica, args=(N, n, steps, warmup, barrier, queue)) for _ in range(procs)]
    for p in ps:
        p.start()
    times = [queue.get() for _ in ps]
    for p in ps:
        p.join()
    dt = max(times)
    return (N + 1) ** 2 * n ** 3 * steps * procs / dt, dt


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(args, steps: int):
    """The FP64 oracle, as it stands, on a bounded sample: the same rules at 24^3 (same per-cell
    work per moment), on one core and as one serial replica per host core."""
    n = 24
    v1, t1 = oracle_throughput(args.N, n, steps, 0, 1)
    cores = host_cores()
    vall, tall = oracle_throughput(args.N, n, steps, 0, cores)
    return {"value": vall / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"P{args.N} {n}^3 periodic random-block instance, {steps} steps, one serial numpy "
                      f"FP64 replica per core ({tall:.1f} s)",
            "single_core": {"value": v1 / 1e6, "unit": UNIT, "cores": 1,
                            "sample": f"one replica, {steps} steps ({t1:.1f} s)"},
            "nproc": os.cpu_count(), "cpu_model": cpu_model()}


def run_reference(args, rank, world):
    """--impl reference: the FP64 oracle timed on the host cores (rank 0 only), one serial replica
    per core, each step a step of the 24^3 instance with the workload's rules."""
    if rank != 0:
        return
    n = 24
    cores = host_cores()
    v, dt = oracle_throughput(args.N, n, args.steps, args.warmup, cores)
    value = v / 1e6
    config = dict(workload_config(args))
    config["reference_sample"] = (f"each step: one step of the P{args.N} {n}^3 instance with the same rules on "
                                  f"each of {cores} host cores (FP64 oracle, numpy, one replica per core)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": config["reference_sample"], "nproc": os.cpu_count(),
                             "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.record_traffic:
        record_traffic(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch

    from paper_2004_02833_gb300 import rtpn, synth

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    inst = synth.random_blocks(args.N, args.n, seed=2 + rank)
    tile = tuple(int(x) for x in args.tile.split(","))
    stream = torch.cuda.Stream()
    ctx = rtpn.Context(args.N, inst.shape, inst.h, inst.bc, args.precision, inst.dt)
    ctx.set_stream(stream)
    if args.kernel != "auto" or any(tile) or args.depth:
        ctx.set_kernel(args.kernel, tile, args.depth)
    info = ctx.info()
    with torch.cuda.stream(stream):
        media = [torch.tensor(a, dtype=torch.float32, device="cuda")
                 for a in (inst.sigma_a, inst.sigma_s, inst.q)]
        u0 = torch.tensor(inst.u0, dtype=torch.float32, device="cuda")
    ctx.zero_moments()
    ctx.set_media(*media)
    ctx.set_component(0, u0)
    ctx.step(args.warmup)
    ctx.synchronize()

    # ---- timed region: K full steps, inputs resident in HBM
    clocks = Clocks(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    ctx.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    mcu_step = inst.n_c * inst.shape[0] * inst.shape[1] * inst.shape[2]
    ms, units = aggregate(ms, float(mcu_step * args.steps), dist, device="cuda")
    value = units / (ms / 1e3) / 1e6
    nonfinite = ctx.count_nonfinite()

    # ---- per-launch duration of the dominant kernel (the even and the odd substep pass)
    per_pass = pass_durations(ctx, stream, reps=max(3, min(10, args.steps)))
    s = {"fp32": 4, "bf16": 2, "fp64": 8}[args.precision]
    V = inst.shape[0] * inst.shape[1] * inst.shape[2]
    # algorithmic bytes of one pass: every moment read once, the pass's class written once,
    # plus the media share (12 B per cell per step, i.e. 6 B per pass)
    alg = {cls: V * ((info.n_c + n_a) * s + 6) for cls, n_a in ((0, info.n_even), (1, info.n_odd))}
    dom = max(per_pass, key=lambda c: per_pass[c])
    hbm, peak_kind = peaks()
    achieved = alg[dom] / (per_pass[dom] / 1e3) / 1e9
    kname = {1: "generic", 2: "window", 3: "stage", 4: "fused"}.get(ctx.info().kernel, "?")
    traffic, traffic_src = traffic_per_launch(kname, args.N, args.precision, tuple(ctx.info().tile),
                                              ctx.info().depth, dom, V)
    step_ms = ms / args.steps
    step_bytes = V * (info.n_c * 2 * s + 12)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": traffic, "traffic_source": traffic_src,
                "kernel": f"substep pass ({'even' if dom == 0 else 'odd'} class)",
                "peak_kind": peak_kind,
                "pass_ms": {"even": per_pass[0], "odd": per_pass[1]},
                "step_alg_bytes_per_mcu": step_bytes / mcu_step,
                "step_frac": step_bytes / (step_ms / 1e3) / 1e9 / hbm}

    # ---- end to end through the C ABI with host buffers (inputs u_0 and media; output u_0)
    e2e = None
    if not args.no_e2e:
        e2e = end_to_end(ctx, inst, args, mcu_step, world, dist)

    # the host baseline and the form measurements are one-GPU figures: rank 0 of a one-rank run
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args, steps=5)

    forms = None
    if rank == 0 and world == 1 and not args.no_forms and args.precision == "fp32":
        forms = measure_forms(args, ctx, stream, step_ms, mcu_step)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "bf16": "bf16",
                                                                "fp64": "f64"}[args.precision],
            "data": "synthetic", "config": workload_config(args),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "gpu_launches": 2 * args.steps + 1, "nonfinite": nonfinite, "forms": forms,
            "kernel_used": kname,
            "tile": list(ctx.info().tile), "depth": ctx.info().depth}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


def _guard(fn):
    try:
        return fn()
    except Exception as e:  # a form that fails is reported, the headline line still prints
        return {"error": f"{type(e).__name__}: {e}"}


def measure_forms(args, ctx32, stream, fp32_ms, mcu_step):
    """Speedups of the three systems forms over the plain FP32 path, each at its stated bound."""
    import torch

    from paper_2004_02833_gb300 import rtpn, synth

    out = {}

    def bf16():
        inst = synth.random_blocks(args.N, args.n, seed=2)
        c = rtpn.Context(args.N, inst.shape, inst.h, inst.bc, "bf16", inst.dt)
        c.set_stream(stream)
        c.set_media(*[torch.tensor(a, dtype=torch.float32, device="cuda")
                      for a in (inst.sigma_a, inst.sigma_s, inst.q)])
        c.zero_moments()
        c.set_component(0, torch.tensor(inst.u0, dtype=torch.float32, device="cuda"))
        c.step(3)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        c.step(args.steps)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / args.steps
        # the dominant pass against the copy bandwidth on BF16's algorithmic bytes (2 B per moment)
        info = c.info()
        per_pass = pass_durations(c, stream, reps=5)
        V = inst.shape[0] * inst.shape[1] * inst.shape[2]
        alg = {cls: V * ((info.n_c + n_a) * 2 + 6) for cls, n_a in ((0, info.n_even), (1, info.n_odd))}
        dom = max(per_pass, key=lambda k: per_pass[k])
        hbm, _ = peaks()
        pass_frac = alg[dom] / (per_pass[dom] / 1e3) / 1e9 / hbm
        c.close()
        # accuracy at the stated bounds on the 24^3 instance with the same rules (100 steps)
        small = synth.random_blocks(args.N, 24, seed=2)
        res = {}
        for prec in ("fp64", "fp32", "bf16"):
            with rtpn.Context(args.N, small.shape, small.h, small.bc, prec, small.dt) as s_:
                s_.set_media(small.sigma_a, small.sigma_s, small.q)
                s_.set_moments(small.full_state())
                s_.step(100)
                res[prec] = s_.get_moments()
        ref = res["fp64"]
        err = {p: float(np.abs(res[p] - ref).max() / np.abs(ref).max()) for p in ("fp32", "bf16")}
        # the same errors as relative L2, and pointwise relative where |ref| > 1e-3 max |ref|
        big = np.abs(ref) > 1e-3 * np.abs(ref).max()
        l2 = {p: float(np.linalg.norm(res[p] - ref) / np.linalg.norm(ref)) for p in ("fp32", "bf16")}
        pw = {p: float((np.abs(res[p] - ref)[big] / np.abs(ref)[big]).max()) for p in ("fp32", "bf16")}
        # and over u_0 alone (interface component 0)
        u0e = {p: float(np.abs(res[p][0] - ref[0]).max() / np.abs(ref[0]).max()) for p in ("fp32", "bf16")}
        # the typical size of BF16 storage rounding after 100 steps (201 passes, unit roundoff
        # 2^-8, a random walk); the GPU tests check BF16 against the oracle's rounding model
        estimate = (2 * 100 + 1) ** 0.5 * 2.0 ** -8
        return {"ms_per_step": ms, "speedup_vs_fp32": fp32_ms / ms,
                "value": mcu_step / (ms / 1e3) / 1e6, "unit": UNIT,
                "pass_ms": per_pass, "pass_frac_of_copy_bw": pass_frac,
                "max_rel_err_vs_fp64_100_steps_24cubed": err["bf16"], "rounding_estimate": estimate,
                "rel_l2_err_vs_fp64": l2["bf16"], "pointwise_rel_err_vs_fp64": pw["bf16"],
                "u0_max_rel_err_vs_fp64": u0e["bf16"], "fp32_u0_max_rel_err_vs_fp64": u0e["fp32"],
                "fp32_max_rel_err_vs_fp64_100_steps_24cubed": err["fp32"], "fp32_bound": 1e-5,
                "fp32_rel_l2_err_vs_fp64": l2["fp32"], "fp32_pointwise_rel_err_vs_fp64": pw["fp32"],
                "pointwise_support": "cells and moments with |u_fp64| > 1e-3 max |u_fp64|"}

    def batched():
        insts = synth.batch_instances(64, seed=3)
        res = {}
        for mode in ("grouped", "looped"):
            b = rtpn.Batch([(i.N, i.shape, i.h, i.bc, i.dt) for i in insts], "fp32")
            b.set_stream(stream)
            for c, i in zip(b.instances, insts):
                c.set_media(i.sigma_a, i.sigma_s, i.q)
                c.set_component(0, i.u0)  # every other moment starts at 0 (fresh context)
            if mode == "grouped":
                tile, _ = b.autotune(reps=1)
                res["tile"] = tile
            run = b.step if mode == "grouped" else b.step_looped
            run(3)
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            run(100)
            e.record(stream)
            torch.cuda.synchronize()
            res[mode] = a.elapsed_time(e) / 100
            b.close()
        # every instance alone on its own context with the kernel the library picks for it (the
        # plain FP32 path): the sum is what a launch loop could reach with no gaps between launches
        hbm, _ = peaks()
        by_order = {}
        isolated = 0.0
        for i in insts:
            with rtpn.Context(i.N, i.shape, i.h, i.bc, "fp32", i.dt) as c:
                c.set_stream(stream)
                c.set_media(i.sigma_a, i.sigma_s, i.q)
                c.set_component(0, i.u0)
                c.step(3)
                a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                c.step(20)
                e.record(stream)
                torch.cuda.synchronize()
                ms = a.elapsed_time(e) / 20
                info = c.info()
            V = i.shape[0] * i.shape[1] * i.shape[2]
            alg = V * ((info.n_c + info.n_even) * 4 + 6 + (info.n_c + info.n_odd) * 4 + 6)
            isolated += ms
            g = by_order.setdefault(str(i.N), {"instances": 0, "alg_bytes_per_step": 0, "isolated_ms": 0.0})
            g["instances"] += 1
            g["alg_bytes_per_step"] += alg
            g["isolated_ms"] += ms
        for g in by_order.values():
            g["isolated_frac_of_copy_bw"] = g["alg_bytes_per_step"] / (g["isolated_ms"] / 1e3) / 1e9 / hbm
        alg_all = sum(g["alg_bytes_per_step"] for g in by_order.values())
        frac = {k: alg_all / (res[k] / 1e3) / 1e9 / hbm for k in ("grouped", "looped")}
        mcu = sum(i.n_c * i.shape[0] * i.shape[1] * i.shape[2] for i in insts)
        return {"instances": 64, "ms_per_step_grouped": res["grouped"],
                "ms_per_step_looped": res["looped"], "speedup_vs_looped": res["looped"] / res["grouped"],
                "ms_per_step_isolated_sum": isolated, "speedup_vs_isolated_sum": isolated / res["grouped"],
                "alg_bytes_per_step": alg_all, "grouped_frac_of_copy_bw": frac["grouped"],
                "looped_frac_of_copy_bw": frac["looped"], "by_order": by_order,
                "value": mcu / (res["grouped"] / 1e3) / 1e6, "unit": UNIT, "tile": res["tile"],
                "note": "grouped: one launch per order and pass; looped: a per-instance launch loop of "
                        "the same window kernel; isolated sum: each instance alone with its own "
                        "kernel choice; error bound 1e-5 (FP32) checked in the GPU tests"}

    def adjoint():
        inst = synth.checkerboard(15, 96)
        w = synth.detector_box(96)
        c = rtpn.Context(15, inst.shape, inst.h, inst.bc, "fp32", inst.dt)
        c.set_stream(stream)
        c.set_media(inst.sigma_a, inst.sigma_s, inst.q)
        # warm-up: every kernel of both calls loaded once, and the adjoint's work buffers of this
        # layout allocated (a training loop's steady state: the context keeps them between calls)
        c.step(2)
        c.adjoint(w, 200, ckpt_every=20)
        c.zero_moments()
        c.synchronize()
        t0 = time.perf_counter()
        c.step(200)
        c.synchronize()
        t_fwd = time.perf_counter() - t0
        c.zero_moments()
        c.synchronize()
        t0 = time.perf_counter()
        J, _ = c.adjoint(w, 200, ckpt_every=20)
        t_adj = time.perf_counter() - t0
        kernel = {v: k for k, v in rtpn.KERNEL.items()}.get(c.info().kernel, "?")
        # one segment of 200 steps (every pass's output stored, nothing recomputed) where the
        # device holds it: about 201 states of 0.9 GB
        t_one = None
        state_bytes = c.info().state_bytes
        c.adjoint_release()
        if torch.cuda.mem_get_info()[0] > 1.05 * 205 * state_bytes:
            c.zero_moments()
            c.adjoint(w, 200, ckpt_every=200)
            c.zero_moments()
            c.synchronize()
            t0 = time.perf_counter()
            c.adjoint(w, 200, ckpt_every=200)
            t_one = time.perf_counter() - t0
        c.adjoint_release()
        c.close()
        V = inst.shape[0] * inst.shape[1] * inst.shape[2]
        return {"workload": "P15 96^3 checkerboard, vacuum, 200 steps, checkpoints every 20",
                "kernel": kernel, "J": J, "forward_s": t_fwd, "forward_plus_adjoint_s": t_adj,
                "workspace": "kept from the warm-up call of the same layout",
                "cost_ratio_vs_forward": t_adj / t_fwd,
                "one_segment_s": t_one,
                "one_segment_cost_ratio": (t_one / t_fwd) if t_one else None,
                "speedup_vs_central_fd": (2 * 3 * V * t_fwd) / t_adj,
                "note": "central differences of 3 per-cell fields need 2*3*V forward runs"}

    def fused():
        # the even full step and the odd step of each step in one pass between two state buffers,
        # against the window kernel's two in-place passes, at P7 128^3 (the fused kernel's ring
        # of new even planes fits shared memory up to N = 9)
        inst = synth.random_blocks(7, 128, seed=5)
        V = inst.shape[0] * inst.shape[1] * inst.shape[2]
        k = 200
        res = {}
        for kern in ("window", "fused"):
            c = rtpn.Context(7, inst.shape, inst.h, inst.bc, "fp32", inst.dt)
            c.set_stream(stream)
            c.set_kernel(kern)
            c.set_media(*[torch.tensor(a, dtype=torch.float32, device="cuda")
                          for a in (inst.sigma_a, inst.sigma_s, inst.q)])
            c.zero_moments()
            c.set_component(0, torch.tensor(inst.u0, dtype=torch.float32, device="cuda"))
            c.step(3)
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            c.step(k)
            e.record(stream)
            torch.cuda.synchronize()
            res[kern] = a.elapsed_time(e) / k
            res[kern + "_u0_sum"] = c.sum_u0()
            c.close()
        hbm, _ = peaks()
        # per step: every moment read once and written once, plus 12 B of media factors per cell
        step_bytes = V * (64 * 2 * 4 + 12)
        return {"workload": "P7 128^3 random-block media, periodic, FP32, 200 steps",
                "window_ms_per_step": res["window"], "fused_ms_per_step": res["fused"],
                "speedup_vs_window": res["window"] / res["fused"],
                "fused_step_frac_of_copy_bw": step_bytes / (res["fused"] / 1e3) / 1e9 / hbm,
                "window_step_frac_of_copy_bw": step_bytes / (res["window"] / 1e3) / 1e9 / hbm,
                "u0_sum_rel_diff": abs(res["fused_u0_sum"] - res["window_u0_sum"]) /
                                   max(abs(res["window_u0_sum"]), 1e-300),
                "value": 64 * V / (res["fused"] / 1e3) / 1e6, "unit": UNIT}

    def scattering():
        # anisotropic scattering (Henyey-Greenstein moments f_l = g^l, g = 0.8) at P7 128^3 FP32:
        # the window kernel's anisotropic form against the generic kernel and the isotropic step;
        # the three are timed in turn, twice, and each keeps its faster round
        inst = synth.random_blocks(7, 128, seed=2)
        f = [0.8 ** l for l in range(8)]
        ctxs = {}
        for name, kernel, aniso in (("window_isotropic", "window", False), ("window", "window", True),
                                    ("generic", "generic", True)):
            c = rtpn.Context(7, inst.shape, inst.h, inst.bc, "fp32", inst.dt)
            c.set_stream(stream)
            c.set_kernel(kernel)
            if aniso:
                c.set_scattering(f)
            c.set_media(inst.sigma_a, inst.sigma_s, inst.q)
            c.set_component(0, inst.u0)
            c.step(3)
            ctxs[name] = c
        res = {}
        for _ in range(2):
            for name, c in ctxs.items():
                a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                c.step(50)
                e.record(stream)
                torch.cuda.synchronize()
                ms = a.elapsed_time(e) / 50
                res[name] = min(ms, res.get(name, ms))
        for c in ctxs.values():
            c.close()
        return {"workload": "P7 128^3 random-block media, periodic, FP32, 50 steps, f_l = 0.8^l",
                "ms_per_step": res, "window_vs_isotropic": res["window"] / res["window_isotropic"],
                "speedup_vs_generic": res["generic"] / res["window"],
                "note": "error bound 1e-5 (FP32) against the oracle checked in the GPU tests"}

    def reactor():
        # the reactor-like showcase (Section 5.2) as a P_N convergence study against P39
        from paper_2004_02833_gb300 import showcase

        r = showcase.reactor_convergence(n=64, orders=(3, 7, 19, 29, 39), steps=100)
        r.pop("log10_u0_line_ref")
        return r

    wanted = set(args.forms.split(","))
    for name, fn in (("bf16", bf16), ("fused", fused), ("reactor", reactor), ("batched", batched),
                     ("adjoint", adjoint), ("scattering", scattering)):
        if name in wanted:
            out[name] = _guard(fn)
    return out


def aggregate(local_ms: float, local_units: float, dist=None, device=None):
    """Whole-job figures over ranks: (max time over ranks in ms, units of all ranks).  Ranks run
    independent replicas, so the only communication is this timing reduction."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return local_ms, local_units
    import torch

    t = torch.tensor([local_ms, local_units], dtype=torch.float64, device=device)
    mx = t[:1].clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    tot = t[1:].clone()
    dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    return float(mx.item()), float(tot.item())


def pass_durations(ctx, stream, reps: int):
    """Average duration (ms) of the even and the odd pass, each timed alone with CUDA events on the
    launching stream (one merged-schedule step = even pass + odd pass)."""
    import torch

    out = {}
    for cls in (0, 1):
        evs = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx._pass(cls)
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        out[cls] = sum(a.elapsed_time(b) for a, b in evs) / reps
    return out


def end_to_end(ctx, inst, args, mcu_step, world, dist):
    """One user job through the C ABI with pinned host buffers, every copy inside the timed region:
    upload the media and u_0 and zero the other moments; then every step its passes and a read of
    its metric (the FP64 sum of u_0 after the step's even pass, where u_0 has finished the step) to
    the host; at the end u_0 to the host.  On one rank the same job is timed once more reading the
    whole state back at the end (`full_state`; under torchrun every rank would pin a state of host
    memory)."""
    import torch

    host = [torch.tensor(a, dtype=torch.float32).pin_memory()
            for a in (inst.sigma_a, inst.sigma_s, inst.q, inst.u0)]
    h2d = sum(h.numel() * 4 for h in host)

    def job(out, read):
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        ctx.set_media(host[0], host[1], host[2])
        ctx.zero_moments()
        ctx.set_component(0, host[3])
        # the merged schedule pass by pass, with the step's metric between its even and odd passes
        ctx.substep(1, half=True)
        metrics = []
        for s in range(args.steps):
            ctx.substep(0)
            metrics.append(ctx.sum_u0())
            ctx.substep(1, half=s == args.steps - 1)
        read(out)
        ctx.synchronize()
        dt = time.perf_counter() - t0
        dt_ms, units = aggregate(dt * 1e3, float(mcu_step * args.steps), dist, device="cuda")
        d2h = 8 * args.steps + out.numel() * 4
        return {"value": units / (dt_ms / 1e3) / 1e6, "unit": UNIT,
                "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps}

    u0_out = torch.empty(inst.shape, dtype=torch.float32).pin_memory()
    e2e = job(u0_out, lambda o: ctx.get_component(0, o))
    e2e["job"] = (f"set_media + zero + set u_0 from pinned host, {args.steps} steps each with its sum "
                  f"of u_0 read to the host, then u_0 to pinned host memory")
    if world == 1:
        try:
            full = torch.empty((ctx.info().n_c,) + tuple(inst.shape), dtype=torch.float32, pin_memory=True)
        except RuntimeError:
            full = None
        if full is not None:
            e2e["full_state"] = job(full, lambda o: ctx.get_moments(o))
            e2e["full_state"]["job"] = "the same job reading the whole state back at the end"
            del full
    return e2e


if __name__ == "__main__":
    main()
