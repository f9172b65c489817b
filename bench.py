#!/usr/bin/env python
"""Throughput of the 2D QLA step (Eq. 2e14) on GB300: site-updates/s.

One bench step = ``--qla-steps`` (default 100) time steps of the whole lattice
followed by the FP64 energy reduction (Eq. A13) read back to the host, the
monitoring cadence of the 8192^2 workload.  Default workload: the largest
single-GPU lattice, 16384 x 16384 periodic, unit spacing, an elliptical vacuum
bubble (n = 1, semi-axes 2400 x 1200, tanh edge 8) in a uniform dielectric
n = 2, E_z packet k0 = 0.2, width 600 launched inside the dielectric; FP32
storage and arithmetic, E_z polarisation (q2, q3, q4 live).  The default 200
bench steps are the workload's 20000 time steps.  ``--workload ellipse_8192``
selects the 8192^2 rotated-ellipse lattice.

Prints one JSON line (rank 0).  ``--impl reference`` times the plain CPU
oracle on the host cores instead (bounded samples of the same workload).
Under torchrun each rank runs its own replica of the workload (no data
exchange: weak scaling); the time is the maximum over ranks.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HBM_FALLBACK_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--workload", default="bubble_16384")
    ap.add_argument("--qla-steps", type=int, default=100)
    ap.add_argument("--lane-cols", type=int, default=0, help="marching kernel tuning")
    ap.add_argument("--rows", type=int, default=0, help="marching kernel tuning")
    ap.add_argument("--step-kernel",
                    choices=["auto", "march", "march_plain", "march_step", "march_flow", "tile"],
                    default="auto",
                    help="step kernel (march_plain: no plateau split; march_step: plateau split, "
                         "one launch per step; march_flow: dataflow launches on any lattice)")
    ap.add_argument("--double-single", action="store_true",
                    help="FP64 contexts stepped in double-single arithmetic (QLA_DOUBLE_SINGLE)")
    ap.add_argument("--six-planes", action="store_true",
                    help="evolve all six amplitudes instead of the E_z triple")
    ap.add_argument("--surr-windows", type=int, default=20000)
    ap.add_argument("--surr-train-steps", type=int, default=16000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    return ap.parse_args()


def workload(name):
    from paper_2604_21128_gb300 import inputs
    table = {"ellipse_8192": inputs.ellipse_8192, "bubble_16384": inputs.bubble_16384,
             "ellipse_256": inputs.ellipse_256,
             # the 8192^2 geometry on 4096^2: a small case for ncu captures
             "ellipse_4096": lambda: inputs.scaled(inputs.ellipse_8192(), 4096, 4096, 20000)}
    return table[name]()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


# Arithmetic roofline of the step kernel.  Per site-update the method needs
# 16 collision rotations (8 layers of U_x, 8 of U_y) and 2 potential
# rotations on each live pair (1 pair in E_z mode, 2 with six planes).  FP32:
# a collision rotation with two-word coefficients is 8 FP32 instructions
# (4 per output), a potential rotation 6; FP64: a collision rotation is 3
# (three shears), a potential rotation 4.
# Peaks: FP32 instructions from the unit counts of the device in use (its SM
# count x 128 FP32 lanes x its maximum SM clock); FP64 from the datasheet's
# nominal 1.25 TFLOP/s counted as FMA-class instructions (2 flops each), not
# a measured rate.
FP32_LANES_PER_SM = 128
FP64_NOMINAL_FLOPS = 1.25e12
DEVICE = {"sms": None, "sm_max_mhz": None}


def device_info(dev=None):
    """SM count (from the device) and maximum SM clock (nvidia-smi, else
    MEASURED_PEAKS.json, else the GB300 figure of 2070 MHz)."""
    import torch
    if dev is not None:
        DEVICE["sms"] = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = None
        try:
            out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm",
                                  "--format=csv,noheader,nounits", "-i", str(dev.index or 0)],
                                 capture_output=True, text=True, timeout=20).stdout
            mhz = float(out.strip().splitlines()[0])
        except Exception:
            try:
                with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                    mhz = float(json.load(f)["sm_max_mhz"])
            except Exception:
                mhz = 2070.0
        DEVICE["sm_max_mhz"] = mhz
    return DEVICE


def fp32_inst_peak():
    d = DEVICE
    return d["sms"] * FP32_LANES_PER_SM * d["sm_max_mhz"] * 1e6


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def alu_ops_per_su(P, elt):
    pairs = 1 if P == 3 else 2
    if elt == 4:
        return pairs * (16 * 8 + 2 * 6)
    return pairs * (16 * 3 + 2 * 4)


def ds_ops_per_su(P):
    """Double-single: a rotation is two rows of 23 FP32 instructions (two
    exact products, a two-sum, nine correction FMAs, a fast two-sum); the
    potential rotations take the same form."""
    pairs = 1 if P == 3 else 2
    return pairs * (16 + 2) * 46


def alu_ops_per_su_3d(elt):
    """3D: per axis 8 layers x 2 pairs of collision rotations, then six
    potential rotations (two per axis)."""
    return 3 * 16 * (8 if elt == 4 else 3) + 6 * (6 if elt == 4 else 4)


def roofline(P, elt, su_per_s, traffic, ops=None, pipe=None, **extra):
    """Roofline object for a step kernel that advances ``su_per_s`` site-updates
    per second of its own run time.  The bound is the roof with the lower
    ceiling in site-updates/s (HBM for FP32, the FP64 pipe for FP64); the
    other roof's figures ride along under its name.  pipe overrides the
    arithmetic pipe ("fp32" for double-single steps on FP64 state)."""
    ops = alu_ops_per_su(P, elt) if ops is None else ops
    pipe = pipe or ("fp32" if elt == 4 else "fp64")
    peak_ops = fp32_inst_peak() if pipe == "fp32" else FP64_NOMINAL_FLOPS / 2
    hbm_peak, hbm_kind = peaks()
    bytes_su = 2 * P * elt
    hbm = {"achieved": bytes_su * su_per_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
           "frac": bytes_su * su_per_s / 1e9 / hbm_peak, "peak_kind": hbm_kind,
           "bytes_per_site_update": bytes_su}
    alu = {"achieved": ops * su_per_s / 1e12, "peak": peak_ops / 1e12,
           "unit": "T%s-inst/s" % pipe.upper(),
           "frac": ops * su_per_s / peak_ops,
           "peak_kind": ("derived: %d SMs x %d FP32 lanes x %.0f MHz (device query)"
                         % (DEVICE["sms"], FP32_LANES_PER_SM, DEVICE["sm_max_mhz"])
                         if pipe == "fp32" else
                         "nominal (not measured): 1.25 TFLOP/s FP64 datasheet rate / 2 flops "
                         "per FMA"),
           "ops_per_site_update": ops}
    ceil = {"hbm": hbm_peak * 1e9 / bytes_su, "alu": peak_ops / ops}
    bound = "hbm" if ceil["hbm"] <= ceil["alu"] else "alu"
    other = "alu" if bound == "hbm" else "hbm"
    r = {"bound": bound}
    r.update(hbm if bound == "hbm" else alu)
    r["traffic"] = traffic
    r["ceilings_site_updates_per_s"] = ceil
    r[other] = alu if other == "alu" else hbm
    r.update(extra)
    return r


# ---------------------------------------------------------------------------
# Clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.proc = None
        self.gpu_id = gpu_id

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu_id)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        return self.parse(out)

    @staticmethod
    def parse(out):
        """Median SM clock, max clock and the throttle reasons seen in the
        CSV lines of the nvidia-smi query in FIELDS."""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# Distributed helpers (replicas; the only collectives time the run)
# ---------------------------------------------------------------------------

def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, value):
    """Largest value over the ranks (the run's time is its slowest rank's)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline, and the reference arm)
# ---------------------------------------------------------------------------

def oracle_sample(w, n_full, side, steps, threads=None):
    """Time the oracle on a side x side window of the workload (the medium
    and packet of the full lattice, taken periodic on the window) for
    ``steps`` steps; returns site-updates/s, seconds and the thread count."""
    import numpy as np
    import oracle
    threads = threads or os.cpu_count() or 1
    oracle.set_threads(threads)
    # window straddling the ellipse's left edge, where the packet arrives
    i0 = max(0, int(w.packet.x0 / w.delta) + int(w.packet.width / w.delta) - side // 2)
    j0 = w.ny // 2 - side // 2
    crop = np.ascontiguousarray(n_full[j0:j0 + side, i0:i0 + side])
    q = oracle.packet(crop, w.delta, window=(i0, j0), global_shape=(w.ny, w.nx),
                      **w.packet.as_dict())
    t = time.perf_counter()
    oracle.run(q, crop, w.delta, steps)
    dt = time.perf_counter() - t
    return side * side * steps / dt, dt, oracle.get_threads()


def reference_arm(args):
    world, rank, _ = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0
    if rank != 0:
        return 0
    w = workload(args.workload)
    n_full = w.medium()
    side, per = 512, 2
    for _ in range(args.warmup):
        oracle_sample(w, n_full, side, per)
    total_t, su = 0.0, 0
    for _ in range(args.steps):
        _, dt, threads = oracle_sample(w, n_full, side, per)
        total_t += dt
        su += side * side * per
    value = su / total_t
    sample = ("%d x %d crop of the %s workload (same medium recipe and packet), %d steps per "
              "bench step, plain FP64 CPU oracle" % (side, side, w.name, per))
    line = {"impl": "reference", "metric": "site-updates/s", "value": value,
            "unit": "site-updates/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            # the GPU arm's workload label, so the two lines pair up
            "config": {"workload": w.name + ("_fp32" if args.precision == "fp32" else "_fp64")
                       + ("_ds" if args.double_single and args.precision == "fp64" else "")
                       + ("_6planes" if args.six_planes else "_ez"),
                       "nx": w.nx, "ny": w.ny, "delta": w.delta, "sample": sample},
            "cpu_baseline": {"value": value, "unit": "site-updates/s", "cores": threads,
                             "cpu_model": cpu_model(), "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "site-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def kernel_traffic(k, sites, record):
    """DRAM bytes per step-kernel launch (per step for the 3D passes) from a
    committed ncu record of this workload, if it was taken on the current
    kernel sources with the same steps per launch; else None."""
    path = os.path.join(ROOT, "profiles", record)
    try:
        with open(path) as f:
            rec = json.load(f)
    except Exception:
        return None
    h = hashlib.sha256()
    try:
        for name in rec["sources"]:
            h.update(open(os.path.join(ROOT, "paper_2604_21128_gb300", "csrc", name), "rb").read())
    except (OSError, KeyError):
        return None
    sha = h.hexdigest()
    if sha != rec.get("sources_sha256") or rec.get("time_block") != k:
        return None
    return rec["dram_bytes_per_site_step"] * sites * k


def gpu_arm(args):
    import numpy as np
    import torch

    from paper_2604_21128_gb300 import build as qbuild
    from paper_2604_21128_gb300 import inputs, qla

    world, rank, local = dist_setup()
    if world == 1:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    device_info(dev)
    qbuild.build()
    w = workload(args.workload)
    te = not args.six_planes
    P = 3 if te else 6
    elt = 4 if args.precision == "fp32" else 8
    n_host = torch.from_numpy(w.medium()).pin_memory()
    pk = w.packet.as_dict()
    S = args.qla_steps
    sites = w.nx * w.ny

    stream = torch.cuda.Stream(dev)
    ds = bool(args.double_single and args.precision == "fp64")
    g = qla.Grid(w.nx, w.ny, w.delta, args.precision, te_only=te, stream=stream,
                 double_single=ds)
    g.set_step_kernel(args.step_kernel)
    g.set_march_tuning(args.lane_cols, args.rows)
    g.set_medium(n_host)
    g.set_packet(**pk)
    e0 = g.energy()

    for _ in range(args.warmup):
        g.step(S)
        g.energy()
    torch.cuda.synchronize(dev)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local if world > 1 else 0)
    barrier(world)
    torch.cuda.synchronize(dev)
    launches0 = g.launches
    step_launches = 0
    sampler.start()
    time.sleep(0.3)
    start.record(stream)
    energies = []
    for k in range(args.steps):
        l0 = g.launches
        ev[k][0].record(stream)
        g.step(S)
        ev[k][1].record(stream)
        step_launches += g.launches - l0
        energies.append(g.energy())
    stop.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    launches = g.launches - launches0
    plan = g.march_plan
    flow_rows = g.flow_plan
    elapsed = start.elapsed_time(stop) / 1e3
    step_time = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    elapsed = max_over_ranks(world, elapsed)
    barrier(world)
    su_total = world * args.steps * S * sites
    value = su_total / elapsed
    drift = energies[-1] / e0 - 1 if e0 else float("nan")

    # roofline of the dominant (step) kernel: algorithmic work per launch =
    # per-site-update figure x sites x steps per launch, over the launch's
    # mean duration (CUDA events on the launching stream)
    k_used = S * args.steps / max(step_launches, 1)
    per_launch_s = step_time / max(step_launches, 1)
    kernel_su_per_s = sites * k_used / per_launch_s
    # the committed DRAM records are of the FP32 E_z step kernel, one per
    # workload, taken with the default marching tuning
    traffic = (kernel_traffic(int(round(k_used)), sites,
                              "traffic_%s_fp32_ez.json" % args.workload)
               if args.precision == "fp32" and te and not ds and not args.lane_cols
               and not args.rows and args.step_kernel == "auto" else None)
    g.close()

    e2e = None
    if not args.no_e2e:
        e2e = e2e_run(args, w, te, n_host, pk, world, dev)

    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        side, nst = 4096, 15
        v, dt, threads = oracle_sample(w, n_host.numpy(), side, nst)
        cpu = {"value": v, "unit": "site-updates/s", "cores": threads,
               "cpu_model": cpu_model(), "kind": "oracle",
               "sample": "%d x %d crop of the %s workload, %d steps (%.1f s), plain FP64 "
                         "CPU oracle, OpenMP over rows" % (side, side, w.name, nst, dt)}
        # the same oracle on one thread, and the 256^2 parity workload run in full
        v1, dt1, _ = oracle_sample(w, n_host.numpy(), 1024, 3, threads=1)
        cpu["single_thread"] = {"value": v1, "sample": "1024 x 1024 crop, 3 steps (%.1f s)" % dt1}
        import oracle
        small = inputs.ellipse_256()
        n_small = small.medium()
        q_small = oracle.packet(n_small, small.delta, **small.packet.as_dict())
        oracle.set_threads(threads)
        t0 = time.perf_counter()
        oracle.run(q_small, n_small, small.delta, small.steps)
        dts = time.perf_counter() - t0
        cpu["ellipse_256_full"] = {"value": small.nx * small.ny * small.steps / dts,
                                   "seconds": dts, "steps": small.steps}

    if rank == 0:
        line = {
            "metric": "site-updates/s", "value": value, "unit": "site-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else ("f32x2" if ds else "f64"),
            "data": "synthetic",
            "config": {"workload": w.name + ("_fp32" if elt == 4 else "_fp64")
                       + ("_ds" if ds else "") + ("_ez" if te else "_6planes"),
                       "nx": w.nx, "ny": w.ny, "delta": w.delta,
                       "qla_steps_per_bench_step": S, "planes": P,
                       "potential": "rotation", "steps_per_launch": k_used,
                       "lane_cols": args.lane_cols or "auto", "rows": args.rows or "auto",
                       "step_kernel": args.step_kernel,
                       "plateau_items": "%d of %d work items, %d plateaus" % (plan[1], plan[0],
                                                                             plan[2]),
                       "dataflow": ("%d-row segments, %d steps per launch" % (flow_rows, k_used)
                                    if flow_rows else None),
                       "energy_drift": drift,
                       "l2": "state %.0f MB > 129 MB L2, no flush" % (2 * P * elt * sites / 2e6)},
            "roofline": roofline(P, elt, kernel_su_per_s, traffic,
                                 ops=ds_ops_per_su(P) if ds else None,
                                 pipe="fp32" if ds else None,
                                 kernel_ms=1e3 * per_launch_s,
                                 **({"note": "double-single steps on FP64 state: FP32-pipe "
                                             "instructions; two in-place conversions per "
                                             "%d-step call included" % S} if ds else {})),
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def e2e_run(args, w, te, n_host, pk, world, dev):
    """Same metric through the public API from host buffers: the medium
    copied from pinned host memory, the packet built, every bench step's
    energy read back, the final E_z copied to pinned host memory."""
    import torch
    from paper_2604_21128_gb300 import qla
    stream = torch.cuda.Stream(dev)
    ez = torch.empty((w.ny, w.nx), dtype=torch.float64).pin_memory()
    g = qla.Grid(w.nx, w.ny, w.delta, args.precision, te_only=te, stream=stream,
                 double_single=bool(args.double_single and args.precision == "fp64"))
    g.set_step_kernel(args.step_kernel)
    g.set_march_tuning(args.lane_cols, args.rows)
    S = args.qla_steps
    barrier(world)
    torch.cuda.synchronize(dev)
    t = time.perf_counter()
    g.set_medium(n_host)
    g.set_packet(**pk)
    for _ in range(args.steps):
        g.step(S)
        g.energy()
    qla.qla_fields(g._ctx, w.nx, w.ny, Ez=ez)
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t
    dt = max_over_ranks(world, dt)
    g.close()
    sites = w.nx * w.ny
    return {"value": world * args.steps * S * sites / dt, "unit": "site-updates/s",
            "h2d_bytes_per_step": 8 * sites / args.steps,
            "d2h_bytes_per_step": 8 + 8 * sites / args.steps}


def batch_arm(args):
    """256 uneven lattices (sides 512-2048, seeded) advanced together: the
    batched persistent, graph-captured path.  One bench step = --qla-steps
    steps of every lattice plus all their energies."""
    import numpy as np
    import torch

    from paper_2604_21128_gb300 import build as qbuild
    from paper_2604_21128_gb300 import inputs, qla

    world, rank, local = dist_setup()
    if world == 1:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    device_info(dev)
    qbuild.build()
    ws = inputs.batch_instances()
    sizes = [(w.nx, w.ny) for w in ws]
    sites = sum(w.nx * w.ny for w in ws)
    stream = torch.cuda.Stream(dev)
    b = qla.Batch(sizes, 1.0, args.precision, te_only=True, stream=stream)
    for k, w in enumerate(ws):
        g = b.instance(k)
        g.set_medium(w.medium())
        g.set_packet(**w.packet.as_dict())
    S = args.qla_steps
    if args.lane_cols or args.rows:
        b.set_tuning(args.lane_cols, args.rows)
        tuned = (args.lane_cols or "auto", args.rows or "auto")
    else:
        tuned = b.autotune(trial_steps=2)
    b.run(args.warmup * S, S)
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local if world > 1 else 0)
    barrier(world)
    l0 = b.launches
    sampler.start()
    time.sleep(0.3)
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    t0 = time.perf_counter()
    energies = b.run(args.steps * S, S)
    stop.record(stream)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    elapsed = max_over_ranks(world, start.elapsed_time(stop) / 1e3)
    launches = b.launches - l0
    b.close()
    value = world * args.steps * S * sites / elapsed
    elt = 4 if args.precision == "fp32" else 8
    bytes_per_su = 2 * 3 * elt
    if rank == 0:
        drift = float(np.max(np.abs(energies[-1] / energies[0] - 1)))
        print(json.dumps({
            "metric": "site-updates/s", "value": value, "unit": "site-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": "batch_256_uneven_%s_ez" % args.precision,
                       "instances": len(ws), "sites": sites,
                       "sides": sorted(set(w.nx for w in ws)),
                       "qla_steps_per_bench_step": S, "tuning": list(tuned),
                       "launch": "persistent cooperative kernel per chunk, whole run "
                                 "captured as one CUDA graph",
                       "max_energy_drift": drift,
                       "l2": "state %.1f GB > 129 MB L2, no flush" % (bytes_per_su * sites / 1e9)},
            "roofline": roofline(3, elt, value / world, None,
                                 note="whole-run average (step kernels and energies)"),
            "cpu_baseline": None,
            "e2e": {"value": world * args.steps * S * sites / wall, "unit": "site-updates/s",
                    "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 8 * len(ws),
                    "note": "host wall clock around the graph run"},
            "gpu_launches": launches, "clocks": clocks}), flush=True)
    return 0


def surrogate_arm(args):
    """Learned surrogate on 256^2 lattices: train on windows from the
    library's own runs, then advance 64 chained windows of K = 32 steps on
    held-out lattices with the energy / div B checks and QLA fallback, and
    compare time and final state with plain GPU QLA (the reference run)."""
    import numpy as np
    import torch

    from paper_2604_21128_gb300 import build as qbuild
    from paper_2604_21128_gb300 import inputs, qla
    from paper_2604_21128_gb300 import surrogate as S

    torch.cuda.set_device(0)
    qbuild.build()
    size, K, windows = 256, 32, 64
    t0 = time.perf_counter()
    X, T = S.make_windows(args.surr_windows, size=size, K=K, seed=5, instances=64,
                          restart_every=16)
    t_gen = time.perf_counter() - t0
    net = S.Surrogate(size, size, max_batch=8, seed=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = S.train(net, X, T, steps=args.surr_train_steps, batch=8, lr=1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    target_var = float(T.pow(2).mean())
    del X, T
    rng = np.random.default_rng(20261203)
    rows = []
    for inst in range(4):
        med, pk = inputs.surrogate_instance(rng, size)
        n = inputs.ellipse_medium(size, size, 1.0, **med)
        with qla.Grid(size, size, 1.0, "fp32", te_only=True) as g:
            g.set_medium(n)
            g.set_packet(**pk)
            g.step(K)   # warm the kernels
            g.set_packet(**pk)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g.step(windows * K)
            g.energy()
            t_qla = time.perf_counter() - t0
            ref = g.get_state()
        with qla.Grid(size, size, 1.0, "fp32", te_only=True) as g:
            # the network alone over one window, against QLA and against
            # the zero-change predictor (the state left as it was)
            g.set_medium(n)
            g.set_packet(**pk)
            f0 = S.features(g).unsqueeze(0).contiguous()
            y = net.forward(f0)[0]
            g.step(K)
            d = S.features(g)[..., :3] - f0[0, ..., :3]
            one = float((y - d).norm() / (f0[0, ..., :3] + d).norm())
            zero = float(d.norm() / (f0[0, ..., :3] + d).norm())
        for name, etol, dtol in (("checked", 2e-3, 3e-2), ("unchecked", 1e30, 1e30)):
            with qla.Grid(size, size, 1.0, "fp32", te_only=True) as g:
                g.set_medium(n)
                g.set_packet(**pk)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                acc, _ = net.advance(g, windows, K, etol, dtol)
                torch.cuda.synchronize()
                t_s = time.perf_counter() - t0
                got = g.get_state()
            err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
            rows.append(dict(instance=inst, mode=name, accepted=acc, rel_l2=err,
                             one_window_rel_l2=one, zero_predictor_rel_l2=zero,
                             t_qla_ms=1e3 * t_qla, t_surr_ms=1e3 * t_s, speedup=t_qla / t_s))
    checked = [r for r in rows if r["mode"] == "checked"]
    unchecked = [r for r in rows if r["mode"] == "unchecked"]
    line = {
        "metric": "surrogate speedup over plain GPU QLA at <=1e-2 relative L2 error",
        "value": float(np.mean([r["speedup"] for r in checked])), "unit": "x",
        "n_gpus": 1, "steps": windows, "warmup": 1, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16/f32", "data": "synthetic",
        "config": {"workload": "surrogate_256_K32_64_windows", "train_windows": args.surr_windows,
                   "train_steps": args.surr_train_steps, "train_s": t_train, "gen_s": t_gen,
                   "final_loss_over_target_var": float(np.mean(losses[-100:]) / target_var),
                   "checks": "energy 2e-3, div B 3e-2"},
        "checked": {"rel_l2": float(np.max([r["rel_l2"] for r in checked])),
                    "accepted_windows": int(sum(r["accepted"] for r in checked)),
                    "of_windows": windows * len(checked)},
        "unchecked": {"rel_l2": float(np.max([r["rel_l2"] for r in unchecked])),
                      "speedup": float(np.mean([r["speedup"] for r in unchecked]))},
        "rows": rows,
    }
    print(json.dumps(line), flush=True)
    return 0


def cube_arm(args):
    """3D workload (qla3_*): an E_z packet into a dielectric ellipsoid on a
    256^3 lattice; a bench step is --qla-steps steps (three launches each)
    and one energy read.  The packet state is built here on the host (the
    Dyson map q2 = n E_z and the plane-wave B of a +x wave, q4 = -q2) and
    handed to both arms as input data."""
    import numpy as np
    import torch

    from paper_2604_21128_gb300 import build as qbuild
    from paper_2604_21128_gb300 import inputs, qla

    world, rank, local = dist_setup()
    if world == 1:
        torch.cuda.set_device(0)
    device_info(torch.device("cuda", torch.cuda.current_device()))
    qbuild.build()
    w = inputs.cube_256()
    N, d = w["n"], w["delta"]
    n3 = inputs.ellipsoid_medium3(N, N, N, d, **w["medium"])
    x = np.arange(N) * d
    pk = w["packet"]
    f = np.exp(-(x - pk["x0"]) ** 2 / pk["width"] ** 2) * np.cos(pk["k0"] * (x - pk["x0"]))
    q = np.zeros((6, N, N, N))
    q[2] = n3 * f[None, None, :]
    q[4] = -q[2]
    elt = 4 if args.precision == "fp32" else 8
    S = max(1, args.qla_steps // 5)
    sites = N ** 3
    stream = torch.cuda.Stream()
    ds = bool(args.double_single and args.precision == "fp64")
    g = qla.Grid3(N, N, N, d, args.precision, stream=stream, double_single=ds)
    t_e2e = time.perf_counter()
    g.set_medium(n3)
    g.set_state(q)
    e0 = g.energy()
    for _ in range(args.warmup):
        g.step(S)
        g.energy()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    sampler = ClockSampler(local if world > 1 else 0)
    barrier(world)
    torch.cuda.synchronize()
    l0 = g.launches
    sampler.start()
    time.sleep(0.3)
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for k in range(args.steps):
        ev[k][0].record(stream)
        g.step(S)
        ev[k][1].record(stream)
        e = g.energy()
    stop.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    launches = g.launches - l0
    elapsed = max_over_ranks(world, start.elapsed_time(stop) / 1e3)
    step_time = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    final = g.get_state()
    t_e2e = time.perf_counter() - t_e2e
    g.close()
    value = world * args.steps * S * sites / elapsed
    kernel_su = args.steps * S * sites / step_time
    total_steps = (args.warmup + args.steps) * S
    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        import oracle
        side, nst = 128, 10
        nw = np.ascontiguousarray(n3[:side, :side, :side])
        qw = np.ascontiguousarray(q[:, :side, :side, :side])
        threads = os.cpu_count() or 1
        oracle.set_threads(threads)
        t0 = time.perf_counter()
        oracle.run3(qw, nw, d, nst)
        dt = time.perf_counter() - t0
        cpu = {"value": side ** 3 * nst / dt, "unit": "site-updates/s", "cores": threads,
               "cpu_model": cpu_model(),
               "kind": "oracle",
               "sample": "%d^3 corner of the cube_256 workload (periodic), %d steps (%.1f s), "
                         "plain FP64 CPU oracle" % (side, nst, dt)}
    if rank == 0:
        print(json.dumps({
            "metric": "site-updates/s", "value": value, "unit": "site-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if elt == 4 else ("f32x2" if ds else "f64"), "data": "synthetic",
            "config": {"workload": "cube_256_%s%s_3d" % (args.precision, "_ds" if ds else ""),
                       "n": N, "delta": d,
                       "qla_steps_per_bench_step": S, "planes": 6,
                       "launches_per_qla_step": 2 if elt == 4 or ds else 3,
                       "energy_drift": e / e0 - 1,
                       "l2": "state %.0f MB > 129 MB L2, no flush" % (12 * elt * sites / 1e6)},
            "roofline": roofline(6, elt, kernel_su,
                                 kernel_traffic(1, sites, "traffic_cube256.json") if elt == 4
                                 else None,
                                 ops=(3 * 16 * 2 + 6) * 46 if ds else alu_ops_per_su_3d(elt),
                                 pipe="fp32" if ds else None,
                                 kernel_ms_per_qla_step=1e3 * step_time / (args.steps * S),
                                 note="double-single slices + column pipeline on FP64 state (2 launches; two in-place conversions per call)" if ds else
                                 "automatic step kernel: FP32 slices + column pipeline (2 launches), FP64 per-axis passes (3)"),
            "cpu_baseline": cpu,
            "e2e": {"value": total_steps * sites / t_e2e, "unit": "site-updates/s",
                    "h2d_bytes_per_step": (q.nbytes + n3.nbytes) / (args.steps + args.warmup),
                    "d2h_bytes_per_step": (final.nbytes + 8 * (args.steps + args.warmup + 1))
                                          / (args.steps + args.warmup),
                    "note": "host wall clock: medium and state in, all steps, energies, "
                            "state out"},
            "gpu_launches": launches, "clocks": clocks}), flush=True)
    return 0


def main():
    args = parse()
    if args.workload == "cube_256" and args.impl != "reference":
        return cube_arm(args)
    if args.workload == "surrogate256":
        return surrogate_arm(args)
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload == "batch256":
        return batch_arm(args)
    return gpu_arm(args)


if __name__ == "__main__":
    sys.exit(main())
