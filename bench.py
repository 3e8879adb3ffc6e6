#!/usr/bin/env python
"""Coupled-step throughput (MLUPS) of the ferrofluid compound-droplet step.

Workload: the 1600x200 FP32 production channel (core ferrofluid, chi 2,
rho_r = nu_r = 2, Ca 0.2, Bo_m 3, alpha 90 deg, r1 30, r2 60). One step is
one pass of the whole hot path: phase recovery, multigrid potential solve to
the channel's tolerance, fused forces + MRT/BGK collide-stream, step counter.

The state (69 MB) fits in L2, so a 256 MiB buffer is written between timed
steps and only the step itself sits between the CUDA events. Multi-GPU runs
(torchrun) are independent replicas of the channel, one per GPU.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# more hardware work queues, so that the streams of a batch run concurrently
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

METRIC = "coupled-step MLUPS vs HBM roofline; plain vs batched/adjoint at stated error"
DEFAULT_WORKLOAD = "1600x200"
UNIT = "MLUPS"
FALLBACK_HBM_GBS = 6800.0
# Algorithmic bytes per node of one collide-stream launch in FP32: f read+write
# (18 x 4), g read+write (36 x 4), phi_1, phi_2 read (8), psi' read (4) and the
# stored u_x, u_y, p* (12).
COLLIDE_BYTES_PER_NODE_F32 = 240
# DRAM bytes (read + write) per collide launch measured by ncu, keyed by the hash
# of the kernel source they were taken on, the workload and the collide's tile
# rows (null once the source changes). On 1600x200 the 37 MB of output stays in
# L2 when the launch ends, so only the reads reach DRAM inside the launch.
NCU_TRAFFIC = {
    ("b5b068562d18f977", "1600x200", 4): 38430464 + 242432,
    ("b5b068562d18f977", "1600x200", 8): 38433536 + 257792,
    ("b5b068562d18f977", "9600x1200", 4): 1383248896 + 1206289152,
    ("b5b068562d18f977", "9600x1200", 8): 1383520256 + 1206574080,
}


def _workloads():
    from paper_2410_11129_gb300 import workloads as W
    return {"1600x200": W.C2, "200x40": W.C1, "2400x300": W.C3, "800x100": W.C5,
            "9600x1200": W.ROOF, "900x150-open": W.PAPER}


WORKLOADS = _workloads()


def kernel_source_hash():
    p = os.path.join(ROOT, "paper_2410_11129_gb300", "csrc", "fcd_lbm.cu")
    with open(p, "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi samples (200 ms) of the GPU during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, uuid):
        self.uuid = uuid
        self.rows = []
        self.proc = None
        self.t = None

    def start(self):
        cmd = ["nvidia-smi", "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits",
               "-lms", "200"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.t:
            self.t.join(timeout=5)
        sm, mx, reasons = [], None, set()
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for name, v in zip(self.NAMES, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_throughput(total_ms, nodes, steps, ws, device=None):
    """Whole-job throughput of independent replicas: every rank advanced its own
    channel by `steps` steps; the job takes as long as the slowest rank."""
    if ws > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return nodes * steps * ws / (total_ms * 1e-3) / 1e6, total_ms


def measure_batched(steps, warmup):
    """The 96-instance regime sweep (FP32, Bo_m x Ca x {core, shell}, lengths
    800-2400 x 200, 29 M nodes, 8 GB of state: larger than L2) at one
    tolerance: fcd_batch_step as it stands after its first steps chose a mode
    (value), each mode fixed (the batched kernels: one launch per kernel over a
    tile work list spanning every instance, one multigrid loop for all; and
    every instance's own step graph on its own stream), and the plain method
    looped over the instances on one stream."""
    import torch
    from paper_2410_11129_gb300 import fcd
    from paper_2410_11129_gb300 import workloads as W
    cfgs = [dict(c, precision="fp32") for c in W.regime_sweep()]
    nodes = sum(c["nx"] * c["ny"] for c in cfgs)
    stream = torch.cuda.current_stream()
    batch = fcd.Batch(cfgs)
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(run, warm):
        run(warm)
        torch.cuda.synchronize()
        a.record(stream)
        run(steps)
        z.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(z)

    # The first 6 steps time both modes, one step per call; 4 more in one call
    # instantiate the graphs of a multi-step call (both buffer parities, with and
    # without the macroscopic output), as the warm-up of each fixed mode does.
    t_auto = timed(batch.step, max(warmup, 6) + 4)
    tuning = batch.tuning()
    batch.set_mode(1)
    t_kernels = timed(batch.step, 4)
    batch.set_mode(0)
    t_streams = timed(batch.step, 4)
    L = fcd.load()
    for inst in batch.instances:  # the plain method: one instance after the other
        L.fcd_set_stream(inst.h, stream.cuda_stream)

    def looped(n):
        for _ in range(n):
            for inst in batch.instances:
                inst.step(1)

    t_loop = timed(looped, 2)  # both buffer parities' graphs before the timed steps
    obs = batch.observe(allow=(fcd.FCD_ENOCONV,))
    batch.close()
    v = lambda t: nodes * steps / (t * 1e-3) / 1e6
    return {"workload": "regime sweep, 96 channels 800-2400 x 200, fp32, seed 12345",
            "nodes": nodes, "steps": steps, "mag_tol": cfgs[0]["mag_tol"],
            "value": v(t_auto), "mode_chosen": {1: "batched kernels", 0: "instance streams"}.get(
                tuning["mode"], "timing"),
            "batched_kernels_value": v(t_kernels), "instance_streams_value": v(t_streams),
            "looped_value": v(t_loop), "unit": UNIT, "speedup": v(t_auto) / v(t_loop),
            "collide_tile_height": tuning["tile_h"],
            "max_mag_resid": max(o["mag_resid"] for o in obs)}


def stage_split(ch, flush, steps):
    """Mean per-stage device times (phase recovery, potential solve, collide-stream;
    ms) over `steps` steps with profiling event nodes in the step graph (an L2
    flush before each unless flush is None); returns (stages, steps, ms per step
    with the nodes)."""
    import torch
    ch.set_profiling(True)
    stage = {"phase": 0.0, "solve": 0.0, "collide": 0.0}
    total = 0.0
    for _ in range(steps):
        if flush is not None:
            flush.zero_()
        ch.step(1)
        prof = ch.last_step_profile()  # synchronises on the step's last event
        for k in stage:
            stage[k] += prof[k] / steps
        total += prof["step"] / steps
    ch.set_profiling(False)
    torch.cuda.synchronize()
    return stage, steps, total


def measure_large(steps, warmup, peak, peak_kind):
    """Whole step and collide roofline on the 9600x1200 FP32 channel (11.5 M
    nodes, 2.5 GB of state, far larger than L2): the grid on which the HBM
    fraction is quoted. Timed without event nodes in the step graph; the stage
    split comes from a second pass, as in the main measurement."""
    import torch
    from paper_2410_11129_gb300 import fcd
    cfg = dict(WORKLOADS["9600x1200"])
    N = cfg["nx"] * cfg["ny"]
    ch = fcd.Channel(cfg)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        ch.step(1)
    torch.cuda.synchronize()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    st0 = ch.solver_stats()
    for i in range(steps):  # 2.5 GB of state: no L2 flush needed
        ev0[i].record(stream)
        ch.step(1)
        ev1[i].record(stream)
    torch.cuda.synchronize()
    total = sum(a.elapsed_time(b) for a, b in zip(ev0, ev1))
    st1 = ch.solver_stats()
    stage, prof_steps, prof_ms = stage_split(ch, None, steps)
    tile_h = ch.collide_tile_height()
    ch.close()
    coll = stage["collide"]
    bpn = COLLIDE_BYTES_PER_NODE_F32
    achieved = bpn * N / (coll * 1e-3) / 1e9
    return {"workload": cfg["name"], "steps": steps, "value": N * steps / (total * 1e-3) / 1e6,
            "unit": UNIT, "ms_per_step": total / steps,
            "stage_ms_per_step": stage,
            "stage_split": "%d further steps with per-stage event nodes (%.4f ms per step with them)"
                           % (prof_steps, prof_ms),
            "solver_per_step": {k: (st1[k] - st0[k]) / steps for k in st0},
            "roofline": {"bound": "hbm", "kernel": "collide_kernel (fp32)", "achieved": achieved,
                         "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": NCU_TRAFFIC.get((kernel_source_hash(), "9600x1200", tile_h)),
                         "algorithmic_bytes_per_launch": bpn * N, "launch_ms": coll,
                         "collide_tile_height": tile_h}}


def oracle_rate(cfg, min_seconds, max_steps, warmup=1, threads=1):
    """MLUPS of the FP64 C oracle over a bounded sample, its node loops on
    `threads` host threads (the results do not depend on the count)."""
    import oracle
    oracle.build()
    oracle.set_threads(threads)
    sim = oracle.Sim(dict(cfg, mag_max_iter=100000))
    for _ in range(warmup):
        sim.step(1)
    t0 = time.perf_counter()
    n = 0
    while n < max_steps and (n == 0 or time.perf_counter() - t0 < min_seconds):
        sim.step(1)
        n += 1
    dt = time.perf_counter() - t0
    return cfg["nx"] * cfg["ny"] * n / dt / 1e6, n, dt


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2410_11129_gb300 import workloads as W
    cfg = dict(W.C2)
    budget = float(os.environ.get("FCD_REF_BUDGET_S", "150"))
    import oracle
    oracle.build()
    cores = oracle.max_threads()
    oracle.set_threads(cores)
    sim = oracle.Sim(dict(cfg, mag_max_iter=100000))
    for _ in range(args.warmup):
        sim.step(1)
    times = []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        t0 = time.perf_counter()
        sim.step(1)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_all > budget:
            break
    N = cfg["nx"] * cfg["ny"]
    tot = sum(times)
    value = N * len(times) / tot / 1e6
    sample = ("%s, %d of %d timed steps after %d warm-up steps (whole-grid FP64 oracle steps; "
              "the run stops at a %.0f s budget)" % (cfg["name"], len(times), args.steps,
                                                     args.warmup, budget))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": len(times), "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": cfg["name"], "nx": cfg["nx"], "ny": cfg["ny"],
                   "mag_tol": cfg["mag_tol"], "parallelism": "host, %d threads" % cores},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2410_11129_gb300 import fcd
    from paper_2410_11129_gb300 import workloads as W

    cfg = dict(WORKLOADS[args.workload])
    if args.precision:
        cfg["precision"] = args.precision
        cfg["name"] = cfg["name"].rsplit("-fp", 1)[0] + "-" + args.precision
    N = cfg["nx"] * cfg["ny"]
    ch = fcd.Channel(cfg)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        flush.zero_()
        ch.step(1)
    barrier()
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        uuid = None
    clk = ClockSampler(uuid)
    clk.start()
    time.sleep(0.3)
    n0 = ch.kernel_launches()
    st0 = ch.solver_stats()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    for i in range(args.steps):
        flush.zero_()                 # L2 flush, outside the timed interval
        ev0[i].record(stream)
        ch.step(1)
        ev1[i].record(stream)
    barrier()
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    n1 = ch.kernel_launches()
    st1 = ch.solver_stats()
    obs = ch.observe(allow=(fcd.FCD_ENOCONV,))
    clocks = clk.stop()
    value, total_ms = replica_throughput(sum(step_ms), N, args.steps, ws, dev)
    # Stage split from a separate pass with event nodes in the step graph (they
    # add node latency, so the timed steps above run without them).
    stage, prof_steps, prof_ms = stage_split(ch, flush, min(args.steps, 300))

    # End to end through the C ABI with host buffers: state in (h2d), one step,
    # state out (d2h), every step.
    nb = ch.state_bytes()
    host_in = torch.empty(nb, dtype=torch.uint8, pin_memory=True)
    host_out = torch.empty(nb, dtype=torch.uint8, pin_memory=True)
    ch.get_state(host_in)
    ke = max(3, min(args.steps, 50))
    for _ in range(2):
        ch.set_state(host_in)
        ch.step(1)
        ch.get_state(host_out)
    barrier()
    t0 = time.perf_counter()
    for _ in range(ke):
        ch.set_state(host_in)
        ch.step(1)
        ch.get_state(host_out)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / ke
    e2e = {"value": N * ws / e2e_s / 1e6, "unit": UNIT, "h2d_bytes_per_step": nb,
           "d2h_bytes_per_step": nb, "steps": ke}

    peak, peak_kind = measured_peak()
    coll_ms = stage["collide"]
    bpn = COLLIDE_BYTES_PER_NODE_F32 * (2 if cfg["precision"] == "fp64" else 1)
    achieved = bpn * N / (coll_ms * 1e-3) / 1e9
    h = kernel_source_hash()
    tile_h = ch.collide_tile_height()
    traffic = NCU_TRAFFIC.get((h, args.workload, tile_h))
    roofline = {"bound": "hbm", "kernel": "collide_kernel (%s)" % cfg["precision"],
                "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                "frac": achieved / peak,
                "traffic": traffic,
                "algorithmic_bytes_per_launch": bpn * N, "launch_ms": coll_ms,
                "collide_tile_height": tile_h}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if cfg["precision"] == "fp64" else "f32", "data": "synthetic",
        "config": {"workload": cfg["name"], "nx": cfg["nx"], "ny": cfg["ny"],
                   "precision": cfg["precision"], "mag_tol": cfg["mag_tol"],
                   "l2": "256 MiB buffer written between timed steps",
                   "parallelism": "replicas x%d" % ws},
        "stage_ms_per_step": stage,
        "stage_split": "%d further steps with per-stage event nodes in the step graph "
                       "(%.4f ms per step with them)" % (prof_steps, prof_ms),
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": int(n1 - n0),
        "mag_cycles_last_solve": obs["mag_iters"], "mag_resid_last_solve": obs["mag_resid"],
        "solver_per_step": {k: (st1[k] - st0[k]) / args.steps for k in st0},
        "clocks": clocks,
    }
    if args.large_steps > 0 and args.workload == DEFAULT_WORKLOAD and ws == 1:
        line["large_grid"] = measure_large(args.large_steps, 3, peak, peak_kind)
    if args.gradient_steps > 0 and args.workload == DEFAULT_WORKLOAD and ws == 1:
        try:
            from paper_2410_11129_gb300 import gradient
            line["gradient"] = gradient.compare(WORKLOADS["800x100"], args.gradient_steps)
        except Exception as e:  # reported in the line; the headline numbers stand
            line["gradient"] = {"error": "%s: %s" % (type(e).__name__, e)}
    if args.batched_steps > 0 and args.workload == DEFAULT_WORKLOAD and ws == 1:
        try:
            line["batched"] = measure_batched(args.batched_steps, 3)
        except Exception as e:  # reported in the line; the headline numbers stand
            line["batched"] = {"error": "%s: %s" % (type(e).__name__, e)}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and args.workload == DEFAULT_WORKLOAD:
        import oracle
        cores = oracle.max_threads()
        for threads, key in ((cores, "cpu_baseline"), (1, "cpu_baseline_1thread")):
            v, n, dt = oracle_rate(cfg, min_seconds=10.0, max_steps=60, threads=threads)
            line[key] = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "%s, %d whole-grid FP64 oracle steps (%.1f s) after "
                                   "initialisation and one warm-up step, %d thread(s)"
                                   % (cfg["name"], n, dt, threads)}
    ch.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--gradient-steps", type=int, default=2000,
                    help="steps of the 800x100 gradient comparison, checkpoints every 500 "
                         "(0: skip)")
    ap.add_argument("--large-steps", type=int, default=50,
                    help="steps timed on the 9600x1200 channel (0: skip)")
    ap.add_argument("--batched-steps", type=int, default=10,
                    help="steps of the batched-vs-looped regime sweep (0 skips it)")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS),
                    help="the default is the benchmark workload; the others are extra data points")
    ap.add_argument("--precision", default=None, choices=["fp64", "fp32", "fp32_offset"],
                    help="storage form (default: the workload's)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
