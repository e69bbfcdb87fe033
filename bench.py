#!/usr/bin/env python3
"""Throughput of the ensemble SSA hot path on one GB300: reaction events/s
including grid alignment and the mean/variance reduction.

A step is one full ssa_ensemble_run of the HIV-shaped four-species model
(65,536 trajectories per GPU, t_end = 30, 3001-point grid, FP64 exact mode):
work-counter reset, grid, the simulation kernel (direct method + on-device
time-aligned difference sums), and the finalisation kernel (grid scans,
sums, mean, variance).  Inputs are resident on the device; each step uses a
new seed.  L2 is flushed (256 MiB write) between timed steps, outside the
timed events.

--workload random runs the random 32-species / 128-reaction network instead
(262,144 trajectories, t_end = 10, 1001-point grid), which the library runs
one trajectory per warp with the W32 summation schedule.

--impl reference times the oracle (plain single-threaded C++ per trajectory,
run on all host cores over trajectory-id ranges) on a bounded sample of the
same workload.

With torchrun (N > 1) every rank runs its own shard (trajectory ids offset by
rank * 65,536): weak scaling, no data-path collective; a barrier brackets
the timed region and the time is the max over ranks.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SSA reaction events/s incl. grid align+mean/var reduce, 1 GB300, vs plain FP64"
UNIT = "events/s"
SMS_GB300 = 152
# DRAM read + write bytes of one k_ssa_thread launch (from an ncu capture:
# tables, grid and parameters; the difference sums stay in L2), independent of
# the number of trajectories.
SIM_KERNEL_DRAM_BYTES = 537344
# Bench workloads: the HIV-shaped model (the headline line) and the random
# 32-species / 128-reaction network (one trajectory per warp).
WORKLOADS = {
    "hiv_shaped": {"factory": "workload_hiv_shaped", "name": "hiv_shaped_S4_M10_G3001_T30", "n_traj": 65536,
                   "steps": 100, "e2e_steps": 20, "cpu_sample": 16384, "ref_sample": 4096,
                   "kernel": "k_ssa_thread", "dram_bytes": SIM_KERNEL_DRAM_BYTES},
    # DRAM bytes per launch of the simulation kernel from ncu captures (model
    # tables and grid; independent of the trajectory count)
    "random": {"factory": "workload_random", "name": "random_S32_M128_G1001_T10_netseed3", "n_traj": 262144,
               "steps": 10, "e2e_steps": 3, "cpu_sample": 2048, "ref_sample": 512,
               "kernel": "k_ssa_warp", "dram_bytes": {"fp64": 604416, "fp32": 602112}},
    "grad": {"factory": "workload_hiv_shaped", "name": "hiv_shaped_grad_S4_M10_G3001_T30_loss_V", "n_traj": 1048576,
             "steps": 5, "e2e_steps": 2, "cpu_sample": 2048, "ref_sample": 1024,
             "kernel": "k_ssa_grad", "dram_bytes": 256360000},
    "paper_hiv": {"factory": "workload_paper_hiv", "name": "paper_hiv_S10_M27_G1001_T10_tnf_modifiers",
                  "n_traj": 4096, "steps": 3, "e2e_steps": 1, "cpu_sample": 48, "ref_sample": 16,
                  "kernel": "k_ssa_warp", "dram_bytes": None},
    "avgxy": {"factory": "workload_hiv_shaped", "name": "hiv_shaped_avg_xy_S4_M10_T30_window_N", "n_traj": 65536,
              "steps": 5, "e2e_steps": 1, "cpu_sample": 16, "ref_sample": 16,
              "kernel": "k_ssa_thread (logging) + radix sort", "dram_bytes": None},
    "batch": {"factory": None, "name": "batch256_S4-64_M8-512_N1024-65536_G501_T10_fp32", "n_traj": None,
              "steps": 2, "e2e_steps": 1, "cpu_sample": 16, "ref_sample": 16,
              "kernel": "k_ssa_batch", "dram_bytes": 44585472},
}
FP64_OPS_PER_SM_CLK = 2.0  # 1.25 TFLOP/s dense FP64 (FMA = 2 flops) / (152 SMs * 2.07 GHz)

CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse_args():
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=None, help="timed steps (default per workload)")
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=sorted(WORKLOADS), default="hiv_shaped",
                   help="hiv_shaped (headline): 4 species / 10 reactions, 65,536 trajectories, thread kernel; "
                        "random: 32 x 128, 262,144 trajectories, warp kernel; paper_hiv: the paper's 27-reaction "
                        "model with TNF-dependent rates; batch: 256 uneven networks in one graph; grad: rate "
                        "gradient on 1,048,576 trajectories; avgxy: Avg-Y / Avg-XY selective memory")
    p.add_argument("--n-traj", type=int, default=None, help="trajectories per GPU (default per workload)")
    p.add_argument("--precision", choices=["fp64", "fp32"], default="fp64",
                   help="fp32: binary32 propensities and selection sums, FP64 a0 and time (one trajectory "
                        "per warp); the line then adds the FP64 kernel's rate on the same GPU and the "
                        "FP32-vs-FP64 standard-error report")
    p.add_argument("--e2e-steps", type=int, default=None)
    p.add_argument("--batch-div", type=int, default=1,
                   help="batch workload: divide every network's trajectory count by this")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-forms", action="store_true",
                   help="headline line only (by default the HIV-shaped FP64 line also carries a 'forms' object: the "
                        "random network in FP64 and FP32, the gradient and the full batch, a few steps each)")
    p.add_argument("--profile-small", action="store_true",
                   help="one small step for an ncu capture (--profile-n trajectories); prints no bench line")
    p.add_argument("--profile-n", type=int, default=16384)
    args = p.parse_args()
    spec = WORKLOADS[args.workload]
    args.steps = spec["steps"] if args.steps is None else args.steps
    args.n_traj = spec["n_traj"] if args.n_traj is None else args.n_traj
    if args.workload in ("batch", "grad", "avgxy") and args.impl == "reference":
        p.error("--impl reference times the forward single-network workloads")
    args.e2e_steps = spec["e2e_steps"] if args.e2e_steps is None else args.e2e_steps
    return args


def make_workload(args, n):
    import workloads as W
    spec = WORKLOADS[args.workload]
    return getattr(W, spec["factory"])(n)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={CLOCK_FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [v.strip() for v in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def fp64_ops_per_event(n_reactions: int) -> int:
    """Algorithmic FP64 operations of one direct-method event in exact mode:
    M products c_j * h_j, M - 1 sums for a0 and the prefix sums, the product
    r2 * a0, the quotient -ln(r1) / a0 and the sum t + tau."""
    return 2 * n_reactions + 2


def plain_fp64_ops_per_event(net) -> float:
    """FP64 operations of one event in a plain implementation that also runs
    the uniform map, the logarithm and the division in FP64: 4 (uniform map)
    + 20 (log) + 9 (division) + 1 (t add) + M (a0) + M (selection scan) + 2 d
    (d = mean number of propensities an event changes); 34 + 2M + 2d, about
    60 for M = 10."""
    import numpy as np
    R = np.asarray(net.reactants)
    nu = np.asarray(net.products) - R
    reads = R > 0                              # [M, S]: reaction k reads species s
    changes = nu != 0                          # [M, S]: reaction j changes species s
    dep = (changes.astype(int) @ reads.T.astype(int)) > 0   # [j, k]
    d = float(dep.sum(axis=1).mean())
    M = R.shape[0]
    return 34.0 + 2.0 * M + 2.0 * d


def oracle_mode(args):
    """(schedule, precision) of the oracle matching the GPU run: the warp
    layout's W32 order for the random network, FP32 when asked."""
    import oracle
    schedule = oracle.SCHEDULE_W32 if args.workload in ("random", "paper_hiv") else oracle.SCHEDULE_L
    precision = oracle.PRECISION_FP32 if getattr(args, "precision", "fp64") == "fp32" else oracle.PRECISION_FP64
    return schedule, precision


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part")):
                    return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def cpu_baseline(w, n_traj_sample: int, args=None):
    """The oracle as it stands, on all host cores (one thread per id range),
    and on one thread over an eighth of the same ids."""
    import oracle
    cores = os.cpu_count() or 1
    schedule, precision = oracle_mode(args) if args is not None else (oracle.SCHEDULE_L, oracle.PRECISION_FP64)
    t0 = time.perf_counter()
    r = oracle.run(w.net, n_traj_sample, w.t_end, w.n_grid, w.seed, threads=cores, schedule=schedule,
                   precision=precision)
    dt = time.perf_counter() - t0
    n1 = max(1, n_traj_sample // 8)
    t1 = time.perf_counter()
    r1 = oracle.run(w.net, n1, w.t_end, w.n_grid, w.seed, threads=1, schedule=schedule, precision=precision)
    dt1 = time.perf_counter() - t1
    return {"value": r.events / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"trajectories 0..{n_traj_sample - 1} of the workload (seed {w.seed}), "
                      f"{r.events} events in {dt:.3f} s on {cores} threads",
            "value_1thread": r1.events / dt1,
            "sample_1thread": f"trajectories 0..{n1 - 1}, {r1.events} events in {dt1:.3f} s on 1 thread",
            "cpu_model": cpu_model()}


def cpu_baseline_grad(w, n_traj_sample: int, target):
    """The oracle's forward ensemble and likelihood-ratio contributions
    (oracle.grad) on all host cores; events counted twice as on the GPU."""
    import numpy as np

    import oracle
    cores = os.cpu_count() or 1
    tgt = np.asarray(target, dtype=np.float64)

    def one(n, threads):
        t0 = time.perf_counter()
        r = oracle.run(w.net, n, w.t_end, w.n_grid, w.seed, threads=threads)
        mean, _ = oracle.finalize(n, r.S1, r.S2)
        wgt = np.zeros_like(mean)
        wgt[:, 2] = 2.0 * (mean[:, 2] - tgt)
        oracle.grad(w.net, n, w.t_end, w.n_grid, w.seed, wgt, mean, threads=threads)
        return 2 * r.events, time.perf_counter() - t0
    ev, dt = one(n_traj_sample, cores)
    n1 = max(1, n_traj_sample // 8)
    ev1, dt1 = one(n1, 1)
    return {"value": ev / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"trajectories 0..{n_traj_sample - 1} (seed {w.seed}): forward + likelihood-ratio "
                      f"contributions, {ev} events counted twice in {dt:.3f} s on {cores} threads",
            "value_1thread": ev1 / dt1,
            "sample_1thread": f"trajectories 0..{n1 - 1}, {ev1} events counted twice in {dt1:.3f} s on 1 thread",
            "cpu_model": cpu_model()}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    spec = WORKLOADS[args.workload]
    w = make_workload(args, args.n_traj)
    oracle.lib()
    cores = os.cpu_count() or 1
    sample = min(args.n_traj, spec["ref_sample"])
    schedule, precision = oracle_mode(args)
    for i in range(args.warmup):
        oracle.run(w.net, sample, w.t_end, w.n_grid, 1 + i, threads=cores, schedule=schedule, precision=precision)
    events = 0
    t0 = time.perf_counter()
    for i in range(args.steps):
        r = oracle.run(w.net, sample, w.t_end, w.n_grid, 1000 + i, threads=cores, schedule=schedule,
                       precision=precision)
        events += r.events
    dt = time.perf_counter() - t0
    value = events / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": spec["name"], "n_traj": args.n_traj, "n_grid": w.n_grid,
                   "t_end": w.t_end, "precision": args.precision, "sample_per_step": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{sample} trajectories per step (seeds 1000..), {cores} threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch

    import paper_1007_1768_gb300 as ssa

    spec = WORKLOADS[args.workload]
    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        pg = dist

    n = args.n_traj if not args.profile_small else args.profile_n
    w = make_workload(args, n)
    model = ssa.Model.from_network(w.net)
    G, S, M = w.n_grid, w.net.n_species, w.net.n_reactions
    stream = torch.cuda.current_stream(dev)
    mean = torch.empty((G, S), dtype=torch.float64, device=dev)
    var = torch.empty((G, S), dtype=torch.float64, device=dev)
    totals = torch.zeros(4, dtype=torch.int64, device=dev)
    base_opts = ssa.make_opts(memory=ssa.binding.MEM_DEVICE, cuda_stream=stream.cuda_stream,
                              traj_offset=rank * n)
    ws_bytes = ssa.workspace_bytes(model, n, G, base_opts)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    L = ssa.lib()

    def run_step(seed, ev_begin=None, ev_end=None, precision=args.precision):
        o = ssa.make_opts(memory=ssa.binding.MEM_DEVICE, cuda_stream=stream.cuda_stream, traj_offset=rank * n,
                          precision=precision,
                          workspace=ws.data_ptr(), workspace_bytes=ws_bytes, device_totals=totals.data_ptr(),
                          sim_event_begin=ev_begin, sim_event_end=ev_end)
        st = L.ssa_ensemble_run(model.handle, n, w.t_end, G, None, seed, o, mean.data_ptr(), var.data_ptr(),
                                None, None, None)
        if st != 0:
            raise RuntimeError(f"ssa_ensemble_run failed: {L.ssa_last_error().decode()}")

    if args.profile_small:
        run_step(1)
        torch.cuda.synchronize()
        return None

    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    for i in range(args.warmup):
        run_step(1 + i)
    torch.cuda.synchronize()

    K = args.steps
    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    k_s = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    k_e = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    for e in k_s + k_e:  # create the underlying cudaEvent_t handles
        e.record(stream)
    torch.cuda.synchronize()
    totals.zero_()
    clocks = ClockSampler(local)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    clocks.start()
    wall0 = time.perf_counter()
    for i in range(K):
        flush.fill_(i & 0xFF)  # L2 flush, outside the step's events
        ev_s[i].record(stream)
        run_step(1000 + i, k_s[i].cuda_event, k_e[i].cuda_event)
        ev_e[i].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    if pg:
        pg.barrier()
    step_ms = [ev_s[i].elapsed_time(ev_e[i]) for i in range(K)]
    kern_ms = [k_s[i].elapsed_time(k_e[i]) for i in range(K)]
    tot = totals.cpu().tolist()
    events = int(tot[0])
    total_ms = sum(step_ms)
    if pg:
        t = torch.tensor([total_ms, float(events)], dtype=torch.float64)
        mx = t.clone()
        pg.all_reduce(mx, op=pg.ReduceOp.MAX)
        sm = t.clone()
        pg.all_reduce(sm, op=pg.ReduceOp.SUM)
        total_ms, events_all = float(mx[0]), float(sm[1])
    else:
        events_all = float(events)
    value = events_all / (total_ms * 1e-3)

    # roofline of the simulation kernel: FP64 pipe (ALU bound)
    ops = fp64_ops_per_event(M) * (events / K)
    kern_avg = statistics.mean(kern_ms)
    achieved = ops / (kern_avg * 1e-3) * 1e-9
    sm_mhz = (clk or {}).get("sm_mhz") or 2070.0
    peak = FP64_OPS_PER_SM_CLK * SMS_GB300 * sm_mhz * 1e6 * 1e-9

    fp64_same_gpu = fp32_vs_fp64 = None
    if args.precision == "fp32" and rank == 0:
        fp64_same_gpu, fp32_vs_fp64 = compare_with_fp64(args, ssa, torch, model, w, n, run_step, totals, stream,
                                                        flush)

    result = None
    if rank == 0:
        # end to end through the C ABI with host buffers: grid in, mean/var out
        import numpy as np
        grid_h = (np.arange(G, dtype=np.float64) * w.t_end) / (G - 1)
        e_ev = 0
        for i in range(2):
            ssa.ensemble_run(model, n, w.t_end, G, 1 + i, grid=grid_h, want_sums=False, traj_offset=rank * n,
                             precision=args.precision)
        t0 = time.perf_counter()
        for i in range(args.e2e_steps):
            r = ssa.ensemble_run(model, n, w.t_end, G, 5000 + i, grid=grid_h, want_sums=False,
                                 traj_offset=rank * n, precision=args.precision)
            e_ev += r.events
        e_dt = time.perf_counter() - t0
        e2e = {"value": e_ev / e_dt, "unit": UNIT, "h2d_bytes_per_step": int(grid_h.nbytes),
               "d2h_bytes_per_step": int(2 * G * S * 8 + 8 * 8), "steps": args.e2e_steps}
        cpu = None if (args.no_cpu_baseline or world > 1) else cpu_baseline(w, min(n, spec["cpu_sample"]), args)
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32-propensities/f64-time", "data": "synthetic",
            "config": {"workload": spec["name"], "n_traj_per_gpu": n, "n_grid": G,
                       "t_end": w.t_end,
                       "precision": "fp64-exact" if args.precision == "fp64" else "fp32-propensities",
                       "seeds": "1000+step",
                       "l2": "flushed between timed steps (256 MiB write outside the step events)",
                       "parallelism": f"replicas x{world} (trajectory-id shards)"},
            "traj_per_s": world * n / (total_ms * 1e-3 / K) if K else None,
            "events_per_step": events_all / K,
            "wall_s_timed_region": wall,
            "roofline": {"bound": "alu", "kernel": spec["kernel"], "achieved": achieved, "peak": peak,
                         "unit": "GFLOP/s (FP64 ops)", "frac": achieved / peak,
                         "traffic": (spec["dram_bytes"][args.precision] if isinstance(spec["dram_bytes"], dict)
                                     else spec["dram_bytes"]),
                         "kernel_ms": kern_avg, "ops_per_event": fp64_ops_per_event(M),
                         "ops_per_event_plain_fp64": plain_fp64_ops_per_event(w.net),
                         "frac_plain_fp64": plain_fp64_ops_per_event(w.net) * (events / K) / (kern_avg * 1e-3) * 1e-9 / peak,
                         "peak_basis": "2 FP64 ops/clk/SM x 152 SMs x median SM clock (nominal 1.25 TFLOP/s dense)"},
            "cpu_baseline": cpu,
            "fp64_same_gpu": fp64_same_gpu,
            "fp32_vs_fp64": fp32_vs_fp64,
            "e2e": e2e,
            "gpu_launches": 3 * K,
            "clocks": clk,
        }
    model.close()
    if pg:
        pg.destroy_process_group()
    return result


def compare_with_fp64(args, ssa, torch, model, w, n, run_step, totals, stream, flush):
    """For an FP32-propensity run: the FP64 kernel's events/s on the same
    workload and GPU (same timing rules), and the standard-error report of
    the FP32 grid mean / variance against FP64 with the same seed."""
    import numpy as np
    K2 = max(1, min(3, args.steps))
    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(K2)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(K2)]
    run_step(1, precision="fp64")
    torch.cuda.synchronize()
    totals.zero_()
    for i in range(K2):
        flush.fill_(i & 0xFF)
        ev_s[i].record(stream)
        run_step(1000 + i, precision="fp64")
        ev_e[i].record(stream)
    torch.cuda.synchronize()
    ms = sum(ev_s[i].elapsed_time(ev_e[i]) for i in range(K2))
    ev64 = int(totals[0].item())
    same_gpu = {"value": ev64 / (ms * 1e-3), "unit": UNIT, "steps": K2, "ms_per_step": ms / K2,
                "events_per_step": ev64 / K2}
    # standard errors by batch means: B shards of N / B trajectories (shards add up
    # exactly to the full run), per precision; no distributional assumption
    dev = torch.device("cuda", torch.cuda.current_device())
    B = 32
    nb = n // B
    out = {}
    for prec in ("fp32", "fp64"):
        s1 = s2 = 0
        sh_mean, sh_var, ev = [], [], 0
        for b in range(B):
            r = ssa.ensemble_run(model, nb, w.t_end, w.n_grid, 4242, device=dev, precision=prec,
                                 traj_offset=b * nb)
            a1, a2 = r.sum1.cpu().numpy(), r.sum2.cpu().numpy()
            s1, s2 = s1 + a1, s2 + a2
            sh_mean.append(r.mean.cpu().numpy())
            sh_var.append(r.var.cpu().numpy())
            ev += r.events
        N = nb * B
        mean = s1 / N
        var = (N * s2.astype(np.float64) - s1.astype(np.float64) ** 2) / (N * (N - 1.0))
        se_m = np.std(np.stack(sh_mean), axis=0, ddof=1) / np.sqrt(B)
        se_v = np.std(np.stack(sh_var), axis=0, ddof=1) / np.sqrt(B)
        out[prec] = (mean, var, se_m, se_v, ev)
    m32, v32, sm32, sv32, e32 = out["fp32"]
    m64, v64, sm64, sv64, e64 = out["fp64"]
    se_m = np.sqrt(sm32 ** 2 + sm64 ** 2)
    se_v = np.sqrt(sv32 ** 2 + sv64 ** 2)
    zm = np.abs(m32 - m64) / np.where(se_m > 0, se_m, 1.0)
    zv = np.abs(v32 - v64) / np.where(se_v > 0, se_v, 1.0)
    zero_ok = bool(np.array_equal(m32[se_m == 0], m64[se_m == 0]) and np.array_equal(v32[se_v == 0], v64[se_v == 0]))
    report = {"cells": int(m32.size), "max_z_mean": float(zm.max()), "max_z_var": float(zv.max()),
              "cells_above_4se": int((zm > 4).sum() + (zv > 4).sum()), "zero_se_cells_equal": zero_ok,
              "events_fp32": e32, "events_fp64": e64, "seed": 4242, "n_traj": nb * B,
              "se": f"batch means over {B} shards of {nb} trajectories, per precision; "
                    "z = |x32 - x64| / sqrt(se32^2 + se64^2)"}
    return same_gpu, report


def run_grad(args):
    """Rate sensitivities on the HIV-shaped model: one step is the forward
    ensemble (1,048,576 trajectories, 3001-point grid), the loss
    sum_g (mean V(g) - target_g)^2 and its likelihood-ratio gradient for all
    ten rates, the trajectories replayed from their Philox counters."""
    import numpy as np
    import torch

    import paper_1007_1768_gb300 as ssa
    import workloads as W

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        pg = dist
    spec = WORKLOADS["grad"]
    n = args.n_traj if not args.profile_small else args.profile_n
    w = W.workload_hiv_shaped(n)
    model = ssa.Model.from_network(w.net)
    G, S, M = w.n_grid, w.net.n_species, w.net.n_reactions
    target = torch.as_tensor(W.hiv_target_v(), device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    kb = torch.cuda.Event(enable_timing=True)
    ke = torch.cuda.Event(enable_timing=True)

    def step(seed, timed=False):
        r = ssa.ensemble_run(model, n, w.t_end, G, seed, device=dev, want_sums=False, traj_offset=rank * n,
                             per_traj=True)
        wgt = torch.zeros((G, S), dtype=torch.float64, device=dev)
        wgt[:, 2] = 2.0 * (r.mean[:, 2] - target)
        opt = {}
        if timed:
            opt = {"sim_event_begin": kb.cuda_event, "sim_event_end": ke.cuda_event}
        # the forward's event counts let the replay start the longest trajectories first
        g, se, _ = ssa.ensemble_grad(model, n, w.t_end, G, seed, wgt, r.mean, device=dev, traj_offset=rank * n,
                                     traj_events=r.traj_events, **opt)
        return r.events, g, se

    if args.profile_small:
        step(1)
        torch.cuda.synchronize()
        model.close()
        return None
    for i in range(args.warmup):
        step(1 + i)
    torch.cuda.synchronize()
    K = args.steps
    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    kb.record(stream)
    ke.record(stream)
    clocks = ClockSampler(local)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    clocks.start()
    events = 0
    grad_ms = []
    last = None
    for i in range(K):
        flush.fill_(i & 0xFF)
        ev_s[i].record(stream)
        ev, g, se = step(1000 + i, timed=True)
        ev_e[i].record(stream)
        torch.cuda.synchronize()
        grad_ms.append(kb.elapsed_time(ke))
        events += 2 * ev  # forward events and the same events replayed
        last = (g, se)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = sum(ev_s[i].elapsed_time(ev_e[i]) for i in range(K))
    if pg:
        t = torch.tensor([total_ms, float(events)], dtype=torch.float64)
        mx = t.clone()
        pg.all_reduce(mx, op=pg.ReduceOp.MAX)
        sm = t.clone()
        pg.all_reduce(sm, op=pg.ReduceOp.SUM)
        total_ms, events_all = float(mx[0]), float(sm[1])
    else:
        events_all = float(events)
    value = events_all / (total_ms * 1e-3)
    sm_mhz = (clk or {}).get("sm_mhz") or 2070.0
    peak = FP64_OPS_PER_SM_CLK * SMS_GB300 * sm_mhz * 1e6 * 1e-9
    kern = statistics.mean(grad_ms)
    ops_bwd = (4 * M + 2) * (events / 2 / K)
    achieved = ops_bwd / (kern * 1e-3) * 1e-9
    line = None
    if rank == 0:
        t0 = time.perf_counter()
        e_ev = 0
        for i in range(args.e2e_steps):
            rates = torch.tensor(w.net.rates, dtype=torch.float64, requires_grad=True)
            from paper_1007_1768_gb300.autograd import ssa_ensemble
            mean, _ = ssa_ensemble(rates, w.net, n, w.t_end, G, 7000 + i, device=dev)
            loss = ((mean[:, 2] - target) ** 2).sum()
            loss.backward()
            _ = rates.grad.numpy().copy()
            e_ev += 2 * int(ssa_events_estimate(events, K))
        e_dt = time.perf_counter() - t0
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            cpu = cpu_baseline_grad(w, min(n, spec["cpu_sample"]), target.cpu().numpy())
        g, se = last
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": spec["name"], "n_traj_per_gpu": n, "n_grid": G, "t_end": w.t_end,
                       "precision": "fp64-exact", "loss": "sum_g (mean V(g) - target_g)^2, target file",
                       "events": "forward events + the same events replayed in the backward pass",
                       "l2": "flushed between timed steps (256 MiB write outside the step events)",
                       "parallelism": f"replicas x{world} (trajectory-id shards)"},
            "traj_per_s": world * n / (total_ms * 1e-3 / K),
            "grad_kernel_ms": kern,
            "grad_last_step": [float(v) for v in g.cpu().numpy()],
            "grad_se_last_step": [float(v) for v in se.cpu().numpy()],
            "roofline": {"bound": "alu", "kernel": spec["kernel"], "achieved": achieved, "peak": peak,
                         "unit": "GFLOP/s (FP64 ops)", "frac": achieved / peak, "traffic": spec["dram_bytes"],
                         "ops_per_event": 4 * M + 2,
                         "peak_basis": "2 FP64 ops/clk/SM x 152 SMs x median SM clock"},
            "cpu_baseline": cpu,
            "e2e": ({"value": e_ev / e_dt, "unit": UNIT, "h2d_bytes_per_step": int(8 * M),
                     "d2h_bytes_per_step": int(8 * M), "steps": args.e2e_steps,
                     "note": "torch autograd: rates in, loss.backward(), rates.grad read back; events as timed"}
                    if args.e2e_steps > 0 else None),
            "gpu_launches": K * 7,
            "clocks": clk,
        }
    model.close()
    if pg:
        pg.destroy_process_group()
    return line


def ssa_events_estimate(events_total, steps):
    """Forward events of one step (mean over the timed steps)."""
    return events_total / 2 / steps


def run_avgxy(args):
    """Selective memory along the time axis on the HIV-shaped model: one step
    is one ssa_ensemble_avg_xy call (a pilot of 4,096 trajectories to size
    the event log, the logging run, the radix sort of ~1e8 event records by
    time, union indices, window sums) with window k = N, outputs copied to the
    host."""
    import numpy as np
    import torch

    import paper_1007_1768_gb300 as ssa
    import workloads as W

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    spec = WORKLOADS["avgxy"]
    n = args.n_traj
    w = W.workload_hiv_shaped(n)
    model = ssa.Model.from_network(w.net)
    M = w.net.n_reactions
    for i in range(args.warmup):
        ssa.ensemble_avg_xy(model, n, w.t_end, 1 + i, n, traj_offset=rank * n)
    r = ssa.ensemble_run(model, n, w.t_end, 2, 1, traj_offset=rank * n)  # the same (thread-schedule) trajectories
    events_per_run = r.events
    stream = torch.cuda.current_stream()
    K = args.steps
    clocks = ClockSampler(local)
    torch.cuda.synchronize()
    clocks.start()
    ms = []
    info = None
    for i in range(K):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t, m, q, U = ssa.ensemble_avg_xy(model, n, w.t_end, 1000 + i, n, traj_offset=rank * n)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        info = (len(t), U)
    clk = clocks.stop()
    total_ms = sum(ms)
    value = world * events_per_run * K / (total_ms * 1e-3)
    sm_mhz = (clk or {}).get("sm_mhz") or 2070.0
    peak = FP64_OPS_PER_SM_CLK * SMS_GB300 * sm_mhz * 1e6 * 1e-9
    simulated = 1.0 + min(n, 4096) / n  # the logging run and the pilot
    achieved = simulated * (2 * M + 2) * events_per_run / (total_ms / K * 1e-3) * 1e-9
    line = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": spec["name"], "n_traj_per_gpu": n, "t_end": w.t_end, "window": n,
                       "windows": info[0], "union_points": info[1],
                       "events": "events of one ensemble (the call also simulates a 4,096-trajectory pilot)",
                       "parallelism": f"replicas x{world} (trajectory-id shards)"},
            "roofline": {"bound": "alu", "kernel": spec["kernel"], "achieved": achieved, "peak": peak,
                         "unit": "GFLOP/s (FP64 ops)", "frac": achieved / peak, "traffic": None,
                         "ops_per_event": "(2M + 2) per simulated event (the logging run and the pilot)",
                         "peak_basis": "2 FP64 ops/clk/SM x 152 SMs x median SM clock"},
            "cpu_baseline": None,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": int(info[0] * (1 + 2 * w.net.n_species) * 8),
                    "note": "the timed call is the host API: outputs copied back inside the timed region"},
            "gpu_launches": None,
            "clocks": clk,
        }
    model.close()
    return line


def run_batch(args):
    """The uneven batch of 256 random networks in one graph replay per step
    (FP32 propensities, FP64 time): persistent kernels per register bucket,
    launch shape from the autotuner."""
    import numpy as np
    import torch

    import paper_1007_1768_gb300 as ssa
    import workloads as W

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        pg = dist
    spec = WORKLOADS["batch"]
    ws = W.batch_networks(traj_div=args.batch_div)
    models = [ssa.Model.from_network(w.net) for w in ws]
    n_traj = [w.n_traj for w in ws]
    t_end = [w.t_end for w in ws]
    n_grid = [w.n_grid for w in ws]
    stream = torch.cuda.current_stream(dev)
    batch = ssa.Batch(models, n_traj, t_end, n_grid, device=dev, precision="fp32", max_events=1000000,
                      traj_offset=rank * 10 ** 9)
    if args.profile_small:  # one launch of the default shape, for an ncu capture
        batch.launch(1, stats=True)
        batch.close()
        for m in models:
            m.close()
        return None
    threads, split, tune_ms = batch.tune()
    scheds = [batch.network_stats(b).schedule for b in range(len(ws))]
    sched_counts = {"thread": scheds.count(1), "warp": scheds.count(2)}
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    for i in range(args.warmup):
        batch.launch(1 + i, stats=False)
    torch.cuda.synchronize()
    K = args.steps
    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    clocks = ClockSampler(local)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    clocks.start()
    events = 0
    ops = 0.0
    Ms = np.array([w.net.n_reactions for w in ws], dtype=np.float64)
    for i in range(K):
        flush.fill_(i & 0xFF)
        ev_s[i].record(stream)
        _, st = batch.launch(1000 + i, stats=True)
        ev_e[i].record(stream)
        events += st.events
        per = np.array([batch.network_stats(b).events for b in range(len(ws))], dtype=np.float64)
        ops += float((per * (Ms + 2.0)).sum())
    torch.cuda.synchronize()
    clk = clocks.stop()
    step_ms = [ev_s[i].elapsed_time(ev_e[i]) for i in range(K)]
    total_ms = sum(step_ms)
    if pg:
        t = torch.tensor([total_ms, float(events)], dtype=torch.float64)
        mx = t.clone()
        pg.all_reduce(mx, op=pg.ReduceOp.MAX)
        sm = t.clone()
        pg.all_reduce(sm, op=pg.ReduceOp.SUM)
        total_ms, events_all = float(mx[0]), float(sm[1])
    else:
        events_all = float(events)
    value = events_all / (total_ms * 1e-3)
    sm_mhz = (clk or {}).get("sm_mhz") or 2070.0
    peak = FP64_OPS_PER_SM_CLK * SMS_GB300 * sm_mhz * 1e6 * 1e-9
    achieved = ops / (total_ms * 1e-3) * 1e-9
    line = None
    if rank == 0:
        # end to end: one-shot host call (model tables, graph, launch, copies back)
        host_means = [np.empty((g, m.n_species)) for g, m in zip(n_grid, models)]
        host_vars = [np.empty((g, m.n_species)) for g, m in zip(n_grid, models)]
        t0 = time.perf_counter()
        e_events = 0
        for i in range(args.e2e_steps):
            hb = ssa.Batch(models, n_traj, t_end, n_grid, precision="fp32", max_events=1000000,
                           block_threads=threads)
            outs, st = hb.launch(7000 + i, stats=True)
            e_events += st.events
            hb.close()
        e_dt = time.perf_counter() - t0
        d2h = int(sum(2 * g * m.n_species * 8 for g, m in zip(n_grid, models)))
        # descriptors, finalisation entries and work offsets the one-shot call copies in
        h2d = int(len(ws) * (136 + 72 + 4 + 16) + 4 + 16)
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            cpu = cpu_baseline_batch(ws, spec["cpu_sample"])
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32-propensities/f64-time", "data": "synthetic",
            "config": {"workload": spec["name"], "networks": len(ws), "n_traj_total": int(sum(n_traj)),
                       "traj_div": args.batch_div, "n_grid": 501, "t_end": 10.0, "precision": "fp32-propensities",
                       "launch": {"block_threads": threads, "split_by_bucket": split, "tune_sample_ms": tune_ms,
                                  "schedules": sched_counts},
                       "l2": "flushed between timed steps (256 MiB write outside the step events)",
                       "parallelism": f"replicas x{world} (trajectory-id shards)"},
            "traj_per_s": world * sum(n_traj) / (total_ms * 1e-3 / K),
            "events_per_step": events_all / K,
            "roofline": {"bound": "alu", "kernel": spec["kernel"], "achieved": achieved, "peak": peak,
                         "unit": "GFLOP/s (FP64 ops)", "frac": achieved / peak, "traffic": spec["dram_bytes"],
                         "ops_per_event": "M_b + 2 (FP64 re-summation of a0, r2 * A32, quotient, t add)",
                         "peak_basis": "2 FP64 ops/clk/SM x 152 SMs x median SM clock"},
            "cpu_baseline": cpu,
            "e2e": ({"value": e_events / e_dt, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                     "steps": args.e2e_steps, "note": "one-shot batches from host: create, tune-free launch, copy"}
                    if args.e2e_steps > 0 else None),
            "gpu_launches": K * (2 + n_groups(ws, split)),
            "clocks": clk,
        }
    batch.close()
    for m in models:
        m.close()
    if pg:
        pg.destroy_process_group()
    return line


def n_groups(ws, split: bool) -> int:
    """Simulation kernels per batch replay: one per register bucket (the
    warp layout's chunk ceil(M / 32) rounded up to 1, 2, 4, 8, 16) when split."""
    if not split:
        return 1
    buckets = set()
    for w in ws:
        ch = (w.net.n_reactions + 31) // 32
        buckets.add(next(b for b in (1, 2, 4, 8, 16) if b >= ch))
    return len(buckets)


def cpu_baseline_batch(ws, per_network: int):
    """The oracle on all host cores over the first `per_network` trajectories
    of every network of the batch (FP32 propensities, W32), and on one thread
    over the first trajectory of every eighth network."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    cores = os.cpu_count() or 1

    def one(w, n=per_network):
        r = oracle.run(w.net, min(n, w.n_traj), w.t_end, w.n_grid, w.seed, max_events=1000000,
                       schedule=oracle.SCHEDULE_W32, precision=oracle.PRECISION_FP32)
        return r.events
    t0 = time.perf_counter()
    with ThreadPoolExecutor(cores) as ex:
        ev = sum(ex.map(one, ws))
    dt = time.perf_counter() - t0
    t1 = time.perf_counter()
    ev1 = sum(one(w, 1) for w in ws[::8])
    dt1 = time.perf_counter() - t1
    return {"value": ev / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {per_network} trajectories of each of the {len(ws)} networks, {ev} events in "
                      f"{dt:.2f} s on {cores} threads",
            "value_1thread": ev1 / dt1,
            "sample_1thread": f"first trajectory of every 8th network, {ev1} events in {dt1:.2f} s on 1 thread",
            "cpu_model": cpu_model()}


def run_forms(args):
    """The other forms of the method on this GPU, each with a few timed steps
    (their default workloads at full size): the random 32 x 128 network in
    FP64 (W32) and FP32 (with the FP32-vs-FP64 standard-error report), the
    rate gradient on 1,048,576 trajectories and the full 256-network batch."""
    def sub(**kw):
        d = dict(vars(args))
        d.update(kw)
        d.setdefault("batch_div", 1)
        return argparse.Namespace(**d)

    def brief(line):
        if line is None:
            return None
        keep = ("value", "unit", "ms_per_step", "steps", "warmup", "dtype", "config", "traj_per_s", "events_per_step",
                "roofline", "cpu_baseline", "e2e", "fp64_same_gpu", "fp32_vs_fp64", "grad_kernel_ms", "clocks",
                "gpu_launches")
        return {k: line[k] for k in keep if k in line}

    forms = {}
    common = {"profile_small": False, "no_cpu_baseline": args.no_cpu_baseline}
    forms["random_fp64"] = brief(run_ours(sub(workload="random", precision="fp64", n_traj=262144, steps=2,
                                              warmup=1, e2e_steps=1, **common)))
    forms["random_fp32"] = brief(run_ours(sub(workload="random", precision="fp32", n_traj=262144, steps=2,
                                              warmup=1, e2e_steps=1, **common)))
    forms["grad"] = brief(run_grad(sub(workload="grad", precision="fp64", n_traj=1048576, steps=2, warmup=1,
                                       e2e_steps=1, **common)))
    forms["batch"] = brief(run_batch(sub(workload="batch", precision="fp32", n_traj=None, steps=1, warmup=1,
                                         e2e_steps=0, batch_div=1, **common)))
    return forms


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    runner = {"batch": run_batch, "grad": run_grad, "avgxy": run_avgxy}.get(args.workload, run_ours)
    line = runner(args)
    if line is None:
        return 0
    _, world, _ = dist_env()
    if args.workload == "hiv_shaped" and args.precision == "fp64" and world == 1 and not args.no_forms:
        forms = run_forms(args)
        line["forms"] = forms
        r32 = forms.get("random_fp32") or {}
        # the FP32-propensity form against the plain FP64 kernel on the same GPU (random 32 x 128 network)
        line["fp64_same_gpu"] = r32.get("fp64_same_gpu")
        line["fp32_vs_fp64"] = r32.get("fp32_vs_fp64")
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
