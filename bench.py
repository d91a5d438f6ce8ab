"""Benchmark of the multicanonical Blume-Capel hot path on one GB300.

Workload (N=1): the large first-order configuration, L=48 (110592 sites),
T=0.9, 4096 walkers, seed 3.  One step is one pass of the whole hot path in
the production schedule of that workload (40 iterations x 1000 sweeps, then
10^4 measurement sweeps, i.e. 250 measurement sweeps per iteration):
  1000 typewriter Metropolis sweeps of every walker with the per-sweep
  histogram, the merge, the FP64 weight update and the acceptance-table
  rebuild (one CUDA-graph iteration), then 250 recorded measurement sweeps and
  the FP32 reweighting of the step's series to a 4096-point Delta grid.
Metric: spin-update attempts per second (accepted or not) = walkers x L^3 x
sweeps / time.  "batched" is the graph form, "plain" the same work with one
launch per call and host-driven merges.  The reweighting sub-benchmark times
the FP32 and FP64 paths on a 4096-walker x 10^4-sample series of an L=32,
T=1.4182 run (Delta-grid points per second).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle on the host cores instead (bounded
walker samples of the same workload).  Under torchrun (N > 1) the ranks run
one simulation of N x 4096 walkers at L=48, T=0.9, each rank holding 4096 of
them (weak scaling): after every iteration the ranks' integer histograms are
summed with an NCCL all-reduce on device buffers and every rank runs the same
FP64 weight update (the parallel scheme of Sec. II over GPUs).  Timed with a
barrier and the maximum over ranks.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1502_07214_gb300 import workloads as wl  # noqa: E402

METRIC = "spin-update attempts/s at L=48 T=0.9 (batched)"
UNIT = "attempts/s"


def env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


# DRAM bytes (read + write) per sweep of the benchmark workload, from one ncu
# capture of each kernel in this configuration (a launch of 2 sweeps after
# three 1000-sweep weight iterations): split kernel 926.8 MB read + 848.5 MB
# written, row-scan kernel 1943.5 MB read + 881.9 MB written.  Valid only for
# the kernel source the counters were taken on; empty (traffic reported as
# null) while no capture of the current source exists.
TRAFFIC_PER_SWEEP = {3: (926.811392e6 + 848.504064e6) / 2,
                     4: (1943.472e6 + 881.874176e6) / 2}


# L2 bytes (32-byte sectors through the L2, lts__t_sectors.sum) per sweep from
# the same captures: split kernel 216.3 M sectors, row-scan kernel 338.3 M
# sectors per 2-sweep launch.  Same validity rule as the DRAM traffic.
L2_PER_SWEEP = {3: 216.3e6 * 32 / 2, 4: 338.261052e6 * 32 / 2}

PROBE_KINDS = {0: "IMAD a=a*a+b", 1: "IADD3 a=a+b+c", 2: "LOP3 a=(a&b)^c",
               3: "half IMAD, half IADD3"}


def device_probes(torch, muca, iters=4096, l2_reps=64):
    """Ceilings of this device that the driver's peak file does not hold,
    measured with the library's probe kernels (best of five launches): the
    32-bit integer instruction rate of each probe kind and the L2 read
    bandwidth of a 32 MiB buffer; the SM count from the device properties."""
    props = torch.cuda.get_device_properties(0)
    out = {"sm_count": props.multi_processor_count, "int_ops_per_s": {}}
    for k, name in PROBE_KINDS.items():
        ops, ms = muca.probe_int(k, iters=iters)
        out["int_ops_per_s"][name] = ops
    bw, ms = muca.probe_l2_read(32 << 20, reps=l2_reps)
    out["l2_read_gbs"] = bw / 1e9
    out["l2_buffer_bytes"] = 32 << 20
    return out


def traffic_per_launch(res, sweeps):
    """DRAM traffic of one launch of `sweeps` sweeps, scaled from the ncu
    capture (traffic grows in proportion to the sweeps), or None."""
    b = TRAFFIC_PER_SWEEP.get(res)
    return None if b is None else b * sweeps


def shard_group(L, T, walkers_per_rank, world):
    """With N GPUs the ranks run one simulation of N x walkers_per_rank
    walkers, each rank holding its shard (weak scaling); returns the group
    and the shard option of the context."""
    return {"L": L, "T": T, "n_walkers": walkers_per_rank * world}


def job_rate(ms_local, units_per_rank, world, dist=None, device="cpu"):
    """Whole-job rate over N ranks: every rank's units over the slowest rank's
    time (the maximum of the ranks' timed regions).  Returns (rate, max_ms)."""
    import torch

    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    if dist is not None and world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    return units_per_rank * world / (ms / 1e3), ms


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            with open(p) as f:
                d = json.load(f)
            return d, "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle

    s = wl.LARGE
    L, T = s["L"], s["T"]
    V = L ** 3
    cores = os.cpu_count() or 1
    # calibrate on 60 sweeps of one walker per core, after 20 warm-up sweeps
    oracle.muca_run(L, T, cores, s["seed"], 1, 20, n_threads=cores, want_spins=False)
    t0 = time.perf_counter()
    oracle.muca_run(L, T, cores, s["seed"], 1, 60, n_threads=cores, want_spins=False)
    rate = 60 / max(time.perf_counter() - t0, 1e-3)
    sweeps = max(20, min(20000, int(8.0 * rate)))  # about 8 s per step
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.muca_run(L, T, cores, s["seed"], 1, sweeps, n_threads=cores, want_spins=False)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    attempts = cores * V * sweeps
    tot = sum(times)
    value = attempts * len(times) / tot
    sample = (f"{cores} walkers (one per core) x {sweeps} sweeps of L={L}, T={T} per step, "
              f"one weight update per step")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": "L=48 T=0.9 multicanonical sweeps (oracle sample)",
                   "L": L, "T": T, "walkers": cores, "sweeps_per_step": sweeps},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def cpu_baseline_sample():
    """The oracle as it stands on the host cores, on a bounded walker sample."""
    import oracle

    s = wl.LARGE
    L, T = s["L"], s["T"]
    V = L ** 3
    cores = os.cpu_count() or 1
    # calibrate on 60 sweeps after 20 (the first sweeps run slower), then time a
    # sample of about 15 s
    oracle.muca_run(L, T, cores, s["seed"], 1, 20, n_threads=cores, want_spins=False)
    t0 = time.perf_counter()
    oracle.muca_run(L, T, cores, s["seed"], 1, 60, n_threads=cores, want_spins=False)
    rate = 60 / max(time.perf_counter() - t0, 1e-3)
    sweeps = max(20, min(20000, int(15.0 * rate)))
    t0 = time.perf_counter()
    oracle.muca_run(L, T, cores, s["seed"], 1, sweeps, n_threads=cores, want_spins=False)
    dt = time.perf_counter() - t0
    return {"value": cores * V * sweeps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} walkers x {sweeps} sweeps of L={L} T={T} (+ one weight update), "
                      f"{dt:.1f} s"}


# ---------------------------------------------------------------- our arm
def run_ours(args, rank, world, local_rank):
    import torch

    from paper_1502_07214_gb300 import muca

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    s = wl.LARGE
    L, T, W = s["L"], s["T"], s["n_walkers"]
    V = L ** 3
    sweeps = s["sweeps"]
    meas = s["n_meas"] // s["n_iter"]
    grid = wl.delta_grid(2.964)  # the first-order transition field at T=0.9 (Sec. III)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    from paper_1502_07214_gb300 import shard

    # one simulation over all ranks: each holds 4096 walkers of the group and
    # the histograms are summed over the ranks (NCCL, device buffers) after
    # every iteration; one rank runs the same workload unsharded
    fixed = {}
    if args.sweep_config:
        r_, w_, p_ = (int(x) for x in args.sweep_config.split(","))
        fixed = dict(residency=r_, walkers_per_block=w_, lanes_per_walker=p_)
    ctx = muca.Context([shard_group(L, T, W, world)], seed=s["seed"],
                       shard=(rank, world) if world > 1 else (0, 0), **fixed)
    ctx.reserve_timeseries(meas)
    res, wpb, lanes = ctx.get_config(0)
    launches_per_sweep_call = 1
    # the FP32 reweighting of a step's series: bucket count, bucket scan,
    # record scatter, bucket sums, per-bin statistics and the grid kernel
    reweight_launches = 6

    def iteration():
        if world > 1:
            # the all-reduce sits between the sweeps and the weight update,
            # so the sharded iteration is not one graph
            ctx.sweep_iter(sweeps)
            shard.merge_update(ctx, dist.all_reduce, device=True)
        else:
            ctx.run_graph(1, sweeps)
    attempts_step = W * V * (sweeps + meas)

    def step_batched():
        iteration()
        ctx.reserve_timeseries(meas)  # rewind
        ctx.sweep_iter(meas, record=True)
        return muca.reweight_context(ctx, 0, grid, 32, stream=stream)

    for _ in range(args.warmup):
        step_batched()
    # the timed, plain and end-to-end legs each start from this state (same
    # weights, spins and sweep counter), so they time the same iterations
    ck_fd, ck_path = tempfile.mkstemp(prefix="muca_bench_", suffix=".ck")
    os.close(ck_fd)
    ctx.checkpoint(ck_path)
    clocks = ClockSampler(local_rank)
    clocks.start()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_batched()
    e1.record(stream)
    barrier()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    value, ms = job_rate(ms, attempts_step * args.steps, world, dist, device="cuda")

    # plain form: the same step with one launch per call and host-driven merges;
    # CUDA events on the launching stream around every sweep launch give the
    # sweep kernel's average duration for the roofline
    plain_steps = max(1, min(args.steps, 2))
    ev = []
    ctx.restore(ck_path)
    barrier()
    p0 = time.perf_counter()
    for _ in range(plain_steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.sweep_iter(sweeps)
        b.record(stream)
        ev.append((a, b, sweeps))
        if world > 1:
            shard.merge_update(ctx, dist.all_reduce, device=True)
        else:
            ctx.merge_update()
        ctx.reserve_timeseries(meas)
        ctx.sweep_iter(meas, record=True)
        muca.reweight_context(ctx, 0, grid, 32, stream=stream)
    barrier()
    plain_s = time.perf_counter() - p0
    plain_value = attempts_step * plain_steps * world / plain_s
    kern_ms = [a.elapsed_time(b) for a, b, _ in ev]
    kern_avg_ms = sum(kern_ms) / len(kern_ms)
    attempts_launch = W * V * sweeps

    # end to end through the public API with host buffers: each step also reads
    # back the recorded series and the weights to pinned host memory
    ts_host = torch.empty((meas, 3, W), dtype=torch.int32, pin_memory=True)
    e2e_steps = max(1, min(args.steps, 2))
    ctx.restore(ck_path)
    barrier()
    q0 = time.perf_counter()
    for _ in range(e2e_steps):
        iteration()
        ctx.reserve_timeseries(meas)
        ctx.sweep_iter(meas, record=True)
        muca.reweight_context(ctx, 0, grid, 32, stream=stream)
        rc = muca.lib().muca_get_timeseries(ctx._ctx, 0, ts_host.data_ptr())
        if rc != 0:
            raise RuntimeError(muca.last_error(ctx._ctx))
        ctx.get_lnW(0)
    barrier()
    e2e_s = time.perf_counter() - q0
    e2e_value = attempts_step * e2e_steps * world / e2e_s
    os.remove(ck_path)
    nE = V + 1
    h2d = (nE + 4) * 40 * 4  # table upload of the merge (table rows incl. guards x 40 words)
    d2h = nE * 8 + meas * 3 * W * 4 + nE * 8 + grid.size * 5 * 8  # hist, series, lnW, results
    if world > 1:  # the shard's histogram goes through device buffers, not the host
        d2h -= nE * 8

    # reweighting sub-benchmark (FP32 vs FP64), rank 0 only
    rw = mixed = wu = None
    if rank == 0:
        probes = device_probes(torch, muca)
        disordered = disordered_bench(torch, muca, stream)
        rw = reweight_bench(torch, muca)
        mixed = mixed_bench(torch, muca, stream)
        wu = weight_update_bench(muca)

    if rank == 0:
        pk, pk_kind = peaks()
        # the sweep is bound by the per-walker dependency chain and integer issue;
        # the ALU roofline counts the algorithmic integer operations per attempt
        ops_per_attempt = ALGO_INT_OPS
        # the ceiling is the measured rate of the best integer probe kind
        int_kind, int_peak = max(probes["int_ops_per_s"].items(), key=lambda kv: kv[1])
        achieved_ops = ops_per_attempt * attempts_launch / (kern_avg_ms / 1e3)
        l2_bytes = L2_PER_SWEEP.get(res)
        achieved_l2 = (None if l2_bytes is None
                       else l2_bytes * (attempts_launch / (W * L ** 3)) / (kern_avg_ms / 1e3) / 1e9)
        hbm_peak = float(pk.get("hbm_gbs", 6800.0))
        achieved_hbm = 2.0 * attempts_launch / (kern_avg_ms / 1e3) / 1e9
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": "L=48 T=0.9 4096 walkers: 1000-sweep MUCA iteration "
                                   "(graph) + 250 recorded sweeps + FP32 reweight to 4096 Delta",
                       "L": L, "T": T, "walkers": W, "sweeps_per_step": sweeps + meas,
                       "residency": {1: "global", 2: "smem", 3: "split", 4: "scan"}.get(res, str(res)),
                       "walkers_per_block": wpb, "lanes_per_walker": lanes, "seed": s["seed"],
                       "l2": "inputs larger than L2 (lattice 453 MB int8)"},
            "plain": {"value": plain_value, "unit": UNIT, "steps": plain_steps},
            "roofline": {"bound": "alu", "achieved": achieved_ops / 1e12, "peak": int_peak / 1e12,
                         "unit": "Tops/s", "frac": achieved_ops / int_peak,
                         "traffic": traffic_per_launch(res, sweeps),
                         "kernel": {1: "sweep_global_kernel<false>", 2: "sweep_smem_kernel<false>",
                                    3: "sweep_ws_kernel<false, true>",
                                    4: f"sweep_scan_kernel<{L}>"}.get(res, str(res)),
                         "ops_per_attempt": ops_per_attempt,
                         "peak_source": f"measured: muca_probe_int, {int_kind}, "
                                        f"{probes['sm_count']} SMs x 8 blocks x 256 threads "
                                        "(best of the four probe kinds)",
                         "kernel_ms": kern_avg_ms, "attempts_per_launch": attempts_launch,
                         "hbm": {"achieved_gbs": achieved_hbm, "peak_gbs": hbm_peak,
                                 "frac": achieved_hbm / hbm_peak,
                                 "peak_kind": pk_kind, "bytes_per_attempt": 2},
                         "l2": {"achieved_gbs": achieved_l2, "peak_gbs": probes["l2_read_gbs"],
                                "frac": None if achieved_l2 is None
                                else achieved_l2 / probes["l2_read_gbs"],
                                "bytes_per_sweep": l2_bytes,
                                "peak_source": "measured: muca_probe_l2_read, 32 MiB read "
                                               "64 times per launch",
                                "bytes_source": "ncu lts__t_sectors.sum x 32 B of the "
                                                "kernel's capture"}},
            "probes": probes,
            "disordered": disordered,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": args.steps * (launches_per_sweep_call * 2 + reweight_launches),
            "clocks": clk,
            "reweight": rw,
            "batched_mixed": mixed,
            "weight_update": wu,
        }
        if not args.no_cpu:
            line["cpu_baseline"] = cpu_baseline_sample()
        print(json.dumps(line))
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


# Algorithmic integer operations of one attempt: a quarter of a Philox4x32-10
# block (10 rounds x (2 mul-hi + 2 mul-lo + 2 three-way xor + 2 key adds) / 4 = 20),
# the six-neighbour sum (5), proposal and energy change (6), table index and
# compare (4), conditional update of the spin and the three tallies (5).
ALGO_INT_OPS = 40


def mixed_bench(torch, muca, stream, n_it=2, n_full=None):
    """The batching workload: 24 (L, T) groups of 512 walkers, L = 8..32.  Batched:
    one context, one sweep launch per iteration over all groups, the iteration
    loop captured as a CUDA graph, timed over the workload's whole schedule
    (n_full iterations of 300 sweeps from lnW = 0) and over its first n_it
    iterations.  Plain: one context per (L, T) group, run one after the other,
    one sweep launch per iteration plus a host-driven merge, over the first
    n_it iterations (the ratio compares the same iterations).  Contexts (and
    their autotuning) are set up outside the timed regions."""
    mx = wl.MIXED
    groups = wl.mixed_groups()
    sweeps = mx["sweeps"]
    n_full = mx["n_iter"] if n_full is None else n_full
    per_it = sum(g["n_walkers"] * g["L"] ** 3 for g in groups) * sweeps
    attempts = per_it * n_it

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    # warm-up on a context of its own: module loading and the first capture
    ctx = muca.Context(groups, seed=mx["seed"])
    ctx.run_graph(1, sweeps)
    ctx.close()
    ctx = muca.Context(groups, seed=mx["seed"])
    ms_b = timed(lambda: ctx.run_graph(n_it, sweeps))
    ms_rest = timed(lambda: ctx.run_graph(n_full - n_it, sweeps)) if n_full > n_it else 0.0
    cfgs = sorted({ctx.get_config(i) for i in range(len(groups))})
    ctx.close()
    ms_p = 0.0
    for i, g in enumerate(groups):
        c = muca.Context([g], seed=mx["seed"])

        def run():
            for _ in range(n_it):
                c.sweep_iter(sweeps)
                c.merge_update()

        ms_p += timed(run)
        c.close()
    vb, vp = attempts / (ms_b / 1e3), attempts / (ms_p / 1e3)
    vfull = per_it * n_full / ((ms_b + ms_rest) / 1e3)
    return {"workload": "24 groups: L in {8,12,16,20,24,32} x T in {2.0,1.4182,1.0,0.9}, "
                        f"512 walkers each, {n_full} iterations x {sweeps} sweeps from lnW = 0",
            "unit": UNIT, "batched": vfull, "batched_ms": ms_b + ms_rest,
            f"batched_first_{n_it}": vb, "plain_per_config_first": vp,
            "batched_over_plain_first": vb / vp, "plain_ms_first": ms_p,
            "batched_configs": [{"residency": {1: "global", 2: "smem", 3: "split", 4: "scan"}.get(c[0], str(c[0])),
                                 "walkers_per_block": c[1], "lanes_per_walker": c[2]}
                                for c in cfgs]}


def disordered_bench(torch, muca, stream):
    """The disordered model (couplings per bond, its own kernel): 4096
    walkers of L = 24 with bimodal couplings, one weight iteration of 100
    sweeps as a graph after a warm-up iteration; attempts/s, the kernel's
    average launch duration (CUDA events on the launching stream around
    plain sweep launches) and its HBM roofline at 2 B per attempt."""
    d = wl.DISORDERED
    V = d["L"] ** 3
    J = wl.random_bonds(d["L"], d["j1"], d["j2"], seed=d["bond_seed"])
    ctx = muca.Context([{"L": d["L"], "T": d["T"], "n_walkers": d["n_walkers"]}], seed=d["seed"])
    ctx.set_bonds(0, J)
    ctx.run_graph(1, d["sweeps"])
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    ctx.run_graph(1, d["sweeps"])
    b.record(stream)
    torch.cuda.synchronize()
    ms_graph = a.elapsed_time(b)
    ks = []
    for _ in range(2):
        a.record(stream)
        ctx.sweep_iter(d["sweeps"])
        b.record(stream)
        torch.cuda.synchronize()
        ks.append(a.elapsed_time(b))
        ctx.merge_update()
    cfg = ctx.get_config(0)
    ctx.close()
    attempts = d["n_walkers"] * V * d["sweeps"]
    k_ms = sum(ks) / len(ks)
    pk, pk_kind = peaks()
    hbm = float(pk.get("hbm_gbs", 6800.0))
    gbs = 2.0 * attempts / (k_ms / 1e3) / 1e9
    return {"workload": f"L={d['L']} T={d['T']} {d['n_walkers']} walkers, bimodal couplings "
                        f"{d['j1']}/{d['j2']} (p = 1/2), one iteration of {d['sweeps']} sweeps",
            "unit": UNIT, "value": attempts / (ms_graph / 1e3), "kernel_ms": k_ms,
            "kernel": "sweep_bonds_kernel", "residency": cfg[0],
            "roofline": {"bound": "hbm", "achieved_gbs": gbs, "peak_gbs": hbm,
                         "frac": gbs / hbm, "peak_kind": pk_kind, "bytes_per_attempt": 2}}


def weight_update_bench(muca, reps=20):
    """The host FP64 weight update of the graph step on the benchmark window
    (V + 1 = 110593 bins), both recursions, on a seeded merged histogram of
    4096 walkers x 1000 sweeps spread evenly over the bins (a flat-histogram
    iteration); median of `reps` calls of muca_weight_update."""
    V = wl.LARGE["L"] ** 3
    rng = np.random.default_rng(7)
    n = wl.LARGE["n_walkers"] * wl.LARGE["sweeps"]
    H = rng.multinomial(n, np.full(V + 1, 1.0 / (V + 1))).astype(np.uint64)
    out = {"n_e": V + 1, "entries": n}
    for name, kind in (("plain", muca.REC_PLAIN), ("accumulated", muca.REC_ACCUMULATED)):
        lnW, acc = np.zeros(V + 1), np.zeros(V)
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            muca.weight_update(kind, H, lnW, acc)
            ts.append(time.perf_counter() - t0)
        out[name + "_ms"] = 1e3 * sorted(ts)[len(ts) // 2]
    return out


def reweight_bench(torch, muca):
    s = wl.REWEIGHT
    ej, ed, m, lnW, dt = wl.synthetic_series()
    beta = 1.0 / s["T"]
    V = s["L"] ** 3
    grid = wl.delta_grid(dt)
    dj = torch.from_numpy(ej.ravel()).cuda()
    dd = torch.from_numpy(ed.ravel()).cuda()
    dm = torch.from_numpy(m.ravel()).cuda()
    out = {}
    res = {}
    for p in (32, 64):
        r = muca.reweight(dj, dd, dm, lnW, 0, beta, V, grid, p)  # warm-up
        reps = 5
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            r = muca.reweight(dj, dd, dm, lnW, 0, beta, V, grid, p)
        dt_s = (time.perf_counter() - t0) / reps
        res[p] = r
        out[f"fp{p}_pts_per_s"] = len(grid) / dt_s
        out[f"fp{p}_ms"] = dt_s * 1e3
    # stage A alone (exact integer sums per bin and the per-bin statistics):
    # the same call with an empty Delta grid
    muca.reweight(dj, dd, dm, lnW, 0, beta, V, grid[:0], 32)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(10):
        muca.reweight(dj, dd, dm, lnW, 0, beta, V, grid[:0], 32)
    out["stage_a_ms"] = (time.perf_counter() - t0) / 10 * 1e3
    out["stage_a_input_bytes"] = int(12 * ed.size)
    scale = np.maximum(np.abs(res[64]), 1e-3 * np.abs(res[64]).max(axis=0, keepdims=True))
    err = (np.abs(res[32] - res[64]) / np.where(scale == 0, 1, scale)).max(axis=0)
    out["fp32_vs_fp64_max_rel_err"] = dict(zip(["E_J", "E_Delta", "C", "chi", "U4"],
                                               [float(x) for x in err]))
    out["samples"] = int(ed.size)
    out["grid_points"] = int(len(grid))
    out["pairs_per_s_fp32"] = out["fp32_pts_per_s"] * ed.size
    # Delta*_L and C*_L with 20 jackknife blocks (Sec. III), bracket from the
    # FP64 scan above
    c = res[64][:, 2]
    k = int(np.argmax(c))
    lo, hi = grid[max(k - 8, 0)], grid[min(k + 8, len(grid) - 1)]
    pk = muca.find_peak(dj.view(ed.shape), dd.view(ed.shape), lnW, 0, beta, lo, hi, n_jack=20)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    reps = 3
    for _ in range(reps):
        pk = muca.find_peak(dj.view(ed.shape), dd.view(ed.shape), lnW, 0, beta, lo, hi,
                            n_jack=20)
    out["peak"] = {"delta_star": pk[0], "delta_star_err": pk[1], "c_star": pk[2],
                   "c_star_err": pk[3], "jackknife_blocks": 20, "bisection_steps": 60,
                   "ms": (time.perf_counter() - t0) / reps * 1e3}
    # equal-height field and barrier, split between the phases at e = 0.525
    split = int(0.525 * V)
    eq = muca.equal_height(dd.view(ed.shape), lnW, 0, beta, split, lo - 0.01, hi + 0.01,
                           n_jack=20)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        eq = muca.equal_height(dd.view(ed.shape), lnW, 0, beta, split, lo - 0.01, hi + 0.01,
                               n_jack=20)
    out["equal_height"] = {"delta_eqh": eq[0], "delta_eqh_err": eq[1], "barrier": eq[2],
                           "barrier_err": eq[3], "barrier_over_L2": eq[2] / s["L"] ** 2,
                           "jackknife_blocks": 20,
                           "ms": (time.perf_counter() - t0) / reps * 1e3}
    return out


def run_profile_case(what, cfg):
    """Short fixed launches for profiler captures (not timed): the sweep kernel
    of the benchmark workload in a given configuration "residency,walkers per
    block,lanes per walker" (three 1000-sweep weight iterations, the regime of
    the benchmark's steps, then 2 launches of 2 sweeps; no autotuning trials),
    the disordered model's workload (one 100-sweep iteration, then 2 launches
    of 2 sweeps) or the reweighting of the reweight workload (FP32 then
    FP64)."""
    import torch

    from paper_1502_07214_gb300 import muca

    torch.cuda.set_device(0)
    if what == "sweep":
        s = wl.LARGE
        res, wpb, lanes = (int(x) for x in cfg.split(","))
        ctx = muca.Context([{"L": s["L"], "T": s["T"], "n_walkers": s["n_walkers"]}],
                           seed=s["seed"], residency=res, walkers_per_block=wpb,
                           lanes_per_walker=lanes)
        for _ in range(3):
            ctx.sweep_iter(1000)
            ctx.merge_update()
        for _ in range(2):
            ctx.sweep_iter(2)
        ctx.sync()
        print("profile case: sweep", ctx.get_config(0))
        ctx.close()
    elif what == "bonds":
        d = wl.DISORDERED
        ctx = muca.Context([{"L": d["L"], "T": d["T"], "n_walkers": d["n_walkers"]}],
                           seed=d["seed"])
        ctx.set_bonds(0, wl.random_bonds(d["L"], d["j1"], d["j2"], seed=d["bond_seed"]))
        ctx.sweep_iter(d["sweeps"])
        ctx.merge_update()
        for _ in range(2):
            ctx.sweep_iter(2)
        ctx.sync()
        print("profile case: bonds", ctx.get_config(0))
        ctx.close()
    elif what == "peak":
        # Delta*_L (20, 0 and 200 jackknife blocks) and the equal-height search
        # (20 and 0) on the reweight workload, four calls each, the bracket
        # from an FP64 reweighting as in the benchmark's reweight leg
        r = wl.REWEIGHT
        ej, ed, m, lnW, dt = wl.synthetic_series()
        beta, V = 1.0 / r["T"], r["L"] ** 3
        dj, dd, dm = (torch.from_numpy(a.ravel()).cuda() for a in (ej, ed, m))
        grid = wl.delta_grid(dt)
        c = muca.reweight(dj, dd, dm, lnW, 0, beta, V, grid, 64)[:, 2]
        k = int(np.argmax(c))
        lo, hi = grid[max(k - 8, 0)], grid[min(k + 8, len(grid) - 1)]
        for nj in (20, 0, 200):
            for _ in range(4):
                muca.find_peak(dj.view(ed.shape), dd.view(ed.shape), lnW, 0, beta, lo, hi,
                               n_jack=nj)
        split = int(0.525 * V)
        for nj in (20, 0):
            for _ in range(4):
                muca.equal_height(dd.view(ed.shape), lnW, 0, beta, split, lo - 0.01, hi + 0.01,
                                  n_jack=nj)
        torch.cuda.synchronize()
        print("profile case: peak")
    else:
        r = wl.REWEIGHT
        ej, ed, m, lnW, dt = wl.synthetic_series()
        dev = [torch.from_numpy(a.ravel()).cuda() for a in (ej, ed, m)]
        grid = wl.delta_grid(dt)
        for p in (32, 64):
            muca.reweight(*dev, lnW, 0, 1.0 / r["T"], r["L"] ** 3, grid, p)
        print("profile case: reweight")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--profile", choices=["sweep", "reweight", "probes", "bonds", "peak"],
                    help="run a short untimed case for a profiler capture and exit")
    ap.add_argument("--profile-config", default="1,4,8",
                    help="sweep kernel configuration of --profile sweep")
    ap.add_argument("--sweep-config", default="",
                    help="residency,walkers per block,lanes per walker of the benchmark's "
                         "context instead of the autotuner's choice (for profiler runs, whose "
                         "serialised launches change the autotuner's timings)")
    args = ap.parse_args()
    if args.profile == "probes":
        # the device probes alone, printed as JSON (short runs for a capture)
        import torch

        from paper_1502_07214_gb300 import muca

        print(json.dumps(device_probes(torch, muca, iters=256, l2_reps=4)))
        return
    if args.profile:
        run_profile_case(args.profile, args.profile_config)
        return
    if args.warmup < 3:
        args.warmup = 3
    world = env_int("WORLD_SIZE", 1)
    rank = env_int("RANK", 0)
    local_rank = env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
