"""Throughput benchmark of the QCT hot path on GB300.

One step = one pass of the whole path over one batch: initial conditions
(levels + Philox + Eqs. 5-6), adaptive Dormand-Prince integration of every
trajectory to its stop rule, product analysis, histogram reduction and cross
sections.  Default workload: the batched H2 + Ca sweep, 16 collision
energies x 24 impact parameters x 8,192 trajectories = 3,145,728
trajectories, FP64, in one persistent refill-queue launch.  Inputs (the SoA
state, ~600 MB) are larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line (rank 0).  Under torchrun the global workload is N
copies of the sweep's cells with one global trajectory-id range of N x n
lanes; each rank integrates its contiguous shard (shard_range: rank r holds
ids [r n, (r + 1) n), so per-GPU work is fixed: weak scaling), and every step
ends with the exact int64 sum of the per-cell histograms over the ranks
(merge_histograms, NCCL all_reduce), from which rank 0 reports the merged
cross sections.  Other collectives: the timing barrier and a max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# Per-step operation counts of the integrators' Morse kernels, from ncu's
# sass counters (smsp__sass_thread_inst_executed_op_{dfma,dmul,dadd,ffma,
# fmul,fadd}_pred_on.sum and smsp__sass_thread_inst_executed.sum, divided by
# the launch's attempted lane-steps) on the 3,840-lane sweep subset capped
# at 3,000 attempts (bench.py --lanes 4096 --max-steps 3000 --persistent 0).
# Each set holds the SHA-256 of the kernel sources it was measured on; the
# bench recomputes it and marks the roofline's counts stale when the
# sources have changed since.
#   FP64: 342 DFMA + 137 DMUL + 37 DADD per step (six right-hand sides
#   included) = 516 FP64-pipe instructions, 858 FLOP (DFMA = 2).  The
#   DFMA-chain peak runs one DFMA per pipe slot, so pipe_frac below is the
#   fraction of the FP64 pipe's instruction rate the kernel uses.
FP64_FLOP_PER_STEP = 858
FP64_INSTR_PER_STEP = 516
#   FP32: 393 FFMA + 178 FMUL + 39 FADD = 1,004 FLOP and one DADD (the
#   time) in 787 thread instructions per step (all pipes); the kernel is
#   bound by instruction issue, so issue_frac below is the fraction of the
#   SMs' issue rate (4 warp instructions per SM per cycle) it uses.
FP32_FLOP_PER_STEP = 1004
FP32_THREAD_INSTR_PER_STEP = 787
KERNEL_SOURCES = {
    64: ["integrate.cu", "elem64.cuh", "ff.cuh", "texp.cuh", "exp2_table.inc",
         "dp5_tableau.cuh", "step_ctrl.cuh", "pair_force.cuh"],
    32: ["integrate32.cu", "dp5_tableau.cuh"],
}
COUNTS_SOURCE_SHA256 = {
    64: "130d7d1db1e117053912a66c771d9e78751bcc0dba47250e833458f06a8fefb4",
    32: "70e2932855a88f714f4f7b48b180d82a8b03cd6726c5035bdfd2c9d94b9bb1c1",
}
# DRAM bytes per trajectory of the integrator: ncu dram__bytes_read.sum +
# dram__bytes_write.sum of the same FP64 profile case (1,110,784 B read,
# nothing written back during the launch, for 3,840 lanes), per lane: the
# state is loaded once, everything else is in registers; the 16 KB
# exponential table is read from DRAM once and served from L2 to the other
# blocks.  The figure also holds the fetch of the kernel's code, a fixed
# cost per launch.
DRAM_BYTES_PER_LANE = 1110784 / 3840
# The same for the FP32 kernel (559,360 B read, no table): its state is
# loaded as (value, compensation) pairs from the same FP64 arrays.
DRAM_BYTES_PER_LANE_FP32 = 559360 / 3840


def kernel_sources_sha256(precision: int) -> str:
    """SHA-256 over the integrator sources whose instruction counts the
    constants above record."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2304_02731_gb300", "csrc")
    for f in KERNEL_SOURCES[precision]:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sweep",
                    choices=["sweep", "plain", "mixed", "learned"])
    ap.add_argument("--train-lanes", type=int, default=1_000_000,
                    help="learned: trajectories generated to train the network")
    ap.add_argument("--is-lanes", type=int, default=200_000,
                    help="learned: trajectories per estimate (proposal and uniform)")
    ap.add_argument("--train-epochs", type=int, default=24,
                    help="learned: passes over the training lanes")
    ap.add_argument("--train-batch", type=int, default=8192,
                    help="learned: minibatch rows per Adam step")
    ap.add_argument("--train-lr", type=float, default=2e-3, help="learned: Adam learning rate")
    ap.add_argument("--train-precision", type=int, default=32, choices=[64, 32],
                    help="learned: integrator of the training trajectories (the estimates "
                         "are always FP64)")
    ap.add_argument("--per-cell", type=int, default=8192,
                    help="sweep: trajectories per (E, b) cell")
    ap.add_argument("--lanes", type=int, default=0,
                    help="use a stratified subset of this many lanes (profiling runs)")
    ap.add_argument("--max-steps", type=int, default=1_000_000)
    ap.add_argument("--precision", type=int, default=64, choices=[64, 32],
                    help="32: FP32 integrator with Kahan-compensated updates "
                         "(rtol 1e-6, atol 1e-8), FP64 everywhere else")
    ap.add_argument("--persistent", type=int, default=1, choices=[0, 1, 2, 3],
                    help="0: one thread per trajectory; 1: persistent refill queue; "
                         "2 / 3: three / six lanes per trajectory (FP64, small batches)")
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--blocks-per-sm", type=int, default=0)
    ap.add_argument("--tune", type=int, default=1,
                    help="pick the launch shape with qcams_autotune before timing")
    ap.add_argument("--graph", type=int, default=1,
                    help="capture the step (init, run, reduce) in a CUDA graph")
    ap.add_argument("--cpu-per-cell", type=int, default=32,
                    help="oracle sample for cpu_baseline: lanes per cell")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="default sweep run: skip the short measurements of the other "
                         "workloads (plain study, FP32 sweep, mixed study, learned proposal) "
                         "that follow the timed region")
    return ap.parse_args()


def make_workload(args):
    from paper_2304_02731_gb300 import workloads as W
    if args.workload == "sweep":
        wl = W.sweep_h2_ca(per_cell=args.per_cell)
    elif args.workload == "plain":
        wl = W.plain_h2_ca()
    else:
        wl = W.mixed_ca_h()
    if args.lanes and args.lanes < wl.n:
        per = max(1, args.lanes // wl.n_cells)
        wl = wl.take(W.stratified(wl, per))
    if getattr(args, "precision", 64) == 32:
        wl.integ = dict(W.INTEG_FP32)
        wl.name += "_fp32"
    return wl


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
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
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
            except ValueError:
                continue
            for nm, val in zip(names, p[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# oracle timing (CPU baseline and the reference arm)
# ---------------------------------------------------------------------------
def _oracle_chunk(payload):
    import oracle as O
    specs, sid, E, b, v, j, R0, seed, ids, integ_kw = payload
    systems = [O.system_from_spec(s) for s in specs]
    integ = O.make_integ(**integ_kw)
    t0 = time.perf_counter()
    n = 0
    for k in range(len(E)):
        O.run_lanes(systems, sid[k:k + 1], E[k:k + 1], b[k:k + 1], v[k:k + 1], j[k:k + 1], R0,
                    seed, integ, id_offset=int(ids[k]))
        n += 1
    return n, time.perf_counter() - t0


def oracle_rate(wl, per_cell: int, idx_offset: int = 0):
    """Time the oracle as it stands on a stratified sample of the workload,
    one single-threaded oracle process per host core.  Returns
    (trajectories/s, cores, sample description, lanes)."""
    import multiprocessing as mp
    from paper_2304_02731_gb300 import workloads as W
    import oracle as O
    O.build()
    # lanes idx_offset .. idx_offset + per_cell - 1 of every cell (a fresh
    # sample per reference step)
    idx = W.stratified(wl, per_cell, skip=idx_offset)
    cores = os.cpu_count() or 1
    ids = wl.id_offset + idx
    chunks = np.array_split(np.arange(len(idx)), cores)
    payloads = []
    for c in chunks:
        if len(c) == 0:
            continue
        sel = idx[c]
        payloads.append((wl.systems, wl.sys_id[sel], wl.E[sel], wl.b[sel], wl.v[sel],
                         wl.j[sel], wl.R0, wl.seed, ids[c], dict(wl.integ)))
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(len(payloads)) as pool:
        res = pool.map(_oracle_chunk, payloads)
    wall = time.perf_counter() - t0
    n = sum(r[0] for r in res)
    return n / wall, len(payloads), n, wall


def run_reference(args):
    """Reference arm: the CPU oracle, as it stands, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl = make_workload(args)
    for w in range(args.warmup):
        oracle_rate(wl, 1, idx_offset=w)
    rates, walls, ns = [], [], []
    for k in range(args.steps):
        r, cores, n, wall = oracle_rate(wl, args.cpu_per_cell // 2 or 1,
                                        idx_offset=args.warmup + k)
        rates.append(r)
        walls.append(wall)
        ns.append(n)
    value = sum(ns) / sum(walls)
    sample = (f"{ns[0]} lanes per step: {args.cpu_per_cell // 2 or 1} per (E, b) cell of the "
              f"{wl.name} workload, one single-threaded FP64 oracle process per core")
    line = {"impl": "reference", "metric": "trajectories/s (H2+Ca, FP64 RK45)",
            "value": value, "unit": "trajectories/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(walls)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl.name, "trajectories": wl.n},
            "cpu_baseline": {"value": value, "unit": "trajectories/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "trajectories/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2304_02731_gb300 import build as B
    B.build()
    from paper_2304_02731_gb300 import qcams as Q

    from paper_2304_02731_gb300 import shard as SH
    wl = make_workload(args)
    # this rank's shard of the global id range (N x n lanes, weak scaling)
    wl.id_offset, _ = SH.shard_range(world * wl.n, rank, world)
    integ = Q.make_integ(**wl.integ, persistent=args.persistent, block=args.block,
                         blocks_per_sm=args.blocks_per_sm, max_steps=args.max_steps,
                         precision=args.precision)
    tune = None
    if args.tune and args.persistent == 1 and args.precision == 64:
        # launch shape measured on a stratified sample of the workload
        from paper_2304_02731_gb300 import workloads as W
        per = max(1, min(256, wl.n // wl.n_cells))
        sw = wl.take(W.stratified(wl, per))
        sb = Q.Batch.empty(sw.n, dev, sys_id=sw.sys_id, cell=sw.cell, keep_u=False)
        Q.init_states(sw.systems, sb, sw.E, sw.b, sw.v, sw.j, sw.R0, sw.seed, sw.id_offset)
        best, table = Q.autotune(sw.systems, sb, integ, max_attempts=1500)
        integ = best
        tune = {"sample_lanes": sw.n, "max_attempts": 1500,
                "chosen": {"persistent": best.persistent, "block": best.block,
                           "blocks_per_sm": best.blocks_per_sm},
                "variants": [{k: (round(v, 4) if isinstance(v, float) else v)
                              for k, v in r.items()} for r in table]}
        del sb
    batch = Q.Batch.empty(wl.n, dev, sys_id=wl.sys_id, cell=wl.cell, keep_u=False)
    E_d = torch.as_tensor(wl.E, device=dev)
    b_d = torch.as_tensor(wl.b, device=dev)
    v_d = torch.as_tensor(wl.v, device=dev)
    j_d = torch.as_tensor(wl.j, device=dev)
    hist = torch.empty(wl.n_cells * Q.H_STRIDE, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()

    def step(finalize=False):
        Q.init_states(wl.systems, batch, E_d, b_d, v_d, j_d, wl.R0, wl.seed, wl.id_offset)
        Q.run_batch(wl.systems, batch, integ)
        return Q.reduce_xsec(batch, wl.n_cells, wl.cell_b, wl.cell_w, wl.cell_group,
                             wl.n_groups, hist_out=hist, finalize=finalize)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    graph = None
    if args.graph and args.warmup == 0:
        # the library's per-device context is created (cudaMalloc) by its
        # first call, which must not happen inside a stream capture
        Q.levels(wl.systems, [0], [0], [0])
    if args.graph:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        torch.cuda.synchronize()
        run_step = graph.replay
    else:
        run_step = step

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    integ_ms, analyze_ms, steps_total, rhs_total = [], [], 0, 0
    stream = torch.cuda.current_stream()
    e0.record(stream)
    for _ in range(args.steps):
        run_step()
        if world > 1:
            SH.merge_histograms(hist)    # exact int64 sum over the ranks' shards
        st = Q.last_run_stats()          # synchronises; read after each step's run
        integ_ms.append(st["integrate_ms"])
        analyze_ms.append(st["analyze_ms"])
        steps_total += st["steps"]
        rhs_total += st["rhs"]
    e1.record(stream)
    barrier()
    clock_info = clocks.stop()
    ms = e0.elapsed_time(e1)
    t = torch.tensor([ms], device=dev, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = world * wl.n * args.steps / (ms_max * 1e-3)

    # cross sections of the last timed step, for the record (outside the
    # timing): from the merged histograms when the workload is sharded
    if world > 1:
        cells, groups = Q.xsec_from_hist(hist.cpu().numpy(), wl.cell_b, wl.cell_w,
                                         wl.cell_group, wl.n_groups)
        merged_counts = hist.view(wl.n_cells, Q.H_STRIDE)[:, :6].sum(0).cpu().tolist()
    else:
        _, cells, groups = Q.reduce_xsec(batch, wl.n_cells, wl.cell_b, wl.cell_w, wl.cell_group,
                                         wl.n_groups, hist_out=hist, finalize=True)
        merged_counts = None
    torch.cuda.synchronize()
    hb = batch.host()

    # end-to-end through the public API with host buffers (pinned), copies inside
    e2e = None
    if not args.no_e2e:
        pin = lambda a, dt: torch.as_tensor(a, dtype=dt).pin_memory()
        hE, hb_, hv, hj = (pin(wl.E, torch.float64), pin(wl.b, torch.float64),
                           pin(wl.v, torch.int32), pin(wl.j, torch.int32))
        hsid, hcell = pin(wl.sys_id, torch.int32), pin(wl.cell, torch.int32)
        hhist = torch.empty(wl.n_cells * Q.H_STRIDE, dtype=torch.int64).pin_memory()
        barrier()
        t0 = time.perf_counter()
        e2e_steps = min(args.steps, 3)   # each full-size step is seconds long
        for _ in range(e2e_steps):
            batch.sys_id.copy_(hsid, non_blocking=True)
            batch.cell.copy_(hcell, non_blocking=True)
            E_d.copy_(hE, non_blocking=True)
            b_d.copy_(hb_, non_blocking=True)
            v_d.copy_(hv, non_blocking=True)
            j_d.copy_(hj, non_blocking=True)
            step()
            if world > 1:
                SH.merge_histograms(hist)
            hhist.copy_(hist, non_blocking=True)
        barrier()
        wall = time.perf_counter() - t0
        h2d = sum(x.numel() * x.element_size() for x in (hE, hb_, hv, hj, hsid, hcell))
        e2e = {"value": world * wl.n * e2e_steps / wall, "unit": "trajectories/s",
               "steps": e2e_steps,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(hhist.numel() * 8)}

    # roofline of the dominant kernel (the integrator): the FP64 pipe for
    # the FP64 kernel, the FP32 FMA pipe for the FP32 one
    peak = Q.fma_peak(args.precision)    # measured here: MEASURED_PEAKS.json has no FP64/FP32 figure
    avg_integ_ms = float(np.mean(integ_ms))
    steps_per_launch = steps_total / max(1, args.steps)
    flop_per_step = FP64_FLOP_PER_STEP if args.precision == 64 else FP32_FLOP_PER_STEP
    roofline = {"bound": "alu", "unit": "TFLOP/s", "peak": peak / 1e12,
                "peak_source": f"measured FP{args.precision} FMA-chain microbenchmark "
                               f"(qcams_fma_peak), this run",
                "traffic": ((DRAM_BYTES_PER_LANE if args.precision == 64 else DRAM_BYTES_PER_LANE_FP32)
                            * wl.n if args.workload == "sweep" else None),
                "traffic_note": "ncu dram bytes of the 3,840-lane profile case scaled by lanes"}
    if args.workload in ("sweep", "plain"):
        # FLOP counts are those of the Morse kernel (H2 + Ca systems)
        ach = flop_per_step * steps_per_launch / (avg_integ_ms * 1e-3)
        roofline.update(achieved=ach / 1e12, frac=ach / peak, flop_per_step=flop_per_step)
        if args.precision == 64:
            rate = FP64_INSTR_PER_STEP * steps_per_launch / (avg_integ_ms * 1e-3)
            roofline.update(fp64_instr_per_step=FP64_INSTR_PER_STEP, pipe_frac=rate / (peak / 2))
        else:
            props = torch.cuda.get_device_properties(dev)
            mhz = (clock_info or {}).get("sm_mhz") or 2070.0
            issue = props.multi_processor_count * 4 * 32 * mhz * 1e6   # thread instructions / s
            rate = FP32_THREAD_INSTR_PER_STEP * steps_per_launch / (avg_integ_ms * 1e-3)
            roofline.update(thread_instr_per_step=FP32_THREAD_INSTR_PER_STEP,
                            issue_frac=rate / issue)
    else:
        roofline.update(achieved=None, frac=None)
    counts_current = kernel_sources_sha256(args.precision) == COUNTS_SOURCE_SHA256[args.precision]
    roofline.update(counts_current=counts_current,
                    counts_note=("per-step counts measured on these kernel sources"
                                 if counts_current else
                                 "kernel sources changed since the per-step counts were "
                                 "measured: achieved / frac use stale counts"))
    roofline.update(steps_per_launch=steps_per_launch, integrate_ms=avg_integ_ms,
                    analyze_ms=float(np.mean(analyze_ms)),
                    rest_of_step_ms=ms_max / args.steps - avg_integ_ms,
                    rhs_per_launch=rhs_total / max(1, args.steps))

    cpu = None
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        r, cores, n, wall = oracle_rate(wl, args.cpu_per_cell)
        cpu = {"value": r, "unit": "trajectories/s", "cores": cores, "kind": "oracle",
               "sample": f"{n} lanes ({args.cpu_per_cell} per (E, b) cell), {wall:.1f} s wall "
                         f"on {cores} host cores",
               "seconds_per_trajectory_one_core": cores * wall / max(n, 1),
               "one_core_trajectories_per_s": n / (cores * wall)}

    cls_counts = np.bincount(hb["cls"], minlength=6).tolist()
    line = {
        "metric": f"trajectories/s (H2+Ca, FP{args.precision} RK45)", "value": value,
        "unit": "trajectories/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": f"f{args.precision}",
        "data": "synthetic",
        "config": {"workload": wl.name, "trajectories_per_gpu": wl.n,
                   "launch": {0: "one thread/lane", 1: "persistent refill queue",
                              2: "three lanes/trajectory",
                              3: "six lanes/trajectory"}[integ.persistent]
                   + (", CUDA graph" if graph is not None else "")
                   + (f", block {integ.block or 128} x {integ.blocks_per_sm or 1}/SM variant"
                      if integ.persistent < 2 else
                      f", one warp ({10 if integ.persistent == 2 else 5} trajectories) per block"),
                   "autotune": tune,
                   "rtol": wl.integ["rtol"], "atol": wl.integ["atol"],
                   "arithmetic": ("FP64 state, forces and new-state sums; stage corrections, "
                                  "the error estimate and the exponential's quadratic as "
                                  "float-float (FP32 pairs); error norm in FP32"
                                  if args.precision == 64 else
                                  "FP32 stages with compensated (Kahan) state updates; "
                                  "FP64 time, levels and product analysis"),
                   "l2": "inputs larger than L2 (SoA state > 129 MB)",
                   "parallelism": (f"id-range shards x{world} + int64 all_reduce of the "
                                   f"histograms" if world > 1 else "single GPU")},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": 8 * args.steps,
        "clocks": clock_info,
        "outcomes": {"cls_counts_Q_RAC_RBC_D_AMBIG_FAIL": cls_counts,
                     "merged_cls_counts_all_ranks": merged_counts,
                     "sigma_entries": "Q, R_AC, R_BC, D, AMBIG, FAIL, R_AC+R_BC",
                     "sigma_first_group": groups[0, :, 0].tolist() if groups is not None and
                     len(groups) else None},
    }
    if (rank == 0 and world == 1 and args.workload == "sweep" and args.precision == 64
            and not args.no_extras and not args.lanes):
        line["other_configs"] = run_extras(args, dev)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def time_steps(Q, wl, integ, steps, warmup, dev):
    """Time `steps` graph replays of init -> integrate -> analyse -> reduce
    on workload wl after `warmup` eager steps (CUDA events on the launching
    stream, clocks sampled meanwhile).  Returns a dict of the figures."""
    import torch
    batch = Q.Batch.empty(wl.n, dev, sys_id=wl.sys_id, cell=wl.cell, keep_u=False)
    E_d, b_d = torch.as_tensor(wl.E, device=dev), torch.as_tensor(wl.b, device=dev)
    v_d, j_d = torch.as_tensor(wl.v, device=dev), torch.as_tensor(wl.j, device=dev)
    hist = torch.empty(wl.n_cells * Q.H_STRIDE, dtype=torch.int64, device=dev)

    def step():
        Q.init_states(wl.systems, batch, E_d, b_d, v_d, j_d, wl.R0, wl.seed, wl.id_offset)
        Q.run_batch(wl.systems, batch, integ)
        Q.reduce_xsec(batch, wl.n_cells, hist_out=hist, finalize=False)

    for _ in range(max(1, warmup)):
        step()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    integ_ms, analyze_ms = [], []
    e0.record(stream)
    for _ in range(steps):
        graph.replay()
        st = Q.last_run_stats()
        integ_ms.append(st["integrate_ms"])
        analyze_ms.append(st["analyze_ms"])
    e1.record(stream)
    torch.cuda.synchronize()
    clock_info = clocks.stop()
    ms = e0.elapsed_time(e1) / steps
    _, cells, groups = Q.reduce_xsec(batch, wl.n_cells, wl.cell_b, wl.cell_w, wl.cell_group,
                                     wl.n_groups, hist_out=hist)
    cls = np.bincount(batch.cls.cpu().numpy(), minlength=6).tolist()
    return {"workload": wl.name, "trajectories": wl.n, "steps": steps, "warmup": warmup,
            "value": wl.n / (ms * 1e-3), "unit": "trajectories/s", "ms_per_step": ms,
            "integrate_ms": float(np.mean(integ_ms)), "analyze_ms": float(np.mean(analyze_ms)),
            "launch": (f"{'three' if integ.persistent == 2 else 'six'} lanes per trajectory, "
                       "CUDA graph" if integ.persistent >= 2 else
                       f"persistent refill queue, CUDA graph, block {integ.block or 128} x "
                       f"{integ.blocks_per_sm or 1}/SM variant"),
            "cls_counts_Q_RAC_RBC_D_AMBIG_FAIL": cls, "clocks": clock_info}


def run_extras(args, dev):
    """Short measurements of the other workloads after the headline sweep
    (single GPU, outside its timed region): the 1,000-lane plain study (the
    autotuner's launch, and one thread per trajectory for comparison) and
    the 2,000,000-lane mixed study in FP64 (autotuned launch shape), the
    sweep with the FP32 integrator, and the learned-proposal study."""
    import torch
    from paper_2304_02731_gb300 import qcams as Q
    from paper_2304_02731_gb300 import workloads as W
    out = {}

    def tuned(wl, integ):
        per = max(1, min(256, wl.n // wl.n_cells))
        sw = wl.take(W.stratified(wl, per))
        sb = Q.Batch.empty(sw.n, dev, sys_id=sw.sys_id, cell=sw.cell, keep_u=False)
        Q.init_states(sw.systems, sb, sw.E, sw.b, sw.v, sw.j, sw.R0, sw.seed, sw.id_offset)
        best, _ = Q.autotune(sw.systems, sb, integ, max_attempts=1500)
        return best

    wl = W.plain_h2_ca()
    out["plain_fp64"] = time_steps(Q, wl, tuned(wl, Q.make_integ(**wl.integ, persistent=True)),
                                   5, 3, dev)
    out["plain_fp64_one_thread"] = time_steps(
        Q, wl, Q.make_integ(**wl.integ, persistent=True, block=64, blocks_per_sm=1), 5, 3, dev)
    wl = W.sweep_h2_ca()
    wl.integ = dict(W.INTEG_FP32)
    wl.name += "_fp32"
    out["sweep_fp32"] = time_steps(
        Q, wl, Q.make_integ(**wl.integ, persistent=True, precision=32), 5, 3, dev)
    del wl
    torch.cuda.empty_cache()
    wl = W.mixed_ca_h()
    out["mixed_fp64"] = time_steps(Q, wl, tuned(wl, Q.make_integ(**wl.integ, persistent=True)),
                                   1, 1, dev)
    del wl
    torch.cuda.empty_cache()
    learned = learned_study(argparse.Namespace(train_lanes=1_000_000, is_lanes=200_000,
                                               train_precision=32, warmup=1, train_epochs=24,
                                               train_batch=8192, train_lr=2e-3))
    out["learned"] = {k: learned[k] for k in ("metric", "value", "unit", "config", "training",
                                               "amortised", "clocks")}
    out["learned"]["per_energy_fom_gain"] = [r["fom_gain"] for r in learned["per_energy"]]
    return out


def run_learned(args):
    print(json.dumps(learned_study(args)), flush=True)
    return 0


def learned_study(args):
    """The learned-proposal study: train the outcome network on trajectories
    of the LJ(12,6) Ca-H system drawn like the mixed study, then estimate
    sigma_R = sigma(AC+B) + sigma(BC+A) at E = 0.05, 0.10, 0.15 hartree for
    the most reactive (v, j) with the learned proposal and with uniform
    sampling, from the same number of trajectories.  Reports each estimate,
    its standard error and GPU time, and FOM = 1 / (SE^2 T); the ratio of
    FOMs is the gain in standard error per GPU-second at equal accuracy.

    The training trajectories are integrated with the FP32 integrator by
    default (--train-precision 32): their classes only shape the proposal,
    and every estimate integrates its own lanes in FP64, so the estimator is
    unbiased whatever the labels.  The network costs C = (training-data
    generation + training) seconds once.  Spread over K estimates, an estimate costs T_is + C / K, so its
    amortised FOM ratio is G_K = FOM_u^-1 / (SE_is^2 (T_is + C / K)) and
    the learned proposal wins end to end from K* = C / (T_is (G - 1))
    estimates on (G the per-estimate ratio).  Both are reported, with K = 3
    (the energies of this run) and K*, per energy and overall."""
    import torch
    from paper_2304_02731_gb300 import build as B
    B.build()
    from paper_2304_02731_gb300 import learned as L
    from paper_2304_02731_gb300 import qcams as Q
    from paper_2304_02731_gb300 import workloads as W
    torch.cuda.set_device(0)
    spec_sys = W.SYS_H2_CA_LJ12
    # warm-up: load the generation and training kernels once (a few lanes,
    # a few steps), so that the timed network cost is the steady-state one
    xw, cw, _ = L.generate(spec_sys, 4096, seed=7, precision=args.train_precision)
    L.train(Q.MLP(seed=2), xw, cw, epochs=1, batch=1024, lr=2e-3)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    t0 = time.perf_counter()
    x, cls, host = L.generate(spec_sys, args.train_lanes, seed=101,
                              precision=args.train_precision)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    mlp = Q.MLP(seed=1)
    t0 = time.perf_counter()
    losses = L.train(mlp, x, cls, epochs=args.train_epochs, batch=args.train_batch,
                     lr=args.train_lr)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    cost = t_gen + t_train
    v, j, frac = L.best_state(host)
    energies = (0.05, 0.10, 0.15)
    rows = []
    for E in energies:
        spec = Q.proposal_spec(E, v, j)
        for w in range(args.warmup):
            L.estimate_uniform(spec_sys, spec, 4096, seed=7 + w)
            L.estimate_is(spec_sys, mlp, spec, 4096, seed=9 + w)
        eu = L.estimate_uniform(spec_sys, spec, args.is_lanes, seed=1000)
        eq = L.estimate_is(spec_sys, mlp, spec, args.is_lanes, seed=2000)
        gain = eq.fom / eu.fom
        amort = 1.0 / (eq.se ** 2 * (eq.seconds + cost / len(energies))) / eu.fom
        k_star = cost / (eq.seconds * (gain - 1.0)) if gain > 1.0 else None
        rows.append({"E": E, "uniform": eu.__dict__, "learned": eq.__dict__,
                     "fom_uniform": eu.fom, "fom_learned": eq.fom, "fom_gain": gain,
                     "fom_gain_amortised_over_run": amort,
                     "break_even_estimates": k_star,
                     "agree_sigmas": abs(eq.sigma - eu.sigma) / math.hypot(eq.se, eu.se)})
    clock_info = clocks.stop()
    gains = [r["fom_gain"] for r in rows]
    g_mean = float(np.exp(np.mean(np.log(gains))))
    t_is = float(np.mean([r["learned"]["seconds"] for r in rows]))
    amort = [r["fom_gain_amortised_over_run"] for r in rows]
    line = {"metric": "sigma_R std-error per GPU-second: learned proposal / uniform (FOM ratio)",
            "value": g_mean, "unit": "x",
            "higher_is_better": True, "n_gpus": 1, "dtype": "f64 integration, bf16 network",
            "data": "synthetic",
            "config": {"workload": "LJ(12,6) Ca-H + H2, mixed-study lanes", "train_lanes":
                       args.train_lanes, "train_precision": f"FP{args.train_precision}",
                       "is_lanes_per_estimate": args.is_lanes,
                       "state": {"v": v, "j": j, "train_reactive_fraction": frac}},
            "training": {"generate_s": t_gen, "train_s": t_train, "loss_first": losses[0],
                         "loss_last": losses[-1], "epochs": len(losses),
                         "batch": args.train_batch, "lr": args.train_lr},
            "amortised": {"network_cost_s": cost,
                          "fom_gain_amortised_over_run": float(np.exp(np.mean(np.log(amort)))),
                          "estimates_in_run": len(energies),
                          "break_even_estimates": (cost / (t_is * (g_mean - 1.0))
                                                   if g_mean > 1.0 else None),
                          "break_even_lanes": (cost / (t_is * (g_mean - 1.0)) * args.is_lanes
                                               if g_mean > 1.0 else None),
                          "note": "value is the per-estimate FOM ratio (network already "
                                  "trained); the amortised ratio charges generation + training "
                                  "to the run's estimates"},
            "clocks": clock_info,
            "per_energy": rows}
    return line


def main():
    args = parse()
    if args.workload == "learned":
        return run_learned(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
