#!/usr/bin/env python
"""Benchmark of the batched Burgers hot path on B300.

One step = one pass of the hot path over the batched ensemble workload
(4096 periodic rows x 4096 nodes on [0, 2 pi), seeded random-Fourier u0,
log-uniform nu): CFL time step per row on the device (Eq. 7-8), 2000 explicit
forward-Euler upwind/central steps (Eq. 21) and 200 lagged-coefficient BTCS
steps at 10x that dt (Sec. 2.4, cyclic solves via Sherman-Morrison), both from
u0, in FP32. Value = cell-updates per second over all ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank solves its own 4096 rows (weak scaling, no data-path
collective; NCCL only for the barrier and the max-over-ranks time).
"""
from __future__ import annotations

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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s (explicit & BTCS) vs plain at L2<=1e-5 vs FP64; serve p50/p99"
B_ROWS, N_NODES = 4096, 4096
EXPLICIT_STEPS, BTCS_STEPS, BTCS_DT_FACTOR, CFL = 2000, 200, 10.0, 0.4
CELLS_PER_STEP = B_ROWS * N_NODES * (EXPLICIT_STEPS + BTCS_STEPS)
WORKLOAD = (f"batched ensemble: {B_ROWS} periodic rows x {N_NODES} nodes, random-Fourier u0, "
            f"nu log-U[1e-3,1e-1]; CFL dt on device; {EXPLICIT_STEPS} explicit steps at CFL 0.4 + "
            f"{BTCS_STEPS} BTCS steps at 10x dt, both from u0")
# FMA-pipe FP32 lane-operations per cell-update of the explicit kernel (on
# packed f32x2 pairs, two lane-operations per instruction): the increment
# p (ur - u) - q (u - ul), p = s - r min(u, 0), q = s + r max(u, 0), costs one
# difference (the other is the neighbour's), one FMA each for p and q and two
# FMA that add it to the node's running sum d; evaluating u = uh + d costs one
# more, and every 32 steps three fold d into uh. min and max run on the ALU
# pipe (EXPLICIT_ALU per cell-update).
EXPLICIT_OPS = 6 + 3 / 32
EXPLICIT_ALU = 2
# BTCS: assembly 4 + right-hand side 3 + forward elimination 6 (+1 MUFU rcp) +
# backward 3 + back-substitution 2 + compensated addition 4 (+2 min/max on ALU)
BTCS_OPS = 22
LARGE_EXPLICIT_STEPS, LARGE_BTCS_STEPS = 10000, 100
# RK4 (Eq. 22) on the bench ensemble at the forward-Euler dt. FMA-pipe FP32
# lane-operations per cell-update (packed pairs, as the explicit kernel): u =
# uh + d once per step (1) and the first stage's increment (5: a difference,
# p, q and two FMA); stages 2-4 add the stage offset (1), the increment (5)
# and the weighted accumulation (1); the step adds the sum/6 to d (1); every
# 32 steps a three-operation fold. Plus 8 min/max on the ALU pipe.
RK4_STEPS = 500
RK4_OPS = 6 + 3 * 7 + 1 + 3 / 32
# The method's own work per explicit cell-update (Eq. 21 with the upwind side
# chosen by sign): two differences, the two upwind/central coefficients (|u|,
# two products), two products and two additions into u: 9 FP32 operations,
# the figure the roofline's headline fraction uses (the kernel executes fewer
# FMA-pipe instructions, EXPLICIT_OPS, because its FMAs fuse some of them).
ALG_EXPLICIT_OPS = 9
FP32_LANES = 128


def hbm_peak():
    """HBM copy bandwidth of the B300s (GB/s) and where it came from."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), "measured"
    except Exception:  # noqa: BLE001
        return 6400.0, "fallback"



def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms",
                 "50", "-i", str(self.index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception as e:  # noqa: BLE001
            log("clock sampling unavailable:", e)
            self.proc = None
        return self

    def ready(self, timeout: float = 5.0):
        """Waits for the first sample (the tool's start-up), then counts only
        the samples taken from here on."""
        t0 = time.perf_counter()
        while self.proc is not None and not self.lines and time.perf_counter() - t0 < timeout:
            time.sleep(0.01)
        self.mark = len(self.lines)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:  # noqa: BLE001
            self.proc.kill()
        sm, mx, reasons, pw = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[getattr(self, "mark", 0):]:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                pw.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None,
                "samples": len(sm), "reasons": sorted(reasons)}


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


def shard_ids(rank: int, world: int, rows: int = B_ROWS) -> np.ndarray:
    """Rows of the ensemble owned by `rank`: each rank solves its own `rows`
    instances (weak scaling), instance ids rank*rows .. (rank+1)*rows - 1."""
    return np.arange(rank * rows, (rank + 1) * rows, dtype=np.int64)


def allreduce_max(x: float, world: int) -> float:
    """Max over ranks (the slowest rank sets the job time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def traffic_record(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path)).get(kernel)
    except Exception:  # noqa: BLE001
        return None
    if not rec:
        return None
    h = hashlib.sha256()
    for f in rec.get("sources", []):
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest()[:16] != rec.get("digest"):
        return None
    return rec.get("bytes_per_launch")


# ---------------------------------------------------------------------------
def cpu_baseline_sample(target_s: float = 12.0, ids_offset: int = 0):
    """Oracle (as it stands) on a bounded sample of the workload, all host cores,
    plus the same on one core (a few rows)."""
    import oracle
    from paper_2601_12204_b300 import workloads as W
    threads = oracle.max_threads()

    def run(count, nthreads):
        ens = W.fourier_ensemble(count, N_NODES, ids=np.arange(ids_offset, ids_offset + count))
        dts = np.array([oracle.cfl_dt(ens.row(b), ens.dxs[b], ens.nus[b], CFL)
                        for b in range(count)])
        t0 = time.perf_counter()
        oracle.explicit_batch(ens.u0, ens.offsets, ens.ns, ens.bcs, ens.dxs, ens.nus, dts,
                              np.full(count, EXPLICIT_STEPS), nthreads)
        oracle.btcs_batch(ens.u0, ens.offsets, ens.ns, ens.bcs, ens.dxs, ens.nus,
                          dts * BTCS_DT_FACTOR, np.full(count, BTCS_STEPS), nthreads)
        return time.perf_counter() - t0

    count = threads
    t = run(count, threads)
    if t < target_s / 3:
        count = max(threads, int(count * target_s / max(t, 1e-3)) // threads * threads)
        count = min(count, B_ROWS)
        t = run(count, threads)
    cells = count * N_NODES * (EXPLICIT_STEPS + BTCS_STEPS)
    one = 4
    t1 = run(one, 1)
    return {"value": cells / t, "unit": "cell-updates/s", "cores": threads, "kind": "oracle",
            "sample": f"{count} of {B_ROWS} rows (ids 0..{count - 1}), full {EXPLICIT_STEPS} "
                      f"explicit + {BTCS_STEPS} BTCS steps, FP64 C oracle, {t:.1f} s",
            "one_core": {"value": one * N_NODES * (EXPLICIT_STEPS + BTCS_STEPS) / t1,
                         "cores": 1, "sample": f"rows 0..{one - 1}, same steps, {t1:.2f} s"}}


# ---------------------------------------------------------------------------
def run_reference(args):
    """--impl reference: the FP64 CPU oracle on the host cores, same metric."""
    world, rank, _ = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0
    if rank != 0:
        return
    import oracle
    from paper_2601_12204_b300 import workloads as W
    threads = oracle.max_threads()
    count = threads
    ens = W.fourier_ensemble(count, N_NODES)
    dts = np.array([oracle.cfl_dt(ens.row(b), ens.dxs[b], ens.nus[b], CFL) for b in range(count)])

    def step():
        oracle.explicit_batch(ens.u0, ens.offsets, ens.ns, ens.bcs, ens.dxs, ens.nus, dts,
                              np.full(count, EXPLICIT_STEPS), threads)
        oracle.btcs_batch(ens.u0, ens.offsets, ens.ns, ens.bcs, ens.dxs, ens.nus,
                          dts * BTCS_DT_FACTOR, np.full(count, BTCS_STEPS), threads)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    el = time.perf_counter() - t0
    cells = count * N_NODES * (EXPLICIT_STEPS + BTCS_STEPS) * args.steps
    v = cells / el
    sample = (f"{count} of {B_ROWS} rows per step (one per host thread), full "
              f"{EXPLICIT_STEPS}+{BTCS_STEPS} steps, FP64 C oracle")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "cell-updates/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1000 * el / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "rows_per_step": count, "n": N_NODES},
           "cpu_baseline": {"value": v, "unit": "cell-updates/s", "cores": threads,
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
def run_ours(args):
    import torch

    from paper_2601_12204_b300 import _lib as L
    from paper_2601_12204_b300 import workloads as W
    from paper_2601_12204_b300.api import Batch, Context

    world, rank, local = dist_setup()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    ctx = Context(local)
    F32, F64 = L.BURGERS_F32, L.BURGERS_F64

    t0 = time.perf_counter()
    ids = shard_ids(rank, world)
    ens = W.fourier_ensemble(B_ROWS, N_NODES, ids=ids)
    log(f"[rank {rank}] ensemble generated in {time.perf_counter() - t0:.1f} s")
    u0 = torch.tensor(ens.u0, dtype=torch.float32, device=dev)
    ue = torch.empty_like(u0)
    ub = torch.empty_like(u0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    probe = Batch.from_ensemble(ens, 1.0, 0, F32)
    stream = torch.cuda.current_stream(dev)

    def batches(dt0):
        be = Batch.from_ensemble(ens, dt0, EXPLICIT_STEPS, F32)
        bb = Batch.from_ensemble(ens, dt0 * BTCS_DT_FACTOR, BTCS_STEPS, F32)
        return be, bb

    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    # the timed step: the CFL time step of Eq. 7-8 on the device, then both
    # advances reading it there (no host synchronisation inside the step)
    dtd = torch.empty(B_ROWS, dtype=torch.float64, device=dev)
    bde = Batch.from_ensemble(ens, 1.0, EXPLICIT_STEPS, F32)  # dt comes from dtd
    bdb = Batch.from_ensemble(ens, 1.0, BTCS_STEPS, F32)

    def step(timing):
        e0, e1, e2, e3 = ev(), ev(), ev(), ev()
        e0.record(stream)
        ctx.cfl_dt_device(probe, u0, CFL, dtd)
        ue.copy_(u0)
        e1.record(stream)
        ctx.advance_dt_device(L.BURGERS_EXPLICIT, bde, ue, dtd, 1.0)
        e2.record(stream)
        ub.copy_(u0)
        ctx.advance_dt_device(L.BURGERS_BTCS, bdb, ub, dtd, BTCS_DT_FACTOR)
        e3.record(stream)
        timing.append((e0, e1, e2, e3))

    # launch shapes for this workload from the autotuner (untimed set-up)
    dt_probe = ctx.cfl_dt(probe, u0, CFL)
    be0, bb0 = batches(dt_probe)
    if args.tune_file and os.path.exists(args.tune_file):
        ctx.tune_load(args.tune_file)
        tuned = {"loaded": args.tune_file}
    else:
        tuned = {"explicit_classes": ctx.autotune(L.BURGERS_EXPLICIT, be0, u0, probe_steps=200),
                 "btcs_classes": ctx.autotune(L.BURGERS_BTCS, bb0, u0, probe_steps=50)}
        if args.tune_file:
            ctx.tune_save(args.tune_file)
    tuned["table"] = _tune_lines(ctx)  # "key nt c k" of the shapes the timed steps use
    for _ in range(max(3, args.warmup)):
        flush.zero_()
        step([])
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(local).start().ready()
    lc0 = ctx.launch_count()
    timing = []
    for _ in range(args.steps):
        flush.zero_()
        step(timing)
    torch.cuda.synchronize()
    launches = ctx.launch_count() - lc0
    clk = clocks.stop()
    barrier(world)
    tot = sum(a.elapsed_time(d) for a, b, c, d in timing)
    t_expl = statistics.median(b.elapsed_time(c) for a, b, c, d in timing)
    t_btcs = statistics.median(c.elapsed_time(d) for a, b, c, d in timing)
    tot_max = allreduce_max(tot, world)
    ms_per_step = tot_max / args.steps
    value = CELLS_PER_STEP * world / (ms_per_step / 1000.0)

    res = {"metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world,
           "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms_per_step,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic (seeded random-Fourier ensemble, no dataset)",
           "config": {"workload": WORKLOAD, "global_batch": B_ROWS * world, "n": N_NODES,
                      "explicit_steps": EXPLICIT_STEPS, "btcs_steps": BTCS_STEPS,
                      "l2": "256 MiB buffer written between timed steps (flush)",
                      "parallelism": f"rows sharded over {world} rank(s), no data-path collective"},
           "gpu_launches": int(launches), "clocks": clk, "autotuned": tuned}

    # ---- roofline of the dominant kernel (explicit resident, FP32 issue bound)
    sms = ctx.get(L.BURGERS_INFO_SM_COUNT)
    peak_ops = sms * FP32_LANES * 2032e6 / 1e12
    # measured FMA issue rates (burgers_fma_peak), right after the timed region
    fma32 = ctx.fma_peak(L.BURGERS_F32) / 1e12
    fma64 = ctx.fma_peak(L.BURGERS_F64) / 1e12
    cells_e = B_ROWS * N_NODES * EXPLICIT_STEPS / (t_expl / 1000.0)
    ach = ALG_EXPLICIT_OPS * cells_e / 1e12
    ach_x = EXPLICIT_OPS * cells_e / 1e12
    res["roofline"] = {
        "bound": "alu", "kernel": "k_explicit_resident<float, tuned shape, exact>",
        "achieved": ach, "peak": peak_ops, "unit": "Tops/s (FP32 lane-operations)",
        "frac": ach / peak_ops, "traffic": traffic_record("explicit_resident_f32_4096"),
        "per_unit": f"{ALG_EXPLICIT_OPS} FP32 operations per cell-update (the method's work, Eq. 21); "
                    f"4096 rows x 4096 nodes x 2000 steps per launch",
        "peak_note": f"{sms} SMs x {FP32_LANES} FP32 lanes x 2032 MHz (max SM clock)",
        "peak_measured": fma32, "frac_measured": ach / fma32,
        "peak_measured_note": "burgers_fma_peak: 8 independent FMA chains x 2048 threads per SM, "
                              "at the clock of the run",
        "executed": {"per_unit": f"{EXPLICIT_OPS:.4g} FMA-pipe FP32 lane-operations per cell-update "
                                 f"(what the kernel executes, on packed f32x2 pairs) + "
                                 f"{EXPLICIT_ALU} min/max on the ALU pipe",
                     "achieved": ach_x, "frac": ach_x / peak_ops, "frac_measured": ach_x / fma32},
        "kernel_ms": t_expl}
    achb = BTCS_OPS * B_ROWS * N_NODES * BTCS_STEPS / (t_btcs / 1000.0) / 1e12
    res["roofline_btcs"] = {"bound": "alu", "kernel": "k_btcs_resident<float, tuned shape, exact>",
                            "achieved": achb, "peak": peak_ops, "unit": "Tops/s (FP32 lane-instructions)",
                            "frac": achb / peak_ops, "kernel_ms": t_btcs,
                            "traffic": traffic_record("btcs_resident_f32_4096"),
                            "peak_measured": fma32, "frac_measured": achb / fma32,
                            "per_unit": f"{BTCS_OPS} FMA-pipe FP32 instr + 1 MUFU rcp + 2 ALU per cell-update"}
    res["fma_peak_measured"] = {"fp32_tops": fma32, "fp64_tops": fma64,
                                "unit": "T lane-FMA/s"}
    res["explicit_cups"] = B_ROWS * N_NODES * EXPLICIT_STEPS / (t_expl / 1000.0)
    res["btcs_cups"] = B_ROWS * N_NODES * BTCS_STEPS / (t_btcs / 1000.0)

    if not args.quick:
        res.update(extras(args, ctx, ens, u0, batches, probe, dev, world, rank))
        if args.serve_seconds > 0 and world == 1:
            log("serving ...")
            res["serve"] = serve_bench(ctx, dev, args.serve_seconds, rate=args.serve_rate)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        log("cpu baseline ...")
        res["cpu_baseline"] = cpu_baseline_sample()
    ctx.close()
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def differentiation_bench(ctx, dev):
    """Differentiation workload: J = 1/2 |u(T) - target|^2 over B = 1024 periodic rows of
    2048 nodes (random-Fourier u0; the target is the same run from the
    ensemble of the next seed, with a dt per row that satisfies the CFL limit
    of both initial fields), 2000 explicit / 200 BTCS steps, gradients by
    the hand-written adjoint with sqrt-step checkpointing. Times the forward
    call and the adjoint call (which recomputes the forward states from its
    checkpoints, then runs the reverse sweep); FP32 gradients against the
    FP64 GPU gradients of the same problem."""
    import torch

    from paper_2601_12204_b300 import _lib as L
    from paper_2601_12204_b300 import workloads as W
    from paper_2601_12204_b300.api import Batch
    from paper_2601_12204_b300.diagnostics import fp32_gradient_bar, trajectory_stats
    F32, F64 = L.BURGERS_F32, L.BURGERS_F64
    rows, n = 1024, 2048
    ens = W.fourier_ensemble(rows, n)
    tgt = W.fourier_ensemble(rows, n, seed=W.DEFAULT_SEED + 1)
    u64 = torch.tensor(ens.u0, dtype=torch.float64, device=dev)
    t64 = torch.tensor(tgt.u0, dtype=torch.float64, device=dev)
    probe = Batch.from_ensemble(ens, 1.0, 0, F64)
    # one dt per row that is stable for both runs (the target's u0 can be larger)
    dt0 = np.minimum(ctx.cfl_dt(probe, u64, CFL), ctx.cfl_dt(probe, t64, CFL))
    del t64
    stream = torch.cuda.current_stream()
    out = {"rows": rows, "n": n, "ckpt_stride": "ceil(sqrt(nsteps))"}
    for name, scheme, steps, fac in (("explicit", L.BURGERS_EXPLICIT, EXPLICIT_STEPS, 1.0),
                                     ("btcs", L.BURGERS_BTCS, BTCS_STEPS, BTCS_DT_FACTOR)):
        grads = {}
        rec = {"steps": steps}
        for dt_, tdt in ((F64, torch.float64), (F32, torch.float32)):
            b = Batch.from_ensemble(ens, dt0 * fac, steps, dt_)
            u0 = torch.tensor(ens.u0, dtype=tdt, device=dev)
            ut = torch.tensor(tgt.u0, dtype=tdt, device=dev)
            ctx.advance(scheme, b, ut)          # target: the next seed's run
            uT = u0.clone()
            ctx.advance(scheme, b, uT)          # warm
            uT = u0.clone()
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.advance(scheme, b, uT)
            z.record(stream)
            torch.cuda.synchronize()
            t_fwd = a.elapsed_time(z) / 1000.0
            gT = uT - ut
            gu0 = torch.empty_like(u0)
            gnu = torch.empty(rows, dtype=torch.float64, device=dev)
            ctx.adjoint(scheme, b, u0, gT, gu0, gnu)   # warm (workspace)
            a.record(stream)
            ctx.adjoint(scheme, b, u0, gT, gu0, gnu)
            z.record(stream)
            torch.cuda.synchronize()
            t_adj = a.elapsed_time(z) / 1000.0
            grads[dt_] = (gu0.double(), gnu.clone())
            k = math.ceil(math.sqrt(steps))
            nck = math.ceil(steps / k)
            # checkpoints (FP32: state + compensation term) and k + 1 segment states per row
            ck = ((2 * nck + k + 1) * 4 if dt_ == F32 else (nck + k + 1) * 8) * n * rows
            tag = "fp64" if dt_ == F64 else "fp32"
            rec[tag] = {"forward_cups": rows * n * steps / t_fwd,
                        "adjoint_s": t_adj, "forward_s": t_fwd, "adjoint_over_forward": t_adj / t_fwd,
                        "gradient_cups": rows * n * steps / t_adj,
                        "checkpoint_workspace_bytes": ck}
        g64, n64 = grads[F64]
        g32, n32 = grads[F32]
        gb = Batch.from_ensemble(ens, dt0 * fac, steps, F64)
        rel, _ = ctx.rel_l2(gb, g32, g64)
        a64 = g64.view(rows, n).abs().amax(dim=1).cpu().numpy()
        fin32 = torch.isfinite(g32.view(rows, n)).all(dim=1).cpu().numpy() & np.isfinite(n32.cpu().numpy())
        ok = fin32 & np.isfinite(a64) & np.isfinite(n64.cpu().numpy())
        dnu = ((n32 - n64).abs() / n64.abs()[torch.from_numpy(ok).to(dev)].max()).cpu().numpy()
        rec["grad_u0_fp64_row_absmax"] = {"max": float(np.max(a64)), "median": float(np.median(a64))}
        rec["rows_with_nonfinite_fp32_gradient"] = int(np.sum(~fin32))
        rec["grad_u0_fp32_vs_fp64_rel_l2"] = {"max": float(np.max(rel[ok])), "median": float(np.median(rel[ok])),
                                              "rows": int(np.sum(ok))}
        rec["grad_nu_fp32_vs_fp64_max_rel"] = float(np.max(dnu[ok]))
        # per-row bar: 1e-4, widened by the row's conditioning (the FP64 gradient's
        # change per unit trajectory deviation when u0 is rounded to FP32, times
        # the FP32 trajectory's deviation), 1e-2 where the FP32 trajectory takes
        # another upwind side than the FP64 one somewhere (another branch of the
        # piecewise smooth solution map)
        ur = u64.float().double()
        ut64 = torch.tensor(tgt.u0, dtype=torch.float64, device=dev)
        uT = ur.clone()
        ctx.advance(scheme, gb, uT)
        ctx.advance(scheme, gb, ut64)
        g64r = torch.empty_like(ur)
        ctx.adjoint(scheme, gb, ur, uT - ut64, g64r, torch.empty(rows, dtype=torch.float64, device=dev))
        stats = trajectory_stats(ctx, scheme, gb, u64, steps)
        bar = fp32_gradient_bar(g64.view(rows, n).cpu().numpy(), g64r.view(rows, n).cpu().numpy(), stats)
        del ur, ut64, uT, g64r
        flips = stats["flips"]
        above = ok & (rel > 1e-4)
        rec["grad_u0_fp32_vs_fp64_per_row_bar"] = {
            "rows_within_bar": int(np.sum(ok & (rel <= bar))), "rows": int(np.sum(ok)),
            "rows_above_1e-4": [{"row": int(b), "rel": float(rel[b]), "bar": float(bar[b]),
                                 "flips": int(flips[b])} for b in np.nonzero(above)[0]],
            "bar_max": float(np.max(bar[ok])), "bar_median": float(np.median(bar[ok])),
            "flip_free_rows": {"rows": int(np.sum(ok & (flips == 0))),
                               "max": float(np.max(rel[ok & (flips == 0)])),
                               "median": float(np.median(rel[ok & (flips == 0)]))},
            "note": ("bar = 1e-4 + 4 kappa dev32 (kappa: FP64 gradient change per unit trajectory "
                     "deviation under u0 -> fp32(u0); dev32: max |u32 - u64| over nodes and steps); "
                     "1e-2 where [u > 0] differs between the exact FP32 and FP64 trajectories "
                     "(flips)")}
        out[name] = rec
    out["note"] = ("gradient_cups = forward cell-updates of the problem per second of the adjoint call "
                   "(checkpoint recompute + reverse sweep); checkpoint workspace per row = ceil(steps/k) "
                   "checkpoints (FP32: state + compensation) + k + 1 segment states, k = ceil(sqrt(steps))")
    return out


def _tune_lines(ctx):
    """The context's tuning table as text lines ("key nt c k")."""
    import tempfile
    path = os.path.join(tempfile.mkdtemp(), "tune.txt")
    ctx.tune_save(path)
    with open(path) as f:
        return [ln for ln in f.read().splitlines() if ln and not ln.startswith("#")]


def short_rows_bench(dev, steps: int = 100):
    """Many short BTCS rows (periodic random-Fourier ensembles, 10x the CFL dt):
    the partitioned resident kernel and the per-thread Thomas kernel side by
    side, each forced through the tuning table of a context of its own, and
    the library's default choice; FP32 and FP64 throughput, each path's
    relative L2 difference to the default path of the same precision, and
    each path's FP32 result against its FP64 one, per row relative to the
    row's norm at t_final and to its initial norm (these rows decay by up to
    three orders of magnitude over the run, which inflates the first). Parity
    with the oracle at these shapes is a test."""
    import tempfile

    import torch

    from paper_2601_12204_b300 import _lib as L
    from paper_2601_12204_b300 import workloads as W
    from paper_2601_12204_b300.api import Batch, Context
    # (rows, n): the partitioned kernel's shape and the Thomas kernel's
    # (threads, layout mode) of that capacity class, per dtype
    part = {32: (32, 1), 64: (32, 2), 256: (32, 8), 512: (64, 8)}
    thomas = {(0, 32): (256, 2), (0, 64): (256, 0), (0, 256): (32, 2), (0, 512): (64, 1),
              (1, 32): (128, 0), (1, 64): (64, 1), (1, 256): (64, 1), (1, 512): (64, 1)}
    out = {"steps": steps, "dt": "10x CFL", "note": "cell-updates/s; default = the library's own "
           "choice (per-thread Thomas for classes of <= 64 FP32 / <= 128 FP64 nodes with >= 8192 rows)"}
    for rows, n in ((4096, 256), (16384, 512), (16384, 32), (65536, 64)):
        ens = W.fourier_ensemble(rows, n)
        rec = {}
        res = {}  # (path, dtype name) -> result, FP64 on the device
        u64 = torch.tensor(ens.u0, dtype=torch.float64, device=dev)
        c0 = Context(dev.index or 0)
        try:  # one dt per row for both precisions (from the FP64 state)
            dts = c0.cfl_dt(Batch.from_ensemble(ens, 1.0, 0, L.BURGERS_F64), u64, CFL) * BTCS_DT_FACTOR
        finally:
            c0.close()
        for dt_, tdt, name in ((L.BURGERS_F32, torch.float32, "fp32"), (L.BURGERS_F64, torch.float64, "fp64")):
            u0 = torch.tensor(ens.u0, dtype=tdt, device=dev)
            r = {}
            wdef = None
            for path in ("default", "partitioned", "thomas"):
                ctx = Context(dev.index or 0)
                try:
                    if path != "default":
                        key = lambda ex: (2 << 56) ^ (dt_ << 52) ^ (ex << 48) ^ n  # noqa: E731
                        nt, c, k = ((*part[n], 0) if path == "partitioned"
                                    else (thomas[(dt_, n)][0], n, 1 + thomas[(dt_, n)][1]))
                        p = os.path.join(tempfile.mkdtemp(), "t.txt")
                        with open(p, "w") as f:
                            f.write(f"# forced\n{key(0)} {nt} {c} {k}\n{key(1)} {nt} {c} {k}\n")
                        ctx.tune_load(p)
                    b = Batch.from_ensemble(ens, dts, steps, dt_)
                    ts = []
                    for _ in range(8):  # the first two build the plan and warm the clocks
                        w = u0.clone()
                        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        a.record()
                        ctx.btcs_advance(b, w)
                        z.record()
                        torch.cuda.synchronize()
                        ts.append(a.elapsed_time(z) / 1e3)
                    cups = rows * n * steps / min(ts[2:])
                    w2 = w.double().view(rows, n)
                    if wdef is None:
                        wdef = w2
                    d = (torch.linalg.vector_norm(w2 - wdef, dim=1) /
                         torch.linalg.vector_norm(wdef, dim=1))
                    r[path] = {"cups": cups, "l2_vs_default_max": float(d.max())}
                    res[(path, name)] = w2
                finally:
                    ctx.close()
            rec[name] = r
            del u0
            del wdef
        n0 = torch.linalg.vector_norm(u64.view(rows, n), dim=1)
        for path in ("default", "partitioned", "thomas"):
            w32, w64 = res[(path, "fp32")], res[(path, "fp64")]
            e = torch.linalg.vector_norm(w32 - w64, dim=1)
            rt = e / torch.linalg.vector_norm(w64, dim=1)
            r0 = e / n0
            rec["fp32"][path]["fp32_vs_fp64"] = {
                "max_rel_final": float(rt.max()), "median_rel_final": float(rt.median()),
                "max_rel_initial": float(r0.max())}
        del res, u64
        out[f"{rows}x{n}"] = rec
    return out


def step_ic_bench(ctx, dev, rows: int = 4096, n: int = 4096):
    """Step-IC shock workload (Eq. 20, Sec. 3.4): `rows` Dirichlet rows of n
    nodes on [0, 1] from u0 = 1 left of x = 1/2 and 0 right of it (u(0) = 1,
    u(1) = 0 held), nu log-uniform in [1e-5, 1e-3]; 2000 explicit steps at
    the CFL-0.4 step and 200 BTCS steps at dt = 5 dx / u_max (u_max = 1).
    FP32 throughput and FP32 against the FP64 GPU path on every row (parity
    with the oracle on this workload is a test)."""
    import torch

    from paper_2601_12204_b300 import _lib as L
    from paper_2601_12204_b300 import workloads as W
    from paper_2601_12204_b300.api import Batch
    F32, F64 = L.BURGERS_F32, L.BURGERS_F64
    ens = W.step_ensemble(rows, n)
    stream = torch.cuda.current_stream(dev)
    u32 = torch.tensor(ens.u0, dtype=torch.float32, device=dev)
    u64 = torch.tensor(ens.u0, dtype=torch.float64, device=dev)
    dte = ctx.cfl_dt(Batch.from_ensemble(ens, 1.0, 0, F64), u64, CFL)
    out = {"rows": rows, "n": n, "bc": "Dirichlet u(0)=1, u(1)=0", "nu": "log-U[1e-5,1e-3]"}
    for name, scheme, steps, dts in (("explicit", L.BURGERS_EXPLICIT, EXPLICIT_STEPS, dte),
                                     ("btcs", L.BURGERS_BTCS, BTCS_STEPS, 5.0 * ens.dxs / 1.0)):
        b32 = Batch.from_ensemble(ens, dts, steps, F32)
        b64 = b32.with_fields(dtype=F64)
        w = u32.clone()
        ctx.advance(scheme, b32, w)  # warm
        w.copy_(u32)
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.advance(scheme, b32, w)
        z.record(stream)
        w64 = u64.clone()
        ctx.advance(scheme, b64, w64)
        torch.cuda.synchronize()
        t = a.elapsed_time(z) / 1000.0
        rel, _ = ctx.rel_l2(b32, w, w64)
        out[name] = {"steps": steps, "cups": rows * n * steps / t,
                     "dt": "CFL 0.4" if scheme == L.BURGERS_EXPLICIT else "5 dx / u_max",
                     "l2_fp32_vs_fp64": {"max": float(np.max(rel)), "median": float(np.median(rel))},
                     "range": [float(w.min()), float(w.max())]}
        del w, w64
    return out


def ragged_bench(ctx, dev):
    """Ragged batches (row lengths log-uniform, periodic and Dirichlet mixed,
    random-Fourier u0, nu log-uniform in [1e-3, 1e-1]): 4096 resident rows of
    1025-8192 nodes (500 explicit steps at the CFL-0.4 step, 100 BTCS steps at
    10x it) and 512 cluster rows of 8193-65536 nodes (100 BTCS steps). FP32
    throughput and FP32 against the FP64 GPU path on every row."""
    import torch

    from paper_2601_12204_b300 import _lib as L
    from paper_2601_12204_b300 import workloads as W
    from paper_2601_12204_b300.api import Batch
    F32, F64 = L.BURGERS_F32, L.BURGERS_F64
    stream = torch.cuda.current_stream(dev)
    out = {"note": "cell-updates/s; rows of every length of the range, so nearly all ragged"}
    sets = (("resident", 4096, 1025, 8192, (("explicit", L.BURGERS_EXPLICIT, 500, 1.0),
                                              ("btcs", L.BURGERS_BTCS, 100, BTCS_DT_FACTOR))),
            ("cluster", 512, 8193, 65536, (("btcs", L.BURGERS_BTCS, 100, BTCS_DT_FACTOR),)))
    for name, rows, nmin, nmax, runs in sets:
        ens = W.mixed_ensemble(rows, nmin, nmax, seed=W.DEFAULT_SEED + 7)
        u32 = torch.tensor(ens.u0, dtype=torch.float32, device=dev)
        u64 = torch.tensor(ens.u0, dtype=torch.float64, device=dev)
        dt0 = ctx.cfl_dt(Batch.from_ensemble(ens, 1.0, 0, F64), u64, CFL)
        cells = float(np.sum(ens.ns))
        res = {"rows": rows, "n": [nmin, nmax], "nodes": int(cells)}
        for sname, scheme, steps, fac in runs:
            b32 = Batch.from_ensemble(ens, dt0 * fac, steps, F32)
            b64 = b32.with_fields(dtype=F64)
            w = u32.clone()
            ctx.advance(scheme, b32, w)  # warm
            ts = []
            for _ in range(3):
                w.copy_(u32)
                a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                ctx.advance(scheme, b32, w)
                z.record(stream)
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(z) / 1000.0)
            w64 = u64.clone()
            ctx.advance(scheme, b64, w64)
            torch.cuda.synchronize()
            rel, _ = ctx.rel_l2(b32, w, w64)
            res[sname] = {"steps": steps, "cups": cells * steps / min(ts),
                          "l2_fp32_vs_fp64": {"max": float(np.max(rel)),
                                              "median": float(np.median(rel))}}
            del w, w64
        out[name] = res
        del u32, u64
    return out


def extras(args, ctx, ens, u0, batches, probe, dev, world, rank):
    import torch

    from paper_2601_12204_b300 import _lib as L
    from paper_2601_12204_b300 import workloads as W
    from paper_2601_12204_b300.api import Batch
    F32, F64 = L.BURGERS_F32, L.BURGERS_F64
    out = {}
    stream = torch.cuda.current_stream(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    dt0 = ctx.cfl_dt(probe, u0, CFL)
    be, bb = batches(dt0)

    # ---- FP32 error per result against the FP64 path, and FP64 throughput
    u64 = torch.tensor(ens.u0, dtype=torch.float64, device=dev)
    r32e = u0.clone()
    ctx.explicit_advance(be, r32e)
    r32b = u0.clone()
    ctx.btcs_advance(bb, r32b)
    acc = {}
    fp64 = {}
    for name, b32, r32, steps in (("explicit", be, r32e, EXPLICIT_STEPS), ("btcs", bb, r32b, BTCS_STEPS)):
        b64 = b32.with_fields(dtype=F64)
        r64 = u64.clone()
        a, z = ev(), ev()
        a.record(stream)
        ctx.advance(L.BURGERS_EXPLICIT if name == "explicit" else L.BURGERS_BTCS, b64, r64)
        z.record(stream)
        torch.cuda.synchronize()
        fp64[name + "_cups"] = B_ROWS * N_NODES * steps / (a.elapsed_time(z) / 1000.0)
        rel, _ = ctx.rel_l2(b32, r32, r64)
        acc[name] = {"max": float(np.max(rel)), "median": float(np.median(rel))}
    acc["bound"] = 1e-5
    out["l2_fp32_vs_fp64"] = acc
    # FP64 explicit against the measured FP64 FMA rate: 6 FP64 operations per
    # cell-update (two differences, |u| - u, p, q and the two-FMA update into u)
    f64pk = ctx.fma_peak(L.BURGERS_F64) / 1e12
    fp64["explicit_roofline"] = {"bound": "fp64", "achieved": 6.0 * fp64["explicit_cups"] / 1e12,
                                 "peak_measured": f64pk, "unit": "T FP64 lane-instr/s",
                                 "frac": 6.0 * fp64["explicit_cups"] / 1e12 / f64pk}
    out["fp64"] = fp64
    del u64

    # ---- RK4 (Eq. 22) on the same ensemble and dt: throughput, roofline of the
    # resident kernel, FP32 against FP64
    br = Batch.from_ensemble(ens, dt0, RK4_STEPS, F32)
    ctx.autotune(L.BURGERS_RK4, br, u0, probe_steps=50)
    w = u0.clone()
    ctx.rk4_advance(br, w)  # warm
    torch.cuda.synchronize()
    w.copy_(u0)
    a, z = ev(), ev()
    a.record(stream)
    ctx.rk4_advance(br, w)
    z.record(stream)
    torch.cuda.synchronize()
    t_rk = a.elapsed_time(z) / 1000.0
    w64 = torch.tensor(ens.u0, dtype=torch.float64, device=dev)
    a, z = ev(), ev()
    a.record(stream)
    ctx.rk4_advance(br.with_fields(dtype=F64), w64)
    z.record(stream)
    torch.cuda.synchronize()
    t_rk64 = a.elapsed_time(z) / 1000.0
    rel, _ = ctx.rel_l2(br, w, w64)
    cells = float(B_ROWS) * N_NODES * RK4_STEPS
    ach = RK4_OPS * cells / t_rk / 1e12
    peak_ops = ctx.get(L.BURGERS_INFO_SM_COUNT) * FP32_LANES * 2032e6 / 1e12
    out["rk4"] = {"steps": RK4_STEPS, "cups": cells / t_rk, "fp64_cups": cells / t_rk64,
                  "l2_fp32_vs_fp64": {"max": float(np.max(rel)), "median": float(np.median(rel))},
                  "roofline": {"bound": "alu", "kernel": "k_explicit_resident<float, tuned shape, "
                                                          "exact, RK4>",
                               "achieved": ach, "peak": peak_ops,
                               "unit": "Tops/s (FP32 lane-instructions)",
                               "frac": ach / peak_ops,
                               "per_unit": f"{RK4_OPS:.4g} FMA-pipe FP32 lane-operations per "
                                           "cell-update (packed f32x2 pairs) + 8 min/max on the ALU pipe"}}
    del w, w64

    # ---- further implicit schemes on the same ensemble (resident kernel
    # variants): Crank-Nicolson and 3 Picard iterations at the BTCS dt; 3
    # Newton iterations (central convection, Eq. 11) at the explicit dt on
    # rows whose viscosity is raised to keep the cell Peclet number <= 1.5
    # (central convection needs a resolved grid). FP32 against FP64 each.
    ens_n = ens.subset(np.arange(ens.count))
    for bb_ in range(ens_n.count):
        peak = float(np.max(np.abs(ens_n.row(bb_))))
        ens_n.nus[bb_] = max(ens_n.nus[bb_], peak * ens_n.dxs[bb_] / 1.5)
    variants = {}
    for name, scheme, iters, batch32 in (
            ("cn", L.BURGERS_CN, 1, Batch.from_ensemble(ens, dt0 * BTCS_DT_FACTOR, BTCS_STEPS, F32)),
            ("picard3", L.BURGERS_PICARD, 3,
             Batch.from_ensemble(ens, dt0 * BTCS_DT_FACTOR, BTCS_STEPS, F32)),
            ("newton3", L.BURGERS_NEWTON, 3, Batch.from_ensemble(ens_n, dt0, BTCS_STEPS, F32))):
        ctx.autotune(scheme, batch32, u0, probe_steps=20)
        w = u0.clone()
        ctx.advance(scheme, batch32, w, iters=iters)  # warm
        torch.cuda.synchronize()
        w.copy_(u0)
        a, z = ev(), ev()
        a.record(stream)
        ctx.advance(scheme, batch32, w, iters=iters)
        z.record(stream)
        torch.cuda.synchronize()
        t32 = a.elapsed_time(z) / 1000.0
        w64 = torch.tensor(ens.u0, dtype=torch.float64, device=dev)
        a, z = ev(), ev()
        a.record(stream)
        ctx.advance(scheme, batch32.with_fields(dtype=F64), w64, iters=iters)
        z.record(stream)
        torch.cuda.synchronize()
        t64 = a.elapsed_time(z) / 1000.0
        rel, _ = ctx.rel_l2(batch32, w, w64)
        cells = float(B_ROWS) * N_NODES * BTCS_STEPS
        variants[name] = {"iters": iters, "steps": BTCS_STEPS, "cups": cells / t32,
                          "fp64_cups": cells / t64,
                          "l2_fp32_vs_fp64": {"max": float(np.max(rel)),
                                              "median": float(np.median(rel))}}
        del w, w64
    variants["note"] = ("cell-updates/s counts one node advanced one step whatever the "
                        "iterations per step; CN and Picard at 10x the CFL dt, Newton at the "
                        "CFL dt on viscosity-raised rows (cell Peclet <= 1.5)")
    out["implicit_variants"] = variants
    out["implicit_variants_long"] = long_variants_bench(ctx, dev)
    out["differentiation"] = differentiation_bench(ctx, dev)
    out["step_ic"] = step_ic_bench(ctx, dev)
    out["short_rows_btcs"] = short_rows_bench(dev)
    out["ragged"] = ragged_bench(ctx, dev)

    # ---- plain one-row-per-launch path on a subset, same kernels
    P = 64
    sub = Batch(F32, ens.offsets[:P], N_NODES, 0, ens.dxs[:P], ens.nus[:P], dt0[:P], EXPLICIT_STEPS)
    subb = Batch(F32, ens.offsets[:P], N_NODES, 0, ens.dxs[:P], ens.nus[:P],
                 dt0[:P] * BTCS_DT_FACTOR, BTCS_STEPS)
    ctx.set(L.BURGERS_OPT_PLAIN, 1)
    w = u0.clone()
    ctx.explicit_advance(sub, w)
    ctx.btcs_advance(subb, w)
    torch.cuda.synchronize()
    a, m, z = ev(), ev(), ev()
    a.record(stream)
    ctx.explicit_advance(sub, w)
    m.record(stream)
    ctx.btcs_advance(subb, w)
    z.record(stream)
    torch.cuda.synchronize()
    ctx.set(L.BURGERS_OPT_PLAIN, 0)
    te, tb = a.elapsed_time(m) / 1000.0, m.elapsed_time(z) / 1000.0
    out["plain"] = {"rows": P, "explicit_cups": P * N_NODES * EXPLICIT_STEPS / te,
                    "btcs_cups": P * N_NODES * BTCS_STEPS / tb,
                    "value": P * N_NODES * (EXPLICIT_STEPS + BTCS_STEPS) / (te + tb),
                    "note": "one kernel launch per row (1 CTA), same kernels, sequential on one stream"}

    # ---- e2e through host memory (pinned): H2D inputs + D2H results every step
    hu0 = torch.from_numpy(ens.u0.astype(np.float32)).pin_memory()
    ha = torch.empty_like(hu0).pin_memory()
    hb = torch.empty_like(hu0).pin_memory()
    times = []
    for i in range(1 + min(3, args.steps)):
        ha.copy_(hu0)
        hb.copy_(hu0)
        t0 = time.perf_counter()
        ctx.solve_host(L.BURGERS_EXPLICIT, be, ha)
        ctx.solve_host(L.BURGERS_BTCS, bb, hb)
        t1 = time.perf_counter()
        if i > 0:
            times.append(t1 - t0)
    e2e_t = allreduce_max(statistics.median(times), world)
    out["e2e"] = {"value": CELLS_PER_STEP * world / e2e_t, "unit": "cell-updates/s",
                  "h2d_bytes_per_step": 2 * hu0.numel() * 4, "d2h_bytes_per_step": 2 * hu0.numel() * 4,
                  "note": "burgers_solve_host (explicit) + burgers_solve_host (BTCS) from pinned host "
                          "buffers; dt from the device CFL reduction of the same inputs"}
    del ha, hb, hu0

    out["large_grid"] = large_grid_bench(ctx, dev)
    out["adjoint_long"] = long_adjoint_bench(ctx, dev)
    return out


def long_variants_bench(ctx, dev, rows: int = 512, n: int = 32768, steps: int = 40):
    """Implicit variants on rows longer than the resident capacity: `rows`
    periodic random-Fourier rows of n nodes. Crank-Nicolson and 3 Picard
    iterations at 10x the CFL dt, and 3 Newton iterations at the CFL dt on
    viscosity-raised rows (cell Peclet <= 1.5), by the default routing (FP32:
    the cluster-resident kernel) and through the multi-level solver (cluster
    off); lagged BTCS through the multi-level solver and by the default
    routing for comparison. FP32 and FP64
    throughput, FP32 against FP64 on every row."""
    import torch

    from paper_2601_12204_b300 import _lib as L
    from paper_2601_12204_b300 import workloads as W
    from paper_2601_12204_b300.api import Batch
    F32, F64 = L.BURGERS_F32, L.BURGERS_F64
    stream = torch.cuda.current_stream(dev)
    ens = W.fourier_ensemble(rows, n, seed=1234)
    ens_n = ens.subset(np.arange(ens.count))
    for b in range(ens_n.count):
        peak = float(np.max(np.abs(ens_n.row(b))))
        ens_n.nus[b] = max(ens_n.nus[b], peak * ens_n.dxs[b] / 1.5)
    u32 = torch.tensor(ens.u0, dtype=torch.float32, device=dev)
    u64 = torch.tensor(ens.u0, dtype=torch.float64, device=dev)
    dt0 = ctx.cfl_dt(Batch.from_ensemble(ens, 1.0, 0, F64), u64, CFL)
    cells = float(rows) * n * steps
    out = {"rows": rows, "n": n, "steps": steps, "bc": "periodic",
           "note": "cell-updates/s counts one node advanced one step whatever the iterations"}

    def timed(scheme, b, src, iters):
        w = src.clone()
        ctx.advance(scheme, b, w, iters=iters)  # builds the plan, warms
        ts = []
        for _ in range(3):
            w.copy_(src)
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.advance(scheme, b, w, iters=iters)
            z.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(z) / 1000.0)
        return w, min(ts)

    cases = (("cn", L.BURGERS_CN, 1, ens, BTCS_DT_FACTOR, 1),
             ("cn_multilevel", L.BURGERS_CN, 1, ens, BTCS_DT_FACTOR, 0),
             ("picard3", L.BURGERS_PICARD, 3, ens, BTCS_DT_FACTOR, 1),
             ("picard3_multilevel", L.BURGERS_PICARD, 3, ens, BTCS_DT_FACTOR, 0),
             ("newton3", L.BURGERS_NEWTON, 3, ens_n, 1.0, 1),
             ("newton3_multilevel", L.BURGERS_NEWTON, 3, ens_n, 1.0, 0),
             ("btcs_multilevel", L.BURGERS_BTCS, 1, ens, BTCS_DT_FACTOR, 0),
             ("btcs_default", L.BURGERS_BTCS, 1, ens, BTCS_DT_FACTOR, 1))
    for name, scheme, iters, e, fac, cluster in cases:
        ctx.set(L.BURGERS_OPT_CLUSTER, cluster)
        try:
            b32 = Batch.from_ensemble(e, dt0 * fac, steps, F32)
            b64 = b32.with_fields(dtype=F64)
            w32, t32 = timed(scheme, b32, u32, iters)
            w64, t64 = timed(scheme, b64, u64, iters)
        finally:
            ctx.set(L.BURGERS_OPT_CLUSTER, 1)
        rel, _ = ctx.rel_l2(b32, w32, w64)
        out[name] = {"iters": iters, "dt": f"{fac:g}x CFL", "cups": cells / t32,
                     "fp64_cups": cells / t64,
                     "l2_fp32_vs_fp64": {"max": float(np.max(rel)), "median": float(np.median(rel))}}
        del w32, w64
    del u32, u64
    return out


def long_adjoint_bench(ctx, dev, rows: int = 64, n: int = 65536):
    """Gradients by the long-row adjoint: `rows` periodic random-Fourier rows
    of n nodes (longer than one CTA holds), explicit 200 steps at the CFL
    step and BTCS 20 steps at 10x it, FP32 and FP64; forward cell-updates per
    second of the adjoint call (checkpointed forward, segment recompute and
    reverse sweep) and the forward's own rate for comparison. FP32 dJ/du0
    against FP64 per row."""
    import torch

    from paper_2601_12204_b300 import _lib as L
    from paper_2601_12204_b300 import workloads as W
    from paper_2601_12204_b300.api import Batch
    F32, F64 = L.BURGERS_F32, L.BURGERS_F64
    stream = torch.cuda.current_stream(dev)
    ens = W.fourier_ensemble(rows, n, seed=4242)
    u64 = torch.tensor(ens.u0, dtype=torch.float64, device=dev)
    dt0 = ctx.cfl_dt(Batch.from_ensemble(ens, 1.0, 0, F64), u64, CFL)
    out = {"rows": rows, "n": n, "bc": "periodic"}
    for name, scheme, steps, fac in (("explicit", L.BURGERS_EXPLICIT, 200, 1.0),
                                     ("btcs", L.BURGERS_BTCS, 20, BTCS_DT_FACTOR)):
        rec = {"steps": steps}
        grads = {}
        for dn, dt_, tdt in (("fp32", F32, torch.float32), ("fp64", F64, torch.float64)):
            b = Batch.from_ensemble(ens, dt0 * fac, steps, dt_)
            u0 = u64.to(tdt)
            w = u0.clone()
            ctx.advance(scheme, b, w)  # dJ/du(T) = u(T): J = |u(T)|^2 / 2
            gT = w.clone()
            gu0 = torch.empty_like(u0)
            gnu = torch.zeros(rows, dtype=torch.float64, device=dev)
            ctx.adjoint(scheme, b, u0, gT, gu0, gnu)  # warm: workspace, plans
            torch.cuda.synchronize()
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.adjoint(scheme, b, u0, gT, gu0, gnu)
            z.record(stream)
            torch.cuda.synchronize()
            t_adj = a.elapsed_time(z) / 1e3
            w.copy_(u0)
            a.record(stream)
            ctx.advance(scheme, b, w)
            z.record(stream)
            torch.cuda.synchronize()
            t_fwd = a.elapsed_time(z) / 1e3
            cells = float(rows) * n * steps
            rec[dn] = {"gradient_cups": cells / t_adj, "forward_cups": cells / t_fwd,
                       "adjoint_over_forward": t_adj / t_fwd}
            grads[dn] = gu0.double().view(rows, n)
        d = (torch.linalg.vector_norm(grads["fp32"] - grads["fp64"], dim=1) /
             torch.linalg.vector_norm(grads["fp64"], dim=1))
        rec["grad_u0_fp32_vs_fp64_rel_l2"] = {"max": float(d.max()), "median": float(d.median())}
        out[name] = rec
    out["note"] = ("rows longer than one CTA: explicit one step per pass over tiles, BTCS one "
                   "step per call and transposed solves through the multi-level solver; "
                   "checkpoints every ceil(sqrt(steps)) steps")
    return out


def large_grid_bench(ctx, dev):
    """Large single grid (N = 2^24, periodic, sin x + 0.5 + noise, nu = 1e-3):
    the temporally blocked streaming explicit solve (10000 steps), the
    one-step-per-pass kernel (K = 1) against the HBM roofline, and the
    multi-level BTCS solve (100 steps at 10x dt); FP32 against FP64."""
    import torch

    from paper_2601_12204_b300 import _lib as L
    from paper_2601_12204_b300 import workloads as W
    from paper_2601_12204_b300.api import Batch
    F32, F64 = L.BURGERS_F32, L.BURGERS_F64
    stream = torch.cuda.current_stream(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    lg = W.large_grid(1 << 24)
    nlg = float(lg.ns[0])
    ul = torch.tensor(lg.u0, dtype=torch.float32, device=dev)
    ul64 = torch.tensor(lg.u0, dtype=torch.float64, device=dev)
    pb = Batch.from_ensemble(lg, 1.0, 0, F32)
    dtl = ctx.cfl_dt(pb, ul, CFL)
    large = {}

    def timed(scheme, batch, src):
        w = src.clone()
        adv = ctx.explicit_advance if scheme == L.BURGERS_EXPLICIT else ctx.btcs_advance
        adv(batch, w)  # warm (plan, graph capture)
        torch.cuda.synchronize()
        w.copy_(src)
        a, z = ev(), ev()
        a.record(stream)
        adv(batch, w)
        z.record(stream)
        torch.cuda.synchronize()
        return w, a.elapsed_time(z) / 1000.0

    peak, src = hbm_peak()
    issue_cups = ctx.get(L.BURGERS_INFO_SM_COUNT) * FP32_LANES * 2032e6 / ALG_EXPLICIT_OPS
    for K, steps in ((0, LARGE_EXPLICIT_STEPS), (1, 200), (1, LARGE_EXPLICIT_STEPS)):
        ctx.set(L.BURGERS_OPT_STREAM_K, K)
        b32 = Batch.from_ensemble(lg, dtl, steps, F32)
        w, t = timed(L.BURGERS_EXPLICIT, b32, ul)
        cups = nlg * steps / t
        if K == 0:
            kt = ctx.get(L.BURGERS_OPT_STREAM_K)  # 0: the tuned K
            large["explicit_cups"] = cups
            large["explicit_steps"] = steps
            w64, t64 = timed(L.BURGERS_EXPLICIT, Batch.from_ensemble(lg, dtl, steps, F64), ul64)
            large["explicit_fp64_cups"] = nlg * steps / t64
            rel, _ = ctx.rel_l2(b32, w, w64)
            large["explicit_l2_fp32_vs_fp64"] = float(rel[0])
            del w64
        elif steps == 200:
            # the method's traffic: 4 bytes of u read and 4 written per cell-update
            large["stream_k1_cups"] = cups
            large["stream_k1_gbs_algorithmic"] = 8.0 * cups / 1e9
            large["stream_k1_hbm_frac_algorithmic"] = 8.0 * cups / 1e9 / peak
            large["stream_k1_gbs_moved"] = 10.0 * cups / 1e9
            large["stream_k1_hbm_frac_moved"] = 10.0 * cups / 1e9 / peak
            large["stream_k1_peak"] = {"gbs": peak, "source": src}
        else:
            # K = 1 for the whole run: FP32 against FP64 after 10000 single-step passes
            w64, _ = timed(L.BURGERS_EXPLICIT, Batch.from_ensemble(lg, dtl, steps, F64), ul64)
            rel, _ = ctx.rel_l2(b32, w, w64)
            large["stream_k1_10000_steps"] = {"cups": cups, "l2_fp32_vs_fp64": float(rel[0])}
            del w64
    ctx.set(L.BURGERS_OPT_STREAM_K, 0)
    # the temporally blocked run against min(HBM x K / 8 B, FP32 issue / 9 ops):
    # K from the tuning table's streaming entry if there is one, else the
    # library's default for FP32 forward-Euler windows (8192 nodes; 128 steps
    # per pass on rows of 32 windows or more, else 64)
    kb = 128 if nlg >= 32 * 8192 else 64
    for line in _tune_lines(ctx):
        key, nt, c, k = (int(x) for x in line.split())
        if key >> 56 == 1 and (key >> 52) & 0xF == 0 and k > 0:  # K_EXPLICIT_STREAM, FP32
            kb = min(k, nt * c // 4)
    bound = min(peak * 1e9 * kb / 8.0, issue_cups)
    large["blocked"] = {"K": kb, "cups": large["explicit_cups"], "bound_cups": bound,
                        "frac": large["explicit_cups"] / bound,
                        "bound": "hbm" if peak * 1e9 * kb / 8.0 < issue_cups else "alu",
                        "note": "bound = min(HBM x K / 8 B, SMs x 128 FP32 lanes x 2032 MHz / 9 ops)"}
    bl32 = Batch.from_ensemble(lg, dtl * BTCS_DT_FACTOR, LARGE_BTCS_STEPS, F32)
    bl64 = Batch.from_ensemble(lg, dtl * BTCS_DT_FACTOR, LARGE_BTCS_STEPS, F64)
    w, t = timed(L.BURGERS_BTCS, bl32, ul)
    w64, t64 = timed(L.BURGERS_BTCS, bl64, ul64)
    rel, _ = ctx.rel_l2(bl32, w, w64)
    large["btcs_cups"] = nlg * LARGE_BTCS_STEPS / t
    large["btcs_fp64_cups"] = nlg * LARGE_BTCS_STEPS / t64
    large["btcs_steps"] = LARGE_BTCS_STEPS
    large["btcs_l2_fp32_vs_fp64"] = float(rel[0])
    del w64
    large["note"] = ("N=2^24 periodic, nu=1e-3. Explicit: K=0 tuned temporal blocking, "
                     "K=1 one step per HBM pass (k_explicit_step1): algorithmic 8 B per "
                     "cell-update (u read and written once), moved 10 B (plus the 1-byte FP32 "
                     "compensation term each way), against the HBM copy bandwidth. BTCS at 10x dt "
                     "through the multi-level partitioned solver. l2 = per-row relative L2 of "
                     "FP32 against FP64")
    del ul, ul64, w
    return large


def serve_bench(ctx, dev, duration: float, rate: float = 20000.0, plain_seconds: float = 5.0):
    """Serving workload: Poisson arrivals at `rate` for `duration` s of mixed
    requests through the continuous-batching server; latency = done - submit
    on the server clock. Also the plain path: the same trace served one
    request per launch, in arrival order, for at most `plain_seconds`."""
    import torch

    from paper_2601_12204_b300 import _lib as L
    from paper_2601_12204_b300 import workloads as W
    from paper_2601_12204_b300.api import Batch, Server

    t0 = time.perf_counter()
    trace = W.serving_trace(rate=rate, duration=duration, with_u0=False)
    u0d, offs = W.fourier_rows_torch(trace, dev, torch.float32)
    ns = np.array([q.n for q in trace])
    probe = Batch(L.BURGERS_F32, offs, ns, [q.bc for q in trace], [q.dx for q in trace],
                  [q.nu for q in trace], 1.0, 0)
    dt0 = ctx.cfl_dt(probe, u0d, CFL)
    dts = np.where(np.array([q.scheme for q in trace]) == L.BURGERS_BTCS, BTCS_DT_FACTOR, 1.0) * dt0
    host = u0d.cpu().pin_memory()
    base = host.data_ptr()
    del u0d
    log(f"serving trace: {len(trace)} requests generated in {time.perf_counter() - t0:.1f} s")
    cells = ns.astype(np.float64) * np.array([q.nsteps for q in trace])

    sv = Server(ctx, L.BURGERS_F32, slice_steps=256)
    # warm-up: a handful of requests of each kind
    for q, o, dt in list(zip(trace, offs, dts))[:32]:
        t = sv._submit_ptr(q.scheme, q.bc, q.n, base + 4 * int(o), q.dx, q.nu, dt, 50)
        sv.wait(t, q.n, timeout_s=60)
    import threading
    done = {}
    lock = threading.Lock()
    finished = threading.Event()

    def collector(expected):
        got = 0
        deadline = time.perf_counter() + duration + 600
        while got < expected and time.perf_counter() < deadline:
            tk = sv.wait_any(1.0)
            if tk is None:
                continue
            rc, st = sv.poll_stats(tk)  # the timings only: no copy of the result
            with lock:
                done[tk] = (rc, st.t_submit, st.t_admit, st.t_done)
            got += 1
        finished.set()

    lag = {}
    order = []
    th = threading.Thread(target=collector, args=(len(trace),), daemon=True)
    # the client replays the trace from native code (burgers_serve_submit_timed:
    # no interpreter between the arrivals and the server), and no cyclic
    # garbage collection runs in this process while it does
    reqs = (L.burgers_request * len(trace))()
    for i, (q, o, dt) in enumerate(zip(trace, offs, dts)):
        reqs[i] = L.burgers_request(int(q.scheme), int(q.bc), int(q.n), 0, float(q.dx),
                                    float(q.nu), float(dt), int(q.nsteps), base + 4 * int(o))
    t_arr = np.array([q.t_arrive for q in trace], dtype=np.float64)
    import gc
    gc.collect()
    gc.freeze()
    gc.disable()
    th.start()
    tickets, late_s = sv.submit_timed(reqs, t_arr)
    # how late each request reached the server against its arrival time
    for tk, lt in zip(tickets.tolist(), late_s.tolist()):
        lag[tk] = lt
        order.append(tk)
    late = float(late_s.max()) if len(late_s) else 0.0
    finished.wait(duration + 600)
    gc.enable()
    gc.unfreeze()
    stats = sv.stats()
    sv.close()
    # latency from the request's scheduled arrival: server time from submission
    # to completion plus the submission's lateness, so a client that falls
    # behind the trace cannot hide queueing time
    lat = np.array([done[t][3] - done[t][1] + lag[t] for t in order if t in done and done[t][0] == 0])
    arr = np.array([q.t_arrive for q, t in zip(trace, order) if t in done and done[t][0] == 0])
    t_first = min(done[t][1] for t in order if t in done)
    t_last = max(done[t][3] for t in order if t in done)
    ok = [i for i, t in enumerate(order) if t in done and done[t][0] == 0]
    res = {"requests": len(trace), "completed": len(ok), "rate_req_s": rate,
           "trace_seconds": duration,
           "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
           "p999_ms": 1e3 * float(np.percentile(lat, 99.9)),
           "throughput_cups": float(cells[ok].sum()) / (t_last - t_first),
           "offered_cups": float(cells.sum()) / duration,
           "latency": "from each request's scheduled arrival: server time from submission to "
                      "completion plus the submission's lateness",
           "max_submit_lag_ms": 1e3 * late, "slices": stats["slices"],
           "active_max": stats["active_max"], "pool_bytes": stats["pool_bytes"],
           "pool_used_max": stats["pool_used_max"], "slice_steps": 256, "dtype": "f32",
           "worker_s": {"enqueue": stats["t_enqueue_s"], "slice_wait": stats["t_slice_s"],
                        "copies": stats["t_copy_s"]},
           # device time inside the slices and between them (the device idle
           # while the worker plans), against the server's wall time
           "device_s": {"in_slices": stats["t_gpu_s"], "between_slices": stats["t_gpu_gap_s"],
                        "wall": t_last - t_first},
           # whether the server keeps up: latency of the requests arriving in
           # the first and in the second half of the trace
           "p99_ms_by_half": [1e3 * float(np.percentile(h, 99)) if h.size else None
                              for h in (lat[arr < 0.5 * duration], lat[arr >= 0.5 * duration])]}
    if plain_seconds <= 0:
        return res
    # plain path: one request per launch, FIFO in arrival order
    ctx.set(L.BURGERS_OPT_PLAIN, 1)
    buf = torch.empty(int(ns.max()), dtype=torch.float32, device=dev)
    lat_p, t_end = [], None
    start = time.perf_counter()
    k = 0
    for q, o, dt in zip(trace, offs, dts):
        now = time.perf_counter() - start
        if now > plain_seconds:
            break
        if q.t_arrive > now:
            time.sleep(q.t_arrive - now)
        buf[:q.n].copy_(host[int(o):int(o) + q.n], non_blocking=False)
        b = Batch(L.BURGERS_F32, [0], [q.n], [q.bc], [q.dx], [q.nu], [dt], [q.nsteps])
        ctx.advance(q.scheme, b, buf)
        out = buf[:q.n].cpu()
        del out
        lat_p.append(time.perf_counter() - start - q.t_arrive)
        k += 1
    t_end = time.perf_counter() - start
    ctx.set(L.BURGERS_OPT_PLAIN, 0)
    # requests that had arrived but were still waiting when the plain run stopped
    backlog = [t_end - q.t_arrive for q in trace[k:] if q.t_arrive < t_end]
    allp = np.array(lat_p + backlog)
    res["plain"] = {"completed": k, "seconds": t_end, "backlog_at_stop": len(backlog),
                    "p50_ms_lower_bound": 1e3 * float(np.percentile(allp, 50)),
                    "p99_ms_lower_bound": 1e3 * float(np.percentile(allp, 99)),
                    "throughput_cups": float(cells[:k].sum()) / t_end,
                    "note": "same trace, one request per kernel launch in arrival order; waiting "
                            "requests at the stop count with their wait so far (lower bounds)"}
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--quick", action="store_true", help="skip the side measurements")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tune-file", default=None,
                    help="launch-shape table: loaded if it exists, else written after tuning")
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="length of the Poisson trace of the serving measurement (0 = skip); "
                         "the serving workload is 10 s of arrivals at 20k requests/s")
    ap.add_argument("--serve-rate", type=float, default=20000.0,
                    help="Poisson arrival rate of the serving measurement (requests/s)")
    ap.add_argument("--serve-only", action="store_true",
                    help="run only the serving measurement and print its JSON")
    ap.add_argument("--serve-plain-seconds", type=float, default=5.0,
                    help="time limit of the one-request-per-launch comparison path (0 = skip it)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.serve_only:
        import torch

        from paper_2601_12204_b300.api import Context
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        ctx = Context(0)
        print(json.dumps({"serve": serve_bench(ctx, dev, max(args.serve_seconds, 0.1), rate=args.serve_rate,
                                               plain_seconds=args.serve_plain_seconds)}), flush=True)
        ctx.close()
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
