"""Single-launch workload cases for kernel profiling (ncu) and quick timing.

    python -m paper_2601_12204_b300.cases --case explicit --rows 4096 --n 4096 --steps 200

Each case builds one seeded batch on the device, runs the CFL reduction, then
exactly one advance call of the named scheme (one resident kernel launch, or
the streaming / multi-level launch sequence for long rows), and prints its
CUDA-event time. The adjoint cases (adjoint-explicit, adjoint-btcs) time one
burgers_adjoint call instead (checkpointed forward recompute and reverse
sweep) on dJ/du(T) = u(T), after one untimed forward advance.
"""
from __future__ import annotations

import argparse
import json
import os
import tempfile

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", choices=["explicit", "btcs", "rk4", "adjoint-explicit", "adjoint-btcs"],
                    default="explicit")
    ap.add_argument("--rows", type=int, default=4096)
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--dtype", choices=["f32", "f64"], default="f32")
    ap.add_argument("--dt-factor", type=float, default=None)
    ap.add_argument("--large", action="store_true", help="one row: sin x + 0.5 + noise")
    ap.add_argument("--stream-k", type=int, default=0)
    ap.add_argument("--no-cluster", action="store_true",
                    help="long BTCS rows through the multi-level solver instead of clusters")
    ap.add_argument("--portable-clusters", action="store_true",
                    help="cluster-resident BTCS in clusters of at most 8 CTAs")
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--autotune", action="store_true", help="tune launch shapes first and print the table")
    ap.add_argument("--tune-file", default=None,
                    help="launch-shape table: loaded if it exists, else written after --autotune")
    ap.add_argument("--shape", default=None,
                    help="NTxC: force the resident kernel shape of rows of exactly NT*C nodes "
                         "(a one-entry tuning table), so a profile names its shape on the command line")
    a = ap.parse_args()

    import torch

    from . import _lib as L
    from . import workloads as W
    from .api import Batch, Context

    dt_code = L.BURGERS_F32 if a.dtype == "f32" else L.BURGERS_F64
    tdt = torch.float32 if a.dtype == "f32" else torch.float64
    ens = W.large_grid(a.n) if a.large else W.fourier_ensemble(a.rows, a.n)
    ctx = Context(0)
    if a.stream_k:
        ctx.set(L.BURGERS_OPT_STREAM_K, a.stream_k)
    if a.no_cluster:
        ctx.set(L.BURGERS_OPT_CLUSTER, 0)
    elif a.portable_clusters:
        ctx.set(L.BURGERS_OPT_CLUSTER, 2)
    u0 = torch.tensor(ens.u0, dtype=tdt, device="cuda")
    dt = ctx.cfl_dt(Batch.from_ensemble(ens, 1.0, 0, dt_code), u0, 0.4)
    btcs_like = a.case in ("btcs", "adjoint-btcs")
    fac = a.dt_factor if a.dt_factor is not None else (10.0 if btcs_like else 1.0)
    b = Batch.from_ensemble(ens, dt * fac, a.steps, dt_code)
    scheme = {"explicit": L.BURGERS_EXPLICIT, "btcs": L.BURGERS_BTCS, "rk4": L.BURGERS_RK4,
              "adjoint-explicit": L.BURGERS_EXPLICIT, "adjoint-btcs": L.BURGERS_BTCS}[a.case]
    adjoint = a.case.startswith("adjoint")
    if a.shape:
        nt, c = (int(v) for v in a.shape.lower().split("x"))
        if nt * c != a.n:
            raise SystemExit("--shape needs rows of exactly NT*C nodes")
        kind = {L.BURGERS_EXPLICIT: 0, L.BURGERS_BTCS: 2, L.BURGERS_RK4: 9}[scheme]
        key = (kind << 56) ^ (dt_code << 52) ^ (1 << 48) ^ a.n
        path = os.path.join(tempfile.mkdtemp(), "shape.txt")
        with open(path, "w") as f:
            f.write(f"# forced shape\n{key} {nt} {c} 0\n")
        ctx.tune_load(path)
    elif a.tune_file and os.path.exists(a.tune_file):
        ctx.tune_load(a.tune_file)
    elif a.autotune:
        ntuned = ctx.autotune(scheme, b, u0, probe_steps=min(a.steps, 100))
        path = a.tune_file or os.path.join(tempfile.mkdtemp(), "tune.txt")
        ctx.tune_save(path)
        print(json.dumps({"tuned_classes": ntuned, "table": open(path).read().splitlines()[1:]}))
    times = []
    if adjoint:
        gT = u0.clone()
        ctx.advance(scheme, b, gT)  # dJ/du(T) = u(T): J = |u(T)|^2 / 2
        gu0 = torch.empty_like(u0)
        gnu = torch.empty(ens.count, dtype=torch.float64, device="cuda")
    for _ in range(a.repeat):
        u = u0.clone()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        if adjoint:
            ctx.adjoint(scheme, b, u0, gT, gu0, gnu)
        else:
            ctx.advance(scheme, b, u)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    cells = float(np.sum(ens.ns)) * a.steps
    print(json.dumps({"case": a.case, "rows": int(ens.count), "n": int(ens.ns[0]),
                      "steps": a.steps, "dtype": a.dtype, "ms": times,
                      "cups": cells / (min(times) / 1e3)}))
    ctx.close()


if __name__ == "__main__":
    main()
