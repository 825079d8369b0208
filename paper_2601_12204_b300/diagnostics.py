"""Precision diagnostics of the FP32 path against the FP64 path, on the GPU.

The upwind side of the explicit and BTCS steps switches with the sign of the
node value (H(u) = [u > 0], Sec. 2.2), so the discrete solution map is only
piecewise smooth and its gradient jumps where a node value crosses zero.
Where an FP32 and an FP64 trajectory take a different side at some node and
step, their discrete gradients are those of different branches and may differ
by far more than FP32 rounding. Near forming shocks the map is smooth but
steep: rounding injected at every step moves the FP32 trajectory much further
from the FP64 one than the rounding of u0 alone would, and the gradient moves
with it. ``trajectory_stats`` measures both, per row, on the trajectories the
library's step kernels follow.
"""
from __future__ import annotations

import numpy as np

from . import _lib as L
from .api import Batch, Context


def trajectory_stats(ctx: Context, scheme: int, batch: Batch, u0, steps: int) -> dict:
    """Per row of `batch`, over the states u^k, k = 0 .. steps-1, that the steps
    of `scheme` (BURGERS_EXPLICIT or BURGERS_BTCS) read:

    flips:     number of (node i, step k) with [u_i^k > 0] different in the FP32
               and the FP64 trajectories from u0;
    dev32:     max |u32 - u64| over nodes and steps;
    dev_round: max |u64' - u64| over nodes and steps, u64' the FP64 trajectory
               from u0 rounded to FP32 (the deviation the rounding of the
               input alone causes).

    batch: the rows with their dt (its dtype and nsteps are ignored); u0: the
    initial state as a contiguous CUDA float64 tensor (the FP32 run starts from
    its rounding to FP32). The FP32 state after k steps is taken from a k-step
    launch: a launch's output is the state value its own steps k and later
    read, so this is the trajectory a single long launch follows. The FP64
    trajectories advance one step per launch (FP64 rows carry no split state,
    so this is bitwise the long launch). Returns numpy arrays."""
    import torch

    if scheme not in (L.BURGERS_EXPLICIT, L.BURGERS_BTCS):
        raise ValueError("trajectory_stats: explicit or BTCS only")
    dev = u0.device
    a = batch.arr
    rowid = torch.full((u0.numel(),), batch.count, dtype=torch.int64, device=dev)
    for b in range(batch.count):
        o, n = int(a["offset"][b]), int(a["n"][b])
        rowid[o:o + n] = b
    m = batch.count + 1
    flips = torch.zeros(m, dtype=torch.int64, device=dev)
    dev32 = torch.zeros(m, dtype=torch.float64, device=dev)
    devr = torch.zeros(m, dtype=torch.float64, device=dev)
    one64 = batch.with_fields(dtype=L.BURGERS_F64, nsteps=1)
    u64 = u0.detach().clone()
    u32_0 = u0.detach().float().contiguous()
    u64r = u32_0.double()
    for k in range(steps):
        v32 = u32_0.clone()
        if k > 0:
            ctx.advance(scheme, batch.with_fields(dtype=L.BURGERS_F32, nsteps=k), v32)
        flips.index_add_(0, rowid, ((v32 > 0) != (u64 > 0)).to(torch.int64))
        dev32.scatter_reduce_(0, rowid, (v32.double() - u64).abs(), reduce="amax")
        devr.scatter_reduce_(0, rowid, (u64r - u64).abs(), reduce="amax")
        ctx.advance(scheme, one64, u64)
        ctx.advance(scheme, one64, u64r)
    cut = slice(0, batch.count)
    return {"flips": flips[cut].cpu().numpy().astype(np.int64),
            "dev32": dev32[cut].cpu().numpy(), "dev_round": devr[cut].cpu().numpy()}


def fp32_gradient_bar(g64, g64_round, stats: dict, base: float = 1e-4, safety: float = 4.0,
                      flip_bar: float = 1e-2) -> np.ndarray:
    """Per-row bar for the relative L2 error of an FP32 gradient against the FP64
    one. g64, g64_round: FP64 gradients (rows x n, numpy) from u0 and from u0
    rounded to FP32; stats: trajectory_stats of the same problem. A row with a
    flipped upwind decision gets `flip_bar`. Otherwise the gradient's
    sensitivity to the trajectory, kappa = |g64_round - g64| / |g64| per unit
    dev_round, times the FP32 trajectory's own deviation dev32 (a linear
    estimate of the error it causes), times `safety`, is added to `base`."""
    num = np.linalg.norm(g64_round - g64, axis=1)
    den = np.maximum(np.linalg.norm(g64, axis=1), 1e-300)
    dr = stats["dev_round"]
    kappa = np.where(dr > 0, (num / den) / np.where(dr > 0, dr, 1.0), 0.0)
    bar = base + safety * kappa * stats["dev32"]
    return np.where(stats["flips"] > 0, np.maximum(bar, flip_bar), bar)


__all__ = ["trajectory_stats", "fp32_gradient_bar"]
