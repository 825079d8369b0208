"""GPU parity of the chunk split of ragged FP32 rows.

FP32 BTCS, Crank-Nicolson, Picard, forward-Euler and RK4 (16 nodes a thread
and more) rows shorter than their CTA's capacity NT x C are cut into
t = ceil(n / C) chunks of C or C - 1
nodes, the last tC - n of them one node short, so a chunk's end sits at a
position known when the kernel is compiled; threads past chunk t - 1 hold no
nodes. Cluster rows are spread evenly over their CTAs and each CTA's nodes
are split the same way. The lengths below put the split at its extremes: no
short chunk (n a multiple of C), one short chunk, C - 1 of them, the first
short chunk in the first lane of a warp, the last chunk in the first or the
last lane of a warp, and whole warps without a chunk behind it; both
boundary conditions, against the FP64 oracle at the FP32 bar.
"""
import numpy as np
import pytest

from gpu_helpers import (BTCS, CN, EXPLICIT, F32, NEWTON, PICARD, RK4, assert_parity, oracle_dts,
                         run_gpu, run_oracle)
from test_gpu_implicit import _resolved
from test_gpu_ragged import _concat, _row, tune_key

pytestmark = pytest.mark.gpu

# kernel kinds of the tuning table (csrc/kernels.h)
KIND = {EXPLICIT: 0, BTCS: 2, RK4: 9, CN: 11, PICARD: 12}


def split_lengths(nt, c):
    """Row lengths n = t c - b of the class (NT c / 2, NT c): t chunks, b short."""
    cap = nt * c
    out = set()
    for t in (nt // 2 + 1, nt // 2 + 32, nt // 2 + 33, nt - 32, nt - 31, nt - 1, nt):
        for b in (0, 1, c // 2, c - 1):
            n = t * c - b
            if cap // 2 < n < cap and b <= t:
                out.add(n)
    # the first short chunk in lane 0 of a warp: t - b a multiple of 32
    t = nt - 1
    b = t % 32 if t % 32 <= c - 1 else 0
    if cap // 2 < t * c - b < cap:
        out.add(t * c - b)
    return sorted(out)


CASES = [
    (BTCS, 128, 32), (BTCS, 256, 32), (BTCS, 64, 32), (BTCS, 128, 16), (BTCS, 32, 4),
    (CN, 128, 32), (CN, 64, 32),
    (PICARD, 128, 16),
    (EXPLICIT, 128, 32), (EXPLICIT, 128, 16), (EXPLICIT, 512, 8),
    (RK4, 128, 16), (RK4, 512, 16),
]


@pytest.mark.parametrize("scheme,nt,c", CASES)
def test_chunk_split_extremes(scheme, nt, c, tmp_path):
    from paper_2601_12204_b300.api import Context
    cap = nt * c
    table = tmp_path / "tune.txt"
    table.write_text("# libburgers tuning table: key nt c k\n" + "".join(
        f"{tune_key(KIND[scheme], F32, cap, ex)} {nt} {c} 0\n" for ex in (0, 1)))
    ns = split_lengths(nt, c)
    assert len(ns) >= 8
    ens = _concat([_row(n, bc, seed=11 * n + bc) for n in ns for bc in (0, 1)])
    implicit = scheme in (BTCS, CN, PICARD)
    dts = oracle_dts(ens, 8.0 if implicit else 1.0)
    steps = np.array([9 + (i % 4) for i in range(ens.count)])
    iters = 2 if scheme == PICARD else 1
    ctx = Context(0)
    try:
        ctx.tune_load(str(table))
        got = run_gpu(ctx, scheme, ens, dts, steps, F32, iters=iters)
    finally:
        ctx.close()
    ref = run_oracle(scheme, ens, dts, steps, iters=iters)
    assert_parity(ens, got, ref, F32, f"split s{scheme} {nt}x{c}")


# cluster rows: n nodes over CS = ceil(n / 4096) CTAs of 128 x 32; per CTA
# n / CS nodes (the first n % CS CTAs one more), split into chunks of 32 or 31
CLUSTER_LENGTHS = [
    8193,          # CS 3, 2731 a CTA: 86 chunks, 21 short
    8256,          # CS 3, 2752 a CTA: 86 full chunks
    12289,         # CS 4, 3073 / 3072 a CTA
    20479,         # CS 5, four CTAs of 4096 and one of 4095 (one short chunk)
    4096 * 6 + 5,  # CS 7, 3511 / 3512 a CTA
    40961,         # CS 11
    65535,         # CS 16, fifteen full CTAs and one short chunk in the last
]


# every variant the cluster kernel runs: (scheme, iterations, dt / CFL dt);
# Newton on viscosity-raised rows at the CFL dt (its Jacobian is diagonally
# dominant there)
CLUSTER_CASES = [(BTCS, 1, 8.0), (CN, 1, 8.0), (PICARD, 2, 6.0), (NEWTON, 2, 1.0)]


@pytest.mark.parametrize("scheme,iters,fac", CLUSTER_CASES)
def test_cluster_chunk_split(scheme, iters, fac):
    from paper_2601_12204_b300.api import Context
    ens = _concat([_row(n, bc, seed=5 * n + bc) for n in CLUSTER_LENGTHS for bc in (0, 1)])
    ens = _resolved(ens, scheme)
    dts = oracle_dts(ens, fac)
    steps = np.array([7 + (i % 3) for i in range(ens.count)])
    ctx = Context(0)
    try:
        got = run_gpu(ctx, scheme, ens, dts, steps, F32, iters=iters)
    finally:
        ctx.close()
    ref = run_oracle(scheme, ens, dts, steps, iters=iters)
    assert_parity(ens, got, ref, F32, f"cluster split s{scheme} it{iters}")
