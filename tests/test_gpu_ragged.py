"""GPU parity of ragged rows on every warp path of the resident kernels.

In a row shorter than its CTA's capacity NT x C, the FP64 rows, RK4 and the
BTCS shapes of fewer than 4 nodes a thread run the warp-uniform split: the
warp holding node n-1 runs the general loop, the warps before it the
exact-row loop and the warps after it (padding) skip the update. FP32 BTCS,
Crank-Nicolson and forward-Euler rows on packed pairs are cut into chunks of
C or C - 1 nodes instead (test_gpu_chunk_split.py puts that split at its
extremes). The row lengths below put node n-1 at the first and last node of
a chunk, in the first and last lane of a warp, with and without padding
warps behind it, for shapes forced through the tuning table.
"""
import numpy as np
import pytest

from gpu_helpers import (BTCS, CN, EXPLICIT, F32, F64, RK4, assert_parity, oracle_dts,
                         run_gpu, run_oracle)

pytestmark = pytest.mark.gpu

# kernel kinds of the tuning table (csrc/kernels.h)
KIND = {EXPLICIT: 0, BTCS: 2, RK4: 9, CN: 11}


def tune_key(kind, dtype, cap, exact):
    return (kind << 56) ^ (dtype << 52) ^ (exact << 48) ^ cap


def ragged_lengths(nt, c):
    cap = nt * c
    half = cap // 2
    cand = [half + 1, half + c, half + c + 1, half + 32 * c - 1, half + 32 * c,
            half + 32 * c + 1, cap - 32 * c + 1, cap - c - 1, cap - c, cap - c + 1,
            cap - 1, cap]
    return sorted({n for n in cand if half < n <= cap})


def _row(n, bc, seed):
    from paper_2601_12204_b300 import workloads as W
    x, dx = W.grid(n, bc, 0.0, W.TWO_PI)
    a, phi, nu = W.fourier_coeffs(seed, 99)
    return W.Ensemble(W.fourier_field(x, a, phi), np.zeros(1, np.int64), np.array([n], np.int32),
                      np.array([bc], np.int32), np.array([dx]), np.array([nu]), np.zeros(1),
                      np.array([W.TWO_PI]))


def _concat(parts):
    from paper_2601_12204_b300 import workloads as W
    ns = np.concatenate([p.ns for p in parts])
    offs = np.zeros(ns.size, np.int64)
    offs[1:] = np.cumsum(ns[:-1])
    cat = lambda k: np.concatenate([getattr(p, k) for p in parts])  # noqa: E731
    return W.Ensemble(cat("u0"), offs, ns, cat("bcs"), cat("dxs"), cat("nus"), cat("x0"),
                      cat("length"))


CASES = [
    (EXPLICIT, F32, 256, 16), (EXPLICIT, F32, 128, 32), (EXPLICIT, F32, 512, 8),
    (EXPLICIT, F64, 128, 16),
    (RK4, F32, 512, 8), (RK4, F32, 256, 16),
    (BTCS, F32, 128, 16), (BTCS, F32, 256, 8), (BTCS, F32, 256, 16), (BTCS, F32, 512, 8),
    (BTCS, F32, 64, 32), (BTCS, F32, 128, 32), (BTCS, F32, 256, 32),
    (BTCS, F64, 128, 16),
    (CN, F32, 128, 16), (CN, F32, 128, 32),
]


@pytest.mark.parametrize("scheme,dtype,nt,c", CASES)
def test_ragged_warp_paths(scheme, dtype, nt, c, tmp_path):
    from paper_2601_12204_b300.api import Context
    cap = nt * c
    table = tmp_path / "tune.txt"
    table.write_text("# libburgers tuning table: key nt c k\n" + "".join(
        f"{tune_key(KIND[scheme], dtype, cap, ex)} {nt} {c} 0\n" for ex in (0, 1)))
    ns = ragged_lengths(nt, c)
    ens = _concat([_row(n, bc, seed=7 * n + bc) for n in ns for bc in (0, 1)])
    implicit = scheme in (BTCS, CN)
    dts = oracle_dts(ens, 8.0 if implicit else 1.0)
    steps = np.array([9 + (i % 5) for i in range(ens.count)])
    ctx = Context(0)
    try:
        ctx.tune_load(str(table))
        got = run_gpu(ctx, scheme, ens, dts, steps, dtype)
    finally:
        ctx.close()
    ref = run_oracle(scheme, ens, dts, steps)
    assert_parity(ens, got, ref, dtype, f"ragged s{scheme} {nt}x{c}")


def test_forced_shapes_take_effect(tmp_path):
    """The tuning table drives the shape: two BTCS shapes of one capacity
    class partition the rows differently, so their FP32 results differ in
    rounding (both within the parity bar)."""
    from paper_2601_12204_b300.api import Context
    ens = _concat([_row(n, bc, seed=n + bc) for n in (3000, 3585, 4095) for bc in (0, 1)])
    dts = oracle_dts(ens, 8.0)
    steps = np.full(ens.count, 12)
    outs = []
    for nt, c in ((256, 16), (128, 32)):
        table = tmp_path / f"t{nt}.txt"
        table.write_text("# libburgers tuning table: key nt c k\n" + "".join(
            f"{tune_key(KIND[BTCS], F32, 4096, ex)} {nt} {c} 0\n" for ex in (0, 1)))
        ctx = Context(0)
        try:
            ctx.tune_load(str(table))
            outs.append(run_gpu(ctx, BTCS, ens, dts, steps, F32))
        finally:
            ctx.close()
    assert not np.array_equal(outs[0], outs[1])
    ref = run_oracle(BTCS, ens, dts, steps)
    for o in outs:
        assert_parity(ens, o, ref, F32, "forced shape")
