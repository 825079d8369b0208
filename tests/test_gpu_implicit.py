"""GPU parity of the further implicit schemes (Crank-Nicolson with lagged
upwind coefficients, Picard-iterated implicit upwind, Newton on the Eq. 11
residual) against the FP64 oracle."""
import math

import numpy as np
import pytest

import oracle
from gpu_helpers import (BTCS, CN, F32, F64, NEWTON, PICARD, assert_parity, oracle_dts, run_gpu,
                         run_oracle)
from paper_2601_12204_b300 import _lib as L
from paper_2601_12204_b300 import workloads as W

pytestmark = pytest.mark.gpu

# (scheme, iterations per step, dt as a multiple of the explicit CFL step).
# Newton's Jacobian (central convection) is strictly diagonally dominant while
# r max|w| < 1/2, i.e. up to 1.25x the CFL-0.4 step; the tests stay there.
CASES = [(CN, 1, 8.0), (PICARD, 1, 6.0), (PICARD, 3, 6.0), (NEWTON, 3, 1.0)]


def _resolved(ens, scheme):
    """Central convection (Newton, Eq. 11) is only meaningful on grids that
    resolve the viscous scale: on rows with cell Peclet number max|u| dx/nu
    above 2 it oscillates and its Newton iterates need not converge (even two
    exact solvers then disagree). For Newton the viscosity of each row is
    raised to keep the cell Peclet number at or below 1.5."""
    if scheme == NEWTON:
        for b in range(ens.count):
            peak = float(np.max(np.abs(ens.row(b))))
            ens.nus[b] = max(ens.nus[b], peak * ens.dxs[b] / 1.5)
    return ens


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_12204_b300.api import Context
    c = Context(0)
    yield c
    c.close()


def _fresh(ctx):
    for opt, val in ((L.BURGERS_OPT_RESIDENT_MAX, 0), (L.BURGERS_OPT_PLAIN, 0),
                     (L.BURGERS_OPT_GRAPHS, 1), (L.BURGERS_OPT_STREAM_K, 0)):
        ctx.set(opt, val)


def _one(n, bc, seed):
    x, dx = W.grid(n, bc, 0.0, W.TWO_PI)
    a, phi, nu = W.fourier_coeffs(seed, 97)
    return W.Ensemble(W.fourier_field(x, a, phi), np.zeros(1, np.int64), np.array([n], np.int32),
                      np.array([bc], np.int32), np.array([dx]), np.array([nu]), np.zeros(1),
                      np.array([W.TWO_PI]))


def _concat(parts):
    ns = np.concatenate([p.ns for p in parts])
    offs = np.zeros(ns.size, np.int64)
    offs[1:] = np.cumsum(ns[:-1])
    cat = lambda k: np.concatenate([getattr(p, k) for p in parts])  # noqa: E731
    return W.Ensemble(cat("u0"), offs, ns, cat("bcs"), cat("dxs"), cat("nus"), cat("x0"),
                      cat("length"))


@pytest.mark.parametrize("scheme,iters,fac", CASES)
@pytest.mark.parametrize("dtype", [F64, F32])
def test_plain_sine_n256(ctx, scheme, iters, fac, dtype):
    """N = 256 Dirichlet, u0 = -sin(pi x), nu = 0.01/pi, t_f = 1/pi."""
    _fresh(ctx)
    e = W.plain_sine(256)
    dt0 = oracle.cfl_dt(e.u0, e.dxs[0], e.nus[0], 0.4)
    n = math.ceil(e.meta["t_final"] / dt0)
    dts = np.array([e.meta["t_final"] / n])
    got = run_gpu(ctx, scheme, e, dts, n, dtype, iters=iters)
    ref = run_oracle(scheme, e, dts, n, iters=iters)
    assert_parity(e, got, ref, dtype, f"plain sine s{scheme}")
    assert got[0] == 0.0 and got[-1] == 0.0


@pytest.mark.parametrize("scheme,iters,fac", CASES)
@pytest.mark.parametrize("dtype", [F64, F32])
@pytest.mark.parametrize("bc", [W.PERIODIC, W.DIRICHLET])
def test_exact_shapes(ctx, scheme, iters, fac, dtype, bc):
    """Row lengths equal to the resident capacities (no padding)."""
    _fresh(ctx)
    ns = [32, 64, 256, 1024, 2048, 4096] + ([8192] if dtype == F32 else [])
    rows = []
    for n in ns:
        e = W.fourier_ensemble(2, n, seed=n + 7)
        e.bcs[:] = bc
        rows.append(e)
    ens = _resolved(_concat(rows), scheme)
    dts = oracle_dts(ens, fac)
    got = run_gpu(ctx, scheme, ens, dts, 40, dtype, iters=iters)
    ref = run_oracle(scheme, ens, dts, 40, iters=iters)
    assert_parity(ens, got, ref, dtype, f"exact s{scheme} it{iters} bc{bc}")


@pytest.mark.parametrize("scheme,iters,fac", CASES)
@pytest.mark.parametrize("dtype", [F64, F32])
def test_ragged_mixed_batch(ctx, scheme, iters, fac, dtype):
    _fresh(ctx)
    ens = W.mixed_ensemble(40, 3, 4000, seed=79)
    extra = [3, 4, 5, 33, 255, 1025]
    ens = _resolved(_concat([ens] + [_one(n, bc, seed=n + bc) for n in extra for bc in (0, 1)]),
                    scheme)
    dts = oracle_dts(ens, fac)
    steps = np.random.default_rng(8).integers(0, 60, ens.count)
    got = run_gpu(ctx, scheme, ens, dts, steps, dtype, iters=iters)
    ref = run_oracle(scheme, ens, dts, steps, iters=iters)
    assert_parity(ens, got, ref, dtype, f"ragged s{scheme} it{iters}")


@pytest.mark.parametrize("dtype", [F64, F32])
def test_one_picard_iteration_is_the_btcs_step(ctx, dtype):
    """Picard with one iteration computes exactly the lagged BTCS step."""
    _fresh(ctx)
    ens = W.mixed_ensemble(30, 3, 4000, seed=80)
    dts = oracle_dts(ens, 6.0)
    a = run_gpu(ctx, PICARD, ens, dts, 30, dtype, iters=1)
    b = run_gpu(ctx, BTCS, ens, dts, 30, dtype)
    assert np.array_equal(a, b)


def test_newton_converges_on_the_gpu(ctx):
    """More Newton iterations drive the GPU result to the oracle's fixed
    point of Eq. 11 (residual at rounding level)."""
    _fresh(ctx)
    ens = _resolved(W.fourier_ensemble(4, 1024, seed=21), NEWTON)
    dts = oracle_dts(ens, 1.0)
    got = run_gpu(ctx, NEWTON, ens, dts, 1, F64, iters=6)
    for b in range(ens.count):
        o, n = int(ens.offsets[b]), int(ens.ns[b])
        f = oracle.newton_residual(got[o:o + n], ens.row(b), 0, ens.dxs[b], ens.nus[b], dts[b])
        assert np.max(np.abs(f)) <= 1e-13


# Rows beyond the resident capacity (8192 nodes FP32, 4096 FP64): FP32 rows of
# up to 65536 nodes in a thread-block cluster by default; through the
# multi-level solver, one and two reduction levels (FP32 chunks of 16 nodes and
# a top level of up to 4096 rows: 9000 and 33000 one level, 70001 two; FP64
# chunks of 8 and tops of up to 2048 rows: 9000 one level, 33000 and 70001 two).
LONG_NS = (9000, 33000, 70001)


@pytest.mark.parametrize("scheme,iters,fac", CASES)
@pytest.mark.parametrize("dtype", [F64, F32])
def test_long_rows_multilevel(ctx, scheme, iters, fac, dtype):
    """Long rows of every variant, both BCs, ragged step counts, by the
    default routing against the oracle: FP32 rows of up to 65536 nodes in a
    thread-block cluster, 70001 nodes and every FP64 row through the
    multi-level solver."""
    _fresh(ctx)
    ens = _resolved(_concat([_one(n, bc, seed=n + 5 * bc) for n in LONG_NS for bc in (0, 1)]),
                    scheme)
    dts = oracle_dts(ens, fac)
    steps = np.array([12, 9, 20, 7, 15, 11])
    got = run_gpu(ctx, scheme, ens, dts, steps, dtype, iters=iters)
    ref = run_oracle(scheme, ens, dts, steps, iters=iters)
    assert_parity(ens, got, ref, dtype, f"long s{scheme} it{iters}")


@pytest.mark.parametrize("scheme,iters,fac", CASES)
def test_long_rows_cluster_off(ctx, scheme, iters, fac):
    """FP32 rows of up to 65536 nodes run in a thread-block cluster by
    default; with the cluster off the same rows take the multi-level solver
    (FP32 9000 and 33000 nodes one level, 70001 two) against the oracle."""
    _fresh(ctx)
    ens = _resolved(_concat([_one(n, bc, seed=n + 5 * bc) for n in LONG_NS for bc in (0, 1)]),
                    scheme)
    dts = oracle_dts(ens, fac)
    steps = np.array([12, 9, 20, 7, 15, 11])
    ctx.set(L.BURGERS_OPT_CLUSTER, 0)
    try:
        got = run_gpu(ctx, scheme, ens, dts, steps, F32, iters=iters)
    finally:
        ctx.set(L.BURGERS_OPT_CLUSTER, 1)
    ref = run_oracle(scheme, ens, dts, steps, iters=iters)
    assert_parity(ens, got, ref, F32, f"long cluster off s{scheme} it{iters}")


@pytest.mark.parametrize("scheme,iters,fac", CASES)
@pytest.mark.parametrize("dtype", [F64, F32])
def test_short_rows_forced_multilevel(ctx, scheme, iters, fac, dtype):
    """With the resident limit set to 64 nodes, rows of 100 to 5000 nodes go
    through the multi-level solver too (every top-level shape, rows whose
    steps end at different times, a row with no steps)."""
    _fresh(ctx)
    ctx.set(L.BURGERS_OPT_RESIDENT_MAX, 64)
    try:
        ns = (100, 700, 2049, 5000)
        ens = _resolved(_concat([_one(n, bc, seed=n + 3 + bc) for n in ns for bc in (0, 1)]),
                        scheme)
        dts = oracle_dts(ens, fac)
        steps = np.array([7, 3, 25, 0, 24, 1, 12, 13])
        got = run_gpu(ctx, scheme, ens, dts, steps, dtype, iters=iters)
        ref = run_oracle(scheme, ens, dts, steps, iters=iters)
        assert_parity(ens, got, ref, dtype, f"forced s{scheme} it{iters}")
    finally:
        _fresh(ctx)


@pytest.mark.parametrize("dtype", [F64, F32])
def test_one_picard_iteration_is_the_btcs_step_long(ctx, dtype):
    """On the multi-level path too, one Picard iteration is the lagged BTCS
    step: the same rows at level 0, the same reduction (bitwise)."""
    _fresh(ctx)
    ens = _concat([_one(n, bc, seed=n + bc) for n in (9000, 70001) for bc in (0, 1)])
    dts = oracle_dts(ens, 6.0)
    ctx.set(L.BURGERS_OPT_CLUSTER, 0)
    try:
        a = run_gpu(ctx, PICARD, ens, dts, 10, dtype, iters=1)
        b = run_gpu(ctx, BTCS, ens, dts, 10, dtype)
    finally:
        ctx.set(L.BURGERS_OPT_CLUSTER, 1)
    assert np.array_equal(a, b)


def test_one_picard_iteration_is_the_btcs_step_cluster(ctx):
    """In the cluster-resident kernel (FP32 rows of up to 65536 nodes) one
    Picard iteration is the lagged BTCS step: with the iterate's offset zero
    every added term is exact, and the halo values take the same arithmetic
    (bitwise)."""
    _fresh(ctx)
    ens = _concat([_one(n, bc, seed=n + bc) for n in (9000, 33001, 65000) for bc in (0, 1)])
    dts = oracle_dts(ens, 6.0)
    a = run_gpu(ctx, PICARD, ens, dts, 10, F32, iters=1)
    b = run_gpu(ctx, BTCS, ens, dts, 10, F32)
    assert np.array_equal(a, b)


def test_rejections(ctx):
    """Iteration counts outside [1, 64] are refused before any work is
    queued, and so are long rows of the device-dt entry point (whose
    multi-level rows carry host-computed coefficients)."""
    import torch
    from paper_2601_12204_b300.api import Batch
    _fresh(ctx)
    long_row = _one(20000, 0, 3)
    u = torch.tensor(long_row.u0, device="cuda")
    b = Batch.from_ensemble(long_row, oracle_dts(long_row), 3, F64)
    before = u.clone()
    dt = torch.full((1,), float(oracle_dts(long_row)[0]), dtype=torch.float64, device="cuda")
    for scheme in (CN, PICARD, NEWTON):
        with pytest.raises(Exception):
            ctx.advance_dt_device(scheme, b, u, dt, 1.0, iters=2)
    short = _one(300, 0, 4)
    us = torch.tensor(short.u0, device="cuda")
    bs = Batch.from_ensemble(short, oracle_dts(short), 3, F64)
    for it in (0, 65):
        with pytest.raises(Exception):
            ctx.picard_advance(bs, us, it)
        with pytest.raises(Exception):
            ctx.newton_advance(bs, us, it)
    torch.cuda.synchronize()
    assert torch.equal(u, before)
