"""GPU parity of the RK4 integrator (Eq. 22) against the FP64 oracle."""
import math

import numpy as np
import pytest

import oracle
from gpu_helpers import F32, F64, RK4, assert_parity, oracle_dts, run_gpu, run_oracle
from paper_2601_12204_b300 import _lib as L
from paper_2601_12204_b300 import workloads as W

pytestmark = pytest.mark.gpu


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
    a, phi, nu = W.fourier_coeffs(seed, 98)
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


@pytest.mark.parametrize("dtype", [F64, F32])
def test_rk4_plain_sine_n256(ctx, dtype):
    """N = 256 Dirichlet, u0 = -sin(pi x), nu = 0.01/pi, t_f = 1/pi at the
    forward-Euler CFL step (102 steps)."""
    _fresh(ctx)
    e = W.plain_sine(256)
    dt0 = oracle.cfl_dt(e.u0, e.dxs[0], e.nus[0], 0.4)
    n = math.ceil(e.meta["t_final"] / dt0)
    dts = np.array([e.meta["t_final"] / n])
    got = run_gpu(ctx, RK4, e, dts, n, dtype)
    ref = run_oracle(RK4, e, dts, n)
    assert_parity(e, got, ref, dtype, "rk4 plain sine")
    assert got[0] == 0.0 and got[-1] == 0.0


@pytest.mark.parametrize("dtype", [F64, F32])
@pytest.mark.parametrize("bc", [W.PERIODIC, W.DIRICHLET])
def test_rk4_exact_shapes(ctx, dtype, bc):
    """Row lengths equal to the resident capacities (no padding)."""
    _fresh(ctx)
    ns = [32, 64, 128, 256, 512, 1024, 2048, 4096] + ([8192] if dtype == F32 else [])
    rows = []
    for n in ns:
        e = W.fourier_ensemble(2, n, seed=n + 1)
        e.bcs[:] = bc
        rows.append(e)
    ens = _concat(rows)
    dts = oracle_dts(ens)
    got = run_gpu(ctx, RK4, ens, dts, 120, dtype)
    ref = run_oracle(RK4, ens, dts, 120)
    assert_parity(ens, got, ref, dtype, f"rk4 exact bc{bc}")


@pytest.mark.parametrize("dtype", [F64, F32])
def test_rk4_ragged_mixed_batch(ctx, dtype):
    """Uneven rows from 3 nodes up, both BCs, ragged step counts, one call."""
    _fresh(ctx)
    ens = W.mixed_ensemble(50, 3, 5000 if dtype == F32 else 3000, seed=78)
    extra = [3, 4, 5, 31, 33, 255, 257, 1025, 2049]
    ens = _concat([ens] + [_one(n, bc, seed=n + bc) for n in extra for bc in (0, 1)])
    dts = oracle_dts(ens)
    steps = np.random.default_rng(6).integers(0, 200, ens.count)
    got = run_gpu(ctx, RK4, ens, dts, steps, dtype)
    ref = run_oracle(RK4, ens, dts, steps)
    assert_parity(ens, got, ref, dtype, "rk4 ragged")


@pytest.mark.parametrize("dtype", [F64, F32])
@pytest.mark.parametrize("K", [1, 3, 8])
def test_rk4_streaming(ctx, dtype, K):
    """Long rows through the windowed streaming kernel (4K stale nodes per
    side and pass), several windows per row, both BCs, odd and even passes."""
    _fresh(ctx)
    ctx.set(L.BURGERS_OPT_RESIDENT_MAX, 1024)
    ctx.set(L.BURGERS_OPT_STREAM_K, K)
    try:
        ens = _concat([_one(n, bc, seed=n) for n in (5000, 9001, 70001) for bc in (0, 1)])
        dts = oracle_dts(ens)
        steps = np.array([3 * K + 1, 2 * K, 41, 24, 50, K])
        got = run_gpu(ctx, RK4, ens, dts, steps, dtype)
        ref = run_oracle(RK4, ens, dts, steps)
        assert_parity(ens, got, ref, dtype, f"rk4 stream K{K}")
    finally:
        _fresh(ctx)


@pytest.mark.parametrize("dtype", [F64, F32])
def test_rk4_streaming_default_k(ctx, dtype):
    """Long rows with the untuned RK4 streaming default (FP32: 32 steps a pass,
    128 stale nodes per side; the next window prefetched into shared memory
    while a window runs), both BCs, partial last passes."""
    _fresh(ctx)
    ctx.set(L.BURGERS_OPT_RESIDENT_MAX, 1024)
    try:
        ens = _concat([_one(n, bc, seed=n + bc) for n in (5000, 9001, 70001) for bc in (0, 1)])
        dts = oracle_dts(ens)
        steps = np.array([97, 64, 33, 32, 65, 1])
        got = run_gpu(ctx, RK4, ens, dts, steps, dtype)
        ref = run_oracle(RK4, ens, dts, steps)
        assert_parity(ens, got, ref, dtype, "rk4 stream default K")
    finally:
        _fresh(ctx)


def test_rk4_batched_plain_graphs_bitwise(ctx):
    """Batched, one-row-per-launch, graph and no-graph runs agree bitwise."""
    _fresh(ctx)
    ens = W.mixed_ensemble(20, 3, 3000, seed=13)
    dts = oracle_dts(ens)
    a = run_gpu(ctx, RK4, ens, dts, 60, F32)
    ctx.set(L.BURGERS_OPT_PLAIN, 1)
    c = run_gpu(ctx, RK4, ens, dts, 60, F32)
    ctx.set(L.BURGERS_OPT_PLAIN, 0)
    ctx.set(L.BURGERS_OPT_GRAPHS, 0)
    d = run_gpu(ctx, RK4, ens, dts, 60, F32)
    _fresh(ctx)
    assert np.array_equal(a, c) and np.array_equal(a, d)


def test_rk4_autotune_and_host_solve(ctx):
    """Tuned RK4 shapes still match the oracle; the host-memory entry point
    gives the device result."""
    import torch
    from paper_2601_12204_b300.api import Batch, Context
    _fresh(ctx)
    ens = _concat([W.fourier_ensemble(30, 4096, seed=9), W.fourier_ensemble(30, 1024, seed=10)])
    dts = oracle_dts(ens)
    b = Batch.from_ensemble(ens, dts, 40, F64)
    c2 = Context(0)
    try:
        assert c2.autotune(RK4, b, torch.tensor(ens.u0, device="cuda"), probe_steps=10) >= 1
        got = run_gpu(c2, RK4, ens, dts, 40, F64)
        assert_parity(ens, got, run_oracle(RK4, ens, dts, 40), F64, "rk4 tuned")
        host = np.array(ens.u0, dtype=np.float64)
        c2.solve_host(RK4, b, host)
        assert np.array_equal(host, got)
    finally:
        c2.close()
