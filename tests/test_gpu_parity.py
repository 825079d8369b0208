"""GPU parity: the CUDA path against the FP64 oracle on the same seeded inputs."""
import math

import numpy as np
import pytest

import oracle
from gpu_helpers import (BTCS, EXPLICIT, F32, F64, assert_parity, oracle_dts, run_gpu,
                         run_oracle)
from paper_2601_12204_b300 import _lib as L
from paper_2601_12204_b300 import workloads as W

pytestmark = pytest.mark.gpu

SCHEMES = [EXPLICIT, BTCS]


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
                     (L.BURGERS_OPT_GRAPHS, 1), (L.BURGERS_OPT_STREAM_K, 0),
                     (L.BURGERS_OPT_CLUSTER, 1)):
        ctx.set(opt, val)


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("dtype", [F64, F32])
def test_plain_sine_n256(ctx, scheme, dtype):
    """N = 256 Dirichlet, u0 = -sin(pi x), nu = 0.01/pi, t_f = 1/pi, 102 steps."""
    _fresh(ctx)
    e = W.plain_sine(256)
    dt0 = oracle.cfl_dt(e.u0, e.dxs[0], e.nus[0], 0.4)
    n = math.ceil(e.meta["t_final"] / dt0)
    dts = np.array([e.meta["t_final"] / n])
    assert n == 102
    got = run_gpu(ctx, scheme, e, dts, n, dtype)
    ref = run_oracle(scheme, e, dts, n)
    assert_parity(e, got, ref, dtype, "plain sine")
    # the odd initial condition stays odd on the GPU too
    # (the partitioned solve is not mirror-symmetric in rounding: FP32 bar)
    assert np.max(np.abs(got + got[::-1])) <= (1e-13 if dtype == F64 else 1e-5)


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("dtype", [F64, F32])
@pytest.mark.parametrize("bc", [W.PERIODIC, W.DIRICHLET])
def test_exact_shapes(ctx, scheme, dtype, bc):
    """Row lengths equal to every resident register capacity (no padding)."""
    _fresh(ctx)
    ns = [32, 64, 128, 256, 512, 1024, 2048, 4096]
    if scheme == EXPLICIT:
        ns += [8192, 16384] if dtype == F64 else [8192, 16384, 32768]
    else:
        ns += [8192] if dtype == F32 else []
    rows = []
    for n in ns:
        e = W.fourier_ensemble(2, n, seed=n)
        e.bcs[:] = bc
        rows.append(e)
    ens = _concat(rows)
    dts = oracle_dts(ens, 1.0 if scheme == EXPLICIT else 10.0)
    steps = np.where(ens.ns > 4096, 40, 150)
    got = run_gpu(ctx, scheme, ens, dts, steps, dtype)
    ref = run_oracle(scheme, ens, dts, steps)
    assert_parity(ens, got, ref, dtype, f"exact s{scheme} bc{bc}")


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("dtype", [F64, F32])
def test_ragged_mixed_batch(ctx, scheme, dtype):
    """Uneven rows (n from 3 to several thousand, both BCs, ragged step counts)
    in one call, including lengths just above and below shape capacities."""
    _fresh(ctx)
    nmax = 6000 if (scheme == EXPLICIT or dtype == F32) else 4000
    ens = W.mixed_ensemble(60, 3, nmax, seed=77)
    extra = [3, 4, 5, 31, 33, 63, 65, 255, 257, 1023, 1025, 4095, 4097 if nmax > 4097 else 3999]
    ens = _concat([ens] + [_one(n, bc, seed=n + bc) for n in extra for bc in (0, 1)])
    dts = oracle_dts(ens, 1.0 if scheme == EXPLICIT else 7.0)
    g = np.random.default_rng(5)
    steps = g.integers(0, 300, ens.count)
    got = run_gpu(ctx, scheme, ens, dts, steps, dtype)
    ref = run_oracle(scheme, ens, dts, steps)
    assert_parity(ens, got, ref, dtype, f"ragged s{scheme}")


@pytest.mark.parametrize("dtype", [F64, F32])
@pytest.mark.parametrize("K", [1, 7, 32])
def test_streaming_explicit(ctx, dtype, K):
    """Long rows through the temporally blocked streaming kernel (several
    windows per row, a ragged last window, both BCs, odd and even passes)."""
    _fresh(ctx)
    ctx.set(L.BURGERS_OPT_RESIDENT_MAX, 1024)
    ctx.set(L.BURGERS_OPT_STREAM_K, K)
    try:
        ens = _concat([_one(n, bc, seed=n) for n in (5000, 9001, 70001) for bc in (0, 1)])
        dts = oracle_dts(ens)
        steps = np.array([3 * K + 1, 2 * K, 97, 64, 150, K])
        got = run_gpu(ctx, EXPLICIT, ens, dts, steps, dtype)
        ref = run_oracle(EXPLICIT, ens, dts, steps)
        assert_parity(ens, got, ref, dtype, f"stream K{K}")
    finally:
        _fresh(ctx)


@pytest.mark.parametrize("dtype", [F64, F32])
def test_streaming_explicit_default_windows(ctx, dtype):
    """Rows of 8192 nodes and more with the untuned streaming defaults (FP32:
    windows of 8192 nodes, 64 steps a pass): one window, two, a ragged last
    window, both BCs, partial last passes."""
    _fresh(ctx)
    ctx.set(L.BURGERS_OPT_RESIDENT_MAX, 1024)
    try:
        ens = _concat([_one(n, bc, seed=n + bc) for n in (8192, 9001, 16385, 70001)
                       for bc in (0, 1)])
        dts = oracle_dts(ens)
        steps = np.array([193, 128, 97, 64, 150, 1, 200, 65])
        got = run_gpu(ctx, EXPLICIT, ens, dts, steps, dtype)
        ref = run_oracle(EXPLICIT, ens, dts, steps)
        assert_parity(ens, got, ref, dtype, "stream default K")
    finally:
        _fresh(ctx)


# single-step tile shapes (threads, nodes a thread, bulk-copy stages; 0 = the
# per-tile kernel only) of the K = 1 streaming path
STEP1_SHAPES = {F32: [(512, 8, 0), (512, 8, 3), (512, 8, 4), (256, 16, 4), (128, 16, 6)],
                F64: [(256, 4, 0), (256, 4, 4)]}


@pytest.mark.parametrize("dtype", [F64, F32])
@pytest.mark.parametrize("misalign", [0, 1])
def test_streaming_k1_bulk_tiles(ctx, dtype, misalign, tmp_path):
    """One step per pass (K = 1) with rows at 16-element offsets, for every
    registered single-step shape (set through the tuning table): with bulk
    stages, whole tiles go through the bulk-copy kernel (TMA ring) and row
    tails through the per-tile path in the same launch; misalign = 1 shifts the
    caller's buffer by one element, so every tile takes the per-tile kernel.
    Both BCs, odd and even pass counts, against the oracle; the device error
    word stays 0."""
    key = (8 << 56) ^ (dtype << 52)  # K_EXPLICIT_STEP1, class 0
    try:
        for nt, c, stages in STEP1_SHAPES[dtype]:
            path = tmp_path / f"step1_{nt}_{c}_{stages}.txt"
            path.write_text(f"# step1 shape\n{key} {nt} {c} {stages}\n")
            ctx.tune_load(str(path))
            _k1_bulk_case(ctx, dtype, misalign, nt * c)
    finally:  # back to the library's default shape
        nt, c, stages = STEP1_SHAPES[dtype][0]
        path = tmp_path / "step1_default.txt"
        path.write_text(f"# step1 shape\n{key} {nt} {c} {stages}\n")
        ctx.tune_load(str(path))


def _k1_bulk_case(ctx, dtype, misalign, tile):
    import torch

    from paper_2601_12204_b300.api import Batch
    _fresh(ctx)
    ctx.set(L.BURGERS_OPT_RESIDENT_MAX, 1024)
    ctx.set(L.BURGERS_OPT_STREAM_K, 1)
    try:
        lens = [3 * tile, 5 * tile + 123, 70001, 16 * tile + 16, 2 * tile - 5]
        parts = [_one(n, bc, seed=n + 11 * bc) for n in lens for bc in (0, 1)]
        offs, o = [], 0
        for p in parts:
            offs.append(o)
            o = (o + int(p.ns[0]) + 37 + 15) // 16 * 16  # gaps, 16-element starts
        span = o
        ens = _concat(parts)
        ens.offsets = np.array(offs, np.int64)
        buf = np.full(span + 1, 2.5)
        for b, p in enumerate(parts):
            buf[offs[b]:offs[b] + int(p.ns[0])] = p.u0
        dts = oracle_dts(ens)
        steps = np.array([1, 2, 7, 8, 13, 1, 4, 5, 3, 6])
        tdt = torch.float32 if dtype == F32 else torch.float64
        if misalign:  # a view one element past an allocation's (aligned) start
            base = torch.tensor(np.concatenate([[7.0], buf]), dtype=tdt, device="cuda")
            u = base[1:]
        else:
            u = torch.tensor(buf, dtype=tdt, device="cuda")
        b = Batch(dtype, ens.offsets, ens.ns, ens.bcs, ens.dxs, ens.nus, dts, steps)
        ctx.explicit_advance(b, u)
        torch.cuda.synchronize()
        got_buf = u.cpu().double().numpy()
        ref_ens = _concat(parts)
        ref = run_oracle(EXPLICIT, ref_ens, dts, steps)
        got = np.concatenate([got_buf[offs[i]:offs[i] + int(parts[i].ns[0])] for i in range(len(parts))])
        assert_parity(ref_ens, got, ref, dtype, f"k1 bulk misalign {misalign}")
        mask = np.ones(span + 1, bool)
        for i, p in enumerate(parts):
            mask[offs[i]:offs[i] + int(p.ns[0])] = False
        assert np.all(got_buf[mask] == 2.5)  # gaps untouched
        assert ctx.device_error() == 0
    finally:
        _fresh(ctx)


@pytest.mark.parametrize("dtype", [F64, F32])
def test_multilevel_btcs(ctx, dtype):
    """Long BTCS rows through the multi-level partitioned solver (one and two
    reduction levels, every top shape, both BCs, ragged step counts)."""
    _fresh(ctx)
    ctx.set(L.BURGERS_OPT_RESIDENT_MAX, 64)
    try:
        ns = (100, 700, 5000, 70001)
        ens = _concat([_one(n, bc, seed=n + 3) for n in ns for bc in (0, 1)])
        dts = oracle_dts(ens, 8.0)
        steps = np.array([7, 3, 25, 24, 40, 1, 12, 13])
        got = run_gpu(ctx, BTCS, ens, dts, steps, dtype)
        ref = run_oracle(BTCS, ens, dts, steps)
        assert_parity(ens, got, ref, dtype, "multilevel")
    finally:
        _fresh(ctx)


@pytest.mark.parametrize("dtype", [F64, F32])
def test_large_grid_both_schemes(ctx, dtype):
    """Configuration-3 shape at 2^22 nodes (periodic, sin x + 0.5 + noise,
    nu = 1e-3): streaming explicit (FP32: the default 128 steps a pass, one
    full pass and a partial one) and multi-level BTCS against the oracle."""
    _fresh(ctx)
    ens = W.large_grid(1 << 22)
    dt0 = oracle_dts(ens)
    for scheme, dts, steps in ((EXPLICIT, dt0, 160), (BTCS, dt0 * 10.0, 4)):
        got = run_gpu(ctx, scheme, ens, dts, steps, dtype)
        ref = run_oracle(scheme, ens, dts, steps)
        assert_parity(ens, got, ref, dtype, f"large s{scheme}")


def test_gaps_between_rows_untouched(ctx):
    """Elements outside every row keep their values (streaming and resident)."""
    import torch
    _fresh(ctx)
    ctx.set(L.BURGERS_OPT_RESIDENT_MAX, 1024)
    try:
        from paper_2601_12204_b300.api import Batch
        e = _concat([_one(3000, 0, 1), _one(500, 1, 2)])
        offs = np.array([10, 3100])
        buf = np.full(3700, 7.5)
        for b in range(2):
            buf[offs[b]:offs[b] + e.ns[b]] = e.row(b)
        dts = oracle_dts(e)
        bt = Batch(F64, offs, e.ns, e.bcs, e.dxs, e.nus, dts, [33, 20])
        u = torch.tensor(buf, device="cuda")
        ctx.explicit_advance(bt, u)
        out = u.cpu().numpy()
        mask = np.ones(buf.size, bool)
        for b in range(2):
            mask[offs[b]:offs[b] + e.ns[b]] = False
        assert np.all(out[mask] == 7.5)
    finally:
        _fresh(ctx)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_ensemble_4096x4096_sampled(ctx, scheme):
    """4096 periodic rows x 4096 nodes, FP32 and FP64, 2000 explicit steps at
    CFL 0.4 or 200 BTCS steps at 10x that dt: sampled rows against the oracle
    (relative L2 and elementwise bars), and every FP32 row against the GPU FP64
    result (the FP32 error per row, relative L2 and elementwise)."""
    import torch
    _fresh(ctx)
    ens = W.fourier_ensemble(4096, 4096, seed=W.DEFAULT_SEED)
    dts = oracle_dts(ens, 1.0 if scheme == EXPLICIT else 10.0)
    steps = 2000 if scheme == EXPLICIT else 200
    g32 = run_gpu(ctx, scheme, ens, dts, steps, F32)
    g64 = run_gpu(ctx, scheme, ens, dts, steps, F64)
    ids = np.array([0, 1, 777, 2048, 4095])
    sub = ens.subset(ids)
    ref = run_oracle(scheme, sub, dts[ids], steps)
    for j, b in enumerate(ids):
        o = int(ens.offsets[b])
        so = int(sub.offsets[j])
        r = ref[so:so + 4096]
        assert oracle.rel_l2(g64[o:o + 4096], r) <= 1e-12
        assert oracle.rel_l2(g32[o:o + 4096], r) <= 1e-5
        scale = float(np.max(np.abs(r)))
        assert float(np.max(np.abs(g64[o:o + 4096] - r))) <= 1e-11 * scale
        assert float(np.max(np.abs(g32[o:o + 4096] - r))) <= 1e-4 * scale
    # FP32 vs FP64 on every row, elementwise ...
    a32, a64 = g32.reshape(4096, 4096), g64.reshape(4096, 4096)
    worst = np.max(np.abs(a32 - a64), axis=1) / np.max(np.abs(a64), axis=1)
    assert float(np.max(worst)) <= 1e-4
    # ... and in relative L2 through the GPU norm kernel
    from paper_2601_12204_b300.api import Batch
    b32 = Batch.from_ensemble(ens, dts, steps, F32)
    rel, _ = ctx.rel_l2(b32, torch.tensor(g32, dtype=torch.float32, device="cuda"),
                        torch.tensor(g64, device="cuda"))
    assert float(np.max(rel)) <= 1e-5


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("dtype", [F64, F32])
def test_degenerate_cases(ctx, scheme, dtype):
    _fresh(ctx)
    rows = [_one(3, 0, 1), _one(3, 1, 2), _one(4, 0, 3), _one(700, 0, 4)]
    ens = _concat(rows)
    # constant state rows
    for b, cval in ((2, 1.25),):
        o = ens.offsets[b]
        ens.u0[o:o + ens.ns[b]] = cval
    dts = oracle_dts(ens, 3.0 if scheme == BTCS else 1.0)
    steps = [5, 5, 9, 0]
    got = run_gpu(ctx, scheme, ens, dts, steps, dtype)
    ref = run_oracle(scheme, ens, dts, steps)
    assert_parity(ens, got, ref, dtype, "degenerate")
    o = ens.offsets[3]
    assert np.array_equal(got[o:o + 700], ens.u0[o:o + 700].astype(
        np.float32 if dtype == F32 else np.float64).astype(np.float64))


@pytest.mark.parametrize("scheme", SCHEMES)
def test_inviscid_rows(ctx, scheme):
    """nu = 0: pure upwind convection (s = 0)."""
    _fresh(ctx)
    ens = _concat([_one(n, bc, seed=n) for n in (100, 1000) for bc in (0, 1)])
    ens.nus[:] = 0.0
    dts = oracle_dts(ens, 1.0 if scheme == EXPLICIT else 5.0)
    got = run_gpu(ctx, scheme, ens, dts, 120, F64)
    ref = run_oracle(scheme, ens, dts, 120)
    assert_parity(ens, got, ref, F64, "inviscid")


def test_cfl_dt_matches_oracle(ctx):
    import torch
    from paper_2601_12204_b300.api import Batch
    _fresh(ctx)
    ens = W.mixed_ensemble(40, 3, 40000, seed=9)
    ens.nus[::3] = 0.0
    b = Batch.from_ensemble(ens, 1.0, 0, F64)
    dt = ctx.cfl_dt(b, torch.tensor(ens.u0, device="cuda"), 0.4)
    ref = np.array([oracle.cfl_dt(ens.row(i), ens.dxs[i], ens.nus[i], 0.4) for i in range(ens.count)])
    assert np.array_equal(dt, ref)


def test_rel_l2_matches_oracle(ctx):
    import torch
    from paper_2601_12204_b300.api import Batch
    _fresh(ctx)
    ens = W.mixed_ensemble(30, 3, 50000, seed=10)
    g = np.random.default_rng(0)
    other = ens.u0 + 1e-3 * g.normal(size=ens.u0.size)
    b = Batch.from_ensemble(ens, 1.0, 0, F64)
    rel, rms = ctx.rel_l2(b, torch.tensor(other, device="cuda"), torch.tensor(ens.u0, device="cuda"))
    for i in range(ens.count):
        o, n = ens.offsets[i], ens.ns[i]
        assert rel[i] == pytest.approx(oracle.rel_l2(other[o:o + n], ens.u0[o:o + n]), rel=1e-13)
        assert rms[i] == pytest.approx(oracle.rms(other[o:o + n], ens.u0[o:o + n]), rel=1e-13)
    b32 = Batch.from_ensemble(ens, 1.0, 0, F32)
    rel32, _ = ctx.rel_l2(b32, torch.tensor(other, dtype=torch.float32, device="cuda"),
                          torch.tensor(ens.u0, device="cuda"))
    assert np.all(np.abs(rel32 - rel) <= 1e-6 + 1e-3 * rel)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_plain_graphs_and_determinism_are_bitwise(ctx, scheme):
    """Batched, one-row-per-launch, graph and no-graph runs and repeated runs
    give bitwise identical results (same kernel shape per row)."""
    _fresh(ctx)
    ens = W.mixed_ensemble(25, 3, 3000, seed=12)
    dts = oracle_dts(ens, 1.0 if scheme == EXPLICIT else 4.0)
    a = run_gpu(ctx, scheme, ens, dts, 80, F32)
    b = run_gpu(ctx, scheme, ens, dts, 80, F32)
    ctx.set(L.BURGERS_OPT_PLAIN, 1)
    c = run_gpu(ctx, scheme, ens, dts, 80, F32)
    ctx.set(L.BURGERS_OPT_PLAIN, 0)
    ctx.set(L.BURGERS_OPT_GRAPHS, 0)
    d = run_gpu(ctx, scheme, ens, dts, 80, F32)
    _fresh(ctx)
    assert np.array_equal(a, b) and np.array_equal(a, c) and np.array_equal(a, d)


def test_solve_host_matches_device(ctx):
    _fresh(ctx)
    from paper_2601_12204_b300.api import Batch
    ens = W.mixed_ensemble(12, 10, 2000, seed=13)
    dts = oracle_dts(ens)
    dev = run_gpu(ctx, EXPLICIT, ens, dts, 50, F64)
    host = ens.u0.copy()
    ctx.solve_host(EXPLICIT, Batch.from_ensemble(ens, dts, 50, F64), host)
    assert np.array_equal(host, dev)


def test_invalid_arguments_rejected(ctx):
    import torch
    from paper_2601_12204_b300.api import Batch
    _fresh(ctx)
    u = torch.zeros(100, dtype=torch.float64, device="cuda")
    lib = L.load()
    bad = [
        Batch(F64, [0], [2], [0], [0.1], [0.1], [0.01], [1]),        # n < 3
        Batch(F64, [0], [10], [5], [0.1], [0.1], [0.01], [1]),       # bad bc
        Batch(F64, [0], [10], [0], [0.0], [0.1], [0.01], [1]),       # dx = 0
        Batch(F64, [0], [10], [0], [0.1], [-1.0], [0.01], [1]),      # nu < 0
        Batch(F64, [0], [10], [0], [0.1], [0.1], [0.0], [1]),        # dt = 0
        Batch(F64, [0], [10], [0], [0.1], [0.1], [0.01], [-1]),      # nsteps < 0
        Batch(F64, [0, 5], [10, 10], [0, 0], [0.1] * 2, [0.1] * 2, [0.01] * 2, [1, 1]),  # overlap
    ]
    before = u.clone()
    for b in bad:
        st = lib.burgers_explicit_advance(ctx.h, b.ref(), u.data_ptr(), None)
        assert st == L.BURGERS_EINVAL, L.last_error()
        st = lib.burgers_btcs_advance(ctx.h, b.ref(), u.data_ptr(), None)
        assert st == L.BURGERS_EINVAL
    ok = Batch(F64, [0], [10], [0], [0.1], [0.1], [0.01], [1])
    assert lib.burgers_explicit_advance(ctx.h, ok.ref(), None, None) == L.BURGERS_EINVAL
    assert lib.burgers_explicit_advance(None, ok.ref(), u.data_ptr(), None) == L.BURGERS_EINVAL
    torch.cuda.synchronize()
    assert torch.equal(u, before)


# ---------------------------------------------------------------------------
def _one(n, bc, seed):
    x, dx = W.grid(n, bc, 0.0, W.TWO_PI)
    a, phi, nu = W.fourier_coeffs(seed, 99)
    u0 = W.fourier_field(x, a, phi)
    return W.Ensemble(u0, np.zeros(1, np.int64), np.array([n], np.int32), np.array([bc], np.int32),
                      np.array([dx]), np.array([nu]), np.zeros(1), np.array([W.TWO_PI]))


def _concat(parts):
    u0 = np.concatenate([p.u0 for p in parts])
    ns = np.concatenate([p.ns for p in parts])
    offs = np.zeros(ns.size, np.int64)
    offs[1:] = np.cumsum(ns[:-1])
    cat = lambda k: np.concatenate([getattr(p, k) for p in parts])  # noqa: E731
    return W.Ensemble(u0, offs, ns, cat("bcs"), cat("dxs"), cat("nus"), cat("x0"), cat("length"))


@pytest.mark.parametrize("scheme", SCHEMES)
def test_autotune_then_parity(ctx, scheme, tmp_path):
    """The autotuner picks shapes per capacity class; results with the tuned
    table still match the oracle, and the table survives a save/load."""
    import torch
    from paper_2601_12204_b300.api import Batch, Context
    _fresh(ctx)
    ens = _concat([W.fourier_ensemble(40, 4096, seed=3), W.fourier_ensemble(40, 2048, seed=4),
                   _one(70001, 0, 5)])
    dts = oracle_dts(ens, 1.0 if scheme == EXPLICIT else 8.0)
    steps = 60 if scheme == EXPLICIT else 12
    b = Batch.from_ensemble(ens, dts, steps, F64)
    c2 = Context(0)
    try:
        ntuned = c2.autotune(scheme, b, torch.tensor(ens.u0, device="cuda"), probe_steps=20)
        assert ntuned >= 1
        got = run_gpu(c2, scheme, ens, dts, steps, F64)
        ref = run_oracle(scheme, ens, dts, steps)
        assert_parity(ens, got, ref, F64, "tuned")
        path = str(tmp_path / "tune.txt")
        c2.tune_save(path)
        c3 = Context(0)
        c3.tune_load(path)
        assert np.array_equal(run_gpu(c3, scheme, ens, dts, steps, F64), got)
        c3.close()
        bad = tmp_path / "bad.txt"
        bad.write_text("123 7 7 7\n")
        with pytest.raises(Exception):
            c2.tune_load(str(bad))
    finally:
        c2.close()


@pytest.mark.parametrize("dtype", [F32])
def test_cluster_btcs(ctx, dtype):
    """BTCS rows longer than one CTA resident in a thread-block cluster: every
    cluster size (128-thread CTAs in clusters of 2..16, the sizes above 8
    non-portable; in portable mode 256-thread CTAs for rows past 8 x 4096),
    ragged last CTAs, both BCs, against the oracle and against the multi-level
    solver."""
    _fresh(ctx)
    # a B300 schedules 16-CTA clusters of this kernel
    assert ctx.get(L.BURGERS_INFO_CLUSTER_CTAS_MAX) == 16
    W_ = 4096
    ns = [2 * W_ + 1, 3 * W_ - 5, 3 * W_, 4 * W_ + 33, 5 * W_ - 1, 6 * W_ + 7, 7 * W_, 8 * W_]
    if dtype == F32:
        ns += [9 * W_ + 3, 10 * W_ - 7, 11 * W_ + 1, 12 * W_, 13 * W_ + 5, 14 * W_,
               15 * W_ - 3, 16 * W_]
        # the last CTA ends on a chunk boundary (32 nodes) with padding lanes
        # behind it in the same warp: warp 0 of the last CTA holds the row's last
        # chunk and 22 padding chunks; warp 1 holds 8 real chunks and 24 padding
        ns += [3 * W_ + 320, 2 * W_ + 32 * 40]
    ens = _concat([_one(n, bc, seed=n + bc) for n in ns for bc in (0, 1)])
    dts = oracle_dts(ens, 8.0)
    steps = np.array([5 + (i % 7) for i in range(ens.count)])
    got = run_gpu(ctx, BTCS, ens, dts, steps, dtype)
    ref = run_oracle(BTCS, ens, dts, steps)
    assert_parity(ens, got, ref, dtype, "cluster")
    ctx.set(L.BURGERS_OPT_CLUSTER, 2)
    assert ctx.get(L.BURGERS_OPT_CLUSTER) == 2
    try:
        portable = run_gpu(ctx, BTCS, ens, dts, steps, dtype)
    finally:
        ctx.set(L.BURGERS_OPT_CLUSTER, 1)
    assert_parity(ens, portable, ref, dtype, "cluster (portable sizes)")
    # rows up to 8 x 4096 nodes (the first 8 lengths, both BCs) take the same
    # 128-thread kernels in both modes
    head = int(ens.offsets[16])
    assert np.array_equal(portable[:head], got[:head])
    ctx.set(L.BURGERS_OPT_CLUSTER, 0)
    try:
        ml = run_gpu(ctx, BTCS, ens, dts, steps, dtype)
    finally:
        ctx.set(L.BURGERS_OPT_CLUSTER, 1)
    assert_parity(ens, ml, ref, dtype, "multilevel")
    ctx.set(L.BURGERS_OPT_PLAIN, 1)
    try:
        pl = run_gpu(ctx, BTCS, ens, dts, steps, dtype)
    finally:
        _fresh(ctx)
    assert np.array_equal(pl, got)


def test_ctx_options_round_trip(ctx):
    """burgers_ctx_get reads back what burgers_ctx_set wrote, reports the
    device facts, and rejects unknown keys and out-of-range cluster modes."""
    _fresh(ctx)
    try:
        for opt, val in ((L.BURGERS_OPT_GRAPHS, 0), (L.BURGERS_OPT_PLAIN, 1),
                         (L.BURGERS_OPT_STREAM_K, 7), (L.BURGERS_OPT_RESIDENT_MAX, 1 << 20),
                         (L.BURGERS_OPT_AUTOTUNE, 1), (L.BURGERS_OPT_CLUSTER, 2),
                         (L.BURGERS_OPT_CLUSTER, 0)):
            ctx.set(opt, val)
            assert ctx.get(opt) == val
        import torch
        assert ctx.get(L.BURGERS_INFO_SM_COUNT) == \
            torch.cuda.get_device_properties(0).multi_processor_count
        assert 8 <= ctx.get(L.BURGERS_INFO_CLUSTER_CTAS_MAX) <= 16
        for bad in (3, -1):
            with pytest.raises(Exception):
                ctx.set(L.BURGERS_OPT_CLUSTER, bad)
        with pytest.raises(Exception):
            ctx.get(L.BURGERS_OPT_LAUNCH_COUNT)
        with pytest.raises(Exception):
            ctx.get(12345)
    finally:
        ctx.set(L.BURGERS_OPT_AUTOTUNE, 0)
        _fresh(ctx)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_ensemble_4096x4096_bench_launch(ctx, scheme):
    """The step the bench times, as it times it: 4096 x 4096 FP32, launch
    shapes from the autotuner, the CFL time step on the device and the advance
    reading it there (burgers_cfl_dt_device + burgers_advance_dt_device).
    Sampled rows against the FP64 oracle at the bench's own dt."""
    import torch

    from paper_2601_12204_b300.api import Batch, Context
    ens = W.fourier_ensemble(4096, 4096, seed=W.DEFAULT_SEED)
    factor = 1.0 if scheme == EXPLICIT else 10.0
    steps = 2000 if scheme == EXPLICIT else 200
    c = Context(0)
    try:
        u0 = torch.tensor(ens.u0, dtype=torch.float32, device="cuda")
        probe = Batch.from_ensemble(ens, 1.0, 0, F32)
        dt_host = c.cfl_dt(probe, u0, 0.4)
        c.autotune(scheme, Batch.from_ensemble(ens, dt_host * factor, steps, F32), u0,
                   probe_steps=50)
        dtd = torch.empty(ens.count, dtype=torch.float64, device="cuda")
        b = Batch.from_ensemble(ens, 1.0, steps, F32)
        u = u0.clone()
        c.cfl_dt_device(probe, u0, 0.4, dtd)
        c.advance_dt_device(scheme, b, u, dtd, factor)
        torch.cuda.synchronize()
        got = u.cpu().numpy().astype(np.float64)
        dts = dtd.cpu().numpy() * factor
    finally:
        c.close()
    ids = np.array([3, 1500, 4094])
    sub = ens.subset(ids)
    ref = run_oracle(scheme, sub, dts[ids], steps)
    for j, bi in enumerate(ids):
        o, so = int(ens.offsets[bi]), int(sub.offsets[j])
        r = ref[so:so + 4096]
        assert oracle.rel_l2(got[o:o + 4096], r) <= 1e-5
        assert float(np.max(np.abs(got[o:o + 4096] - r))) <= 1e-4 * float(np.max(np.abs(r)))


# a partitioned resident BTCS shape of each capacity class
PARTITIONED_SHAPE = {32: (32, 1), 64: (32, 2), 128: (32, 4), 256: (32, 8), 512: (64, 8),
                     1024: (128, 8), 2048: (128, 16)}
# (dtype, threads, longest row, layout mode) of every registered per-thread
# Thomas kernel
THOMAS_VARIANTS = [(F32, 256, 32, 0), (F32, 256, 64, 0), (F32, 128, 128, 0), (F32, 64, 256, 0),
                   (F32, 64, 128, 1), (F32, 64, 256, 1), (F32, 64, 512, 1), (F32, 64, 1024, 1),
                   (F32, 64, 2048, 1), (F32, 256, 32, 2), (F32, 128, 64, 2), (F32, 64, 128, 2),
                   (F32, 32, 256, 2), (F64, 128, 32, 0), (F64, 128, 64, 0), (F64, 64, 128, 0),
                   (F64, 64, 64, 1), (F64, 64, 128, 1), (F64, 64, 256, 1), (F64, 64, 512, 1),
                   (F64, 64, 1024, 1), (F64, 128, 32, 2), (F64, 64, 64, 2), (F64, 32, 128, 2)]


@pytest.mark.parametrize("variant", THOMAS_VARIANTS, ids=lambda v: f"d{v[0]}_{v[1]}x{v[2]}g{v[3]}")
def test_thomas_per_thread_btcs(ctx, variant, tmp_path):
    """BTCS rows through the per-thread Thomas kernel (one thread per row, no
    barrier; forced for the capacity class through the tuning table): 2 nt + 7
    rows of ragged lengths in the class (the class of 32 from n = 3), so
    several CTAs and a partial last one, both BCs, ragged step counts, against
    the oracle; the same rows through the partitioned kernel agree too."""
    dtype, nt, nmax, g = variant
    _fresh(ctx)
    rng = np.random.default_rng(nmax + 7 * nt + g)
    lo = 3 if nmax == 32 else nmax // 2 + 1
    lens = list(rng.integers(lo, nmax + 1, 2 * nt + 7)) + [nmax, lo]
    parts = [_one(int(n), int(i % 2), seed=int(n) + 1000 * i) for i, n in enumerate(lens)]
    ens = _concat(parts)
    dts = oracle_dts(ens, 6.0)
    steps = rng.integers(0, 25, ens.count)
    key = lambda ex: (2 << 56) ^ (dtype << 52) ^ (ex << 48) ^ nmax  # noqa: E731  K_BTCS_RESIDENT class
    path = tmp_path / "thomas.txt"
    path.write_text(f"# thomas\n{key(0)} {nt} {nmax} {1 + g}\n{key(1)} {nt} {nmax} {1 + g}\n")
    ctx.tune_load(str(path))
    try:
        got = run_gpu(ctx, BTCS, ens, dts, steps, dtype)
    finally:  # the partitioned kernel for this class again (a one-warp shape of its capacity)
        pt, pc = PARTITIONED_SHAPE[nmax]
        path.write_text(f"# partitioned\n{key(0)} {pt} {pc} 0\n{key(1)} {pt} {pc} 0\n")
        ctx.tune_load(str(path))
    ref = run_oracle(BTCS, ens, dts, steps)
    assert_parity(ens, got, ref, dtype, f"thomas {variant}")
    part = run_gpu(ctx, BTCS, ens, dts, steps, dtype)
    assert_parity(ens, part, ref, dtype, f"partitioned, class {nmax}")


@pytest.mark.parametrize("dtype", [F64, F32])
def test_thomas_default_routing(dtype):
    """A call with many short BTCS rows takes the per-thread Thomas kernel by
    default (classes of 32 and 64 nodes with at least 8192 rows), mixed with
    longer rows that keep the partitioned kernel; sampled rows of every length
    against the oracle (a fresh context: no tuning-table entries)."""
    import torch

    from paper_2601_12204_b300.api import Batch, Context
    rng = np.random.default_rng(41)
    lens = list(rng.integers(17, 65, 9000)) + list(rng.integers(300, 900, 40))
    offs = np.zeros(len(lens), np.int64)
    offs[1:] = np.cumsum(lens[:-1])
    x = np.concatenate([W.grid(int(n), i % 2, 0.0, W.TWO_PI)[0] for i, n in enumerate(lens)])
    u0 = np.sin(x) + 0.3 * np.cos(3 * x + 0.2)
    ens = W.Ensemble(u0, offs, np.array(lens, np.int32), np.arange(len(lens), dtype=np.int32) % 2,
                     np.array([W.grid(int(n), i % 2, 0.0, W.TWO_PI)[1] for i, n in enumerate(lens)]),
                     rng.uniform(1e-3, 5e-2, len(lens)), np.zeros(len(lens)), np.full(len(lens), W.TWO_PI))
    dts = oracle_dts(ens, 6.0)
    steps = rng.integers(1, 20, len(lens))
    c = Context(0)
    try:
        tdt = torch.float32 if dtype == F32 else torch.float64
        u = torch.tensor(ens.u0, dtype=tdt, device="cuda")
        c.btcs_advance(Batch.from_ensemble(ens, dts, steps, dtype), u)
        torch.cuda.synchronize()
        got = u.cpu().double().numpy()
    finally:
        c.close()
    ids = np.concatenate([rng.choice(9000, 60, replace=False), np.arange(9000, 9040)])
    sub = ens.subset(ids)
    ref = run_oracle(BTCS, sub, dts[ids], steps[ids])
    g = np.concatenate([got[offs[i]:offs[i] + lens[i]] for i in ids])
    assert_parity(sub, g, ref, dtype, "default routing")


def _diffusion_bar(dtype, svals):
    """Per-row bar of the strong-diffusion test. The solve is in increment
    form (A delta = Delta(u^n)), whose right-hand side grows with the
    diffusion number s = nu dt / dx^2 while the increment stays O(|u|), so its
    rounding error grows about in proportion to s; and the Sherman-Morrison
    denominator falls as s grows, which amplifies the error in z. FP64 is
    held to the 1e-12 bar scaled by max(1, s) (measured on a B300: 7e-11 at
    s = 1e4 and 1.8e-8 at s = 1e6 on 64-node rows of the partitioned kernel,
    2e-13 s on rows of the per-thread Thomas kernel); FP32 is held to its
    1e-5 bar up to s = 10 and not run beyond (at s = 1e2: 3.4e-6 on a 64-node
    row of the partitioned kernel, 3.8e-5 on a 34-node row of the per-thread
    Thomas kernel)."""
    if dtype == F32:
        return np.full(len(svals), 1e-5)
    return 1e-12 * np.maximum(1.0, np.asarray(svals))


def _assert_rel(ens, got, ref, bars, what):
    for b in range(ens.count):
        o, n = int(ens.offsets[b]), int(ens.ns[b])
        g, r = got[o:o + n], ref[o:o + n]
        assert np.all(np.isfinite(g)), f"{what} row {b}: non-finite"
        rel = oracle.rel_l2(g, r)
        assert rel <= bars[b], f"{what} row {b} (n={n}): rel L2 {rel:.3e} > {bars[b]:.1e}"


@pytest.mark.parametrize("dtype", [F64, F32])
def test_btcs_strong_diffusion_periodic(ctx, dtype, tmp_path):
    """Periodic BTCS at diffusion numbers s = nu dt / dx^2 from 1 to 10
    (FP32) or 1e6 (FP64), where the Sherman-Morrison denominator 1 + v.z falls
    to about 1e-5: resident rows of 64, 512 and 4096 nodes, a
    cluster-resident row of 20000 (FP32), a multi-level row of 70001, and
    many rows of <= 64 nodes forced through the per-thread Thomas kernel,
    against the oracle with the bars of _diffusion_bar."""
    _fresh(ctx)
    smax = 1e1 if dtype == F32 else 1e6
    sgrid = [s for s in (1.0, 1e1, 1e2, 1e4, 1e6) if s <= smax]
    parts, svals = [], []
    for n in (64, 512, 4096, 20000, 70001):
        for s in sgrid:
            parts.append(_one(n, W.PERIODIC, seed=n + int(np.log10(s))))
            svals.append(s)
    ens = _concat(parts)
    ens.nus[:] = 1.0
    dts = np.array(svals) * ens.dxs ** 2
    got = run_gpu(ctx, BTCS, ens, dts, 3, dtype)
    ref = run_oracle(BTCS, ens, dts, 3)
    _assert_rel(ens, got, ref, _diffusion_bar(dtype, svals), "strong diffusion")
    # the per-thread Thomas kernel (class of 64 nodes, forced)
    rng = np.random.default_rng(5)
    lens = rng.integers(33, 65, 300)
    ens = _concat([_one(int(n), W.PERIODIC, seed=int(n) + 17 * i) for i, n in enumerate(lens)])
    ens.nus[:] = 1.0
    svals = 10.0 ** rng.uniform(0, np.log10(smax), ens.count)
    dts = svals * ens.dxs ** 2
    nt = 128 if dtype == F32 else 64
    key = lambda ex: (2 << 56) ^ (dtype << 52) ^ (ex << 48) ^ 64  # noqa: E731
    path = tmp_path / "thomas.txt"
    path.write_text(f"# thomas\n{key(0)} {nt} 64 3\n{key(1)} {nt} 64 3\n")
    ctx.tune_load(str(path))
    try:
        got = run_gpu(ctx, BTCS, ens, dts, 3, dtype)
    finally:
        pt, pc = PARTITIONED_SHAPE[64]
        path.write_text(f"# partitioned\n{key(0)} {pt} {pc} 0\n{key(1)} {pt} {pc} 0\n")
        ctx.tune_load(str(path))
    ref = run_oracle(BTCS, ens, dts, 3)
    _assert_rel(ens, got, ref, _diffusion_bar(dtype, svals), "strong diffusion, per-thread Thomas")
