"""GPU adjoints against the FP64 oracle's discrete adjoints and finite
differences; the torch.autograd binding; configuration-5 sizes."""
import numpy as np
import pytest

import oracle
from gpu_helpers import BTCS, EXPLICIT, F32, F64, oracle_dts, run_oracle
from paper_2601_12204_b300 import workloads as W

pytestmark = pytest.mark.gpu

# gradient bars: FP64 rel-L2 <= 1e-11 (dJ/du0), rel <= 1e-10 (dJ/dnu); FP32
# rel-L2 <= 1e-4 and rel <= 1e-3 against the FP64 oracle gradient. dJ/dnu is
# a sum over all steps and nodes that can cancel to far below its terms, so
# its bar also has an absolute floor at (FP64: 1e-13, FP32: 1e-6) times the
# largest |dJ/dnu| of the batch.
GTOL = {F64: (1e-11, 1e-10, 1e-13), F32: (1e-4, 1e-3, 1e-6)}


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_12204_b300.api import Context
    c = Context(0)
    yield c
    c.close()


def _problem(ens, scheme, steps, factor):
    dts = oracle_dts(ens, factor)
    ens1 = W.Ensemble(ens.u0 + 0.05 * np.cos(np.arange(ens.u0.size) * 0.37), ens.offsets, ens.ns,
                      ens.bcs, ens.dxs, ens.nus, ens.x0, ens.length)
    target = run_oracle(scheme, ens1, dts, steps)
    uT = run_oracle(scheme, ens, dts, steps)
    return dts, uT - target


def _oracle_grads(scheme, ens, dts, steps, gT):
    f = oracle.explicit_adjoint if scheme == EXPLICIT else oracle.btcs_adjoint
    gu0 = np.zeros_like(ens.u0)
    gnu = np.zeros(ens.count)
    st = np.broadcast_to(np.asarray(steps), (ens.count,))
    for b in range(ens.count):
        o, n = ens.offsets[b], ens.ns[b]
        g, gn = f(ens.u0[o:o + n], ens.bcs[b], ens.dxs[b], ens.nus[b], dts[b], int(st[b]),
                  gT[o:o + n])
        gu0[o:o + n] = g
        gnu[b] = gn
    return gu0, gnu


def _gpu_grads(ctx, scheme, ens, dts, steps, gT, dtype, stride=0):
    import torch

    from paper_2601_12204_b300.api import Batch
    tdt = torch.float32 if dtype == F32 else torch.float64
    b = Batch.from_ensemble(ens, dts, steps, dtype)
    u0 = torch.tensor(ens.u0, dtype=tdt, device="cuda")
    g = torch.tensor(gT, dtype=tdt, device="cuda")
    gu0 = torch.zeros_like(u0)
    gnu = torch.zeros(ens.count, dtype=torch.float64, device="cuda")
    ctx.adjoint(scheme, b, u0, g, gu0, gnu, stride)
    torch.cuda.synchronize()
    return gu0.cpu().double().numpy(), gnu.cpu().numpy()


def _check(ens, got, ref, gnu, gnu_ref, dtype, what, mass=None):
    """mass[b]: an estimate of the sum of |terms| of row b's dJ/dnu (see
    _gnu_mass); where given, dJ/dnu may also deviate by the dJ/du0 bar times
    it (the terms carry the adjoint's relative error and cancel in the sum)."""
    tu, tn, tf = GTOL[dtype]
    floor = tf * float(np.max(np.abs(gnu_ref)))
    for b in range(ens.count):
        o, n = ens.offsets[b], ens.ns[b]
        rel = oracle.rel_l2(got[o:o + n], ref[o:o + n])
        assert rel <= tu, f"{what} row {b} (n={n}, bc={ens.bcs[b]}): dJ/du0 rel L2 {rel:.3e}"
        fl = floor if mass is None else max(floor, tu * mass[b])
        assert abs(gnu[b] - gnu_ref[b]) <= tn * abs(gnu_ref[b]) + fl, \
            f"{what} row {b}: dJ/dnu {gnu[b]!r} vs {gnu_ref[b]!r}"


def _gnu_mass(ens, dts, steps, gT, dtype=F64):
    """Per row, steps * (dt/dx^2) * sum_i |gT_i| |u0_{i+1} - 2 u0_i + u0_{i-1}|:
    the size of the terms dJ/dnu sums (lambda and the state stay of the order
    of gT and u0 over these runs). FP32 adds what the Laplacian of an FP32
    state cannot resolve, 8 eps32 |u0_i| per node: on fine grids (70001 nodes
    on [0, 2 pi)) the Laplacian itself is of that size, so FP32 dJ/dnu is
    bounded by it there."""
    st = np.broadcast_to(np.asarray(steps), (ens.count,))
    out = np.zeros(ens.count)
    eps = 8 * 2.0 ** -24 if dtype == F32 else 0.0
    for b in range(ens.count):
        o, n = ens.offsets[b], ens.ns[b]
        u, g = ens.u0[o:o + n], gT[o:o + n]
        lap = np.abs(np.roll(u, -1) - 2 * u + np.roll(u, 1)) + eps * np.abs(u)
        out[b] = int(st[b]) * dts[b] / ens.dxs[b] ** 2 * float(np.sum(np.abs(g) * lap))
    return out


@pytest.mark.parametrize("scheme", [EXPLICIT, BTCS])
@pytest.mark.parametrize("dtype", [F64, F32])
def test_adjoint_matches_oracle(ctx, scheme, dtype):
    ens = W.mixed_ensemble(24, 5, 2000, seed=31)
    steps = 60 if scheme == EXPLICIT else 20
    factor = 1.0 if scheme == EXPLICIT else 6.0
    dts, gT = _problem(ens, scheme, steps, factor)
    ref, gnu_ref = _oracle_grads(scheme, ens, dts, steps, gT)
    got, gnu = _gpu_grads(ctx, scheme, ens, dts, steps, gT, dtype)
    _check(ens, got, ref, gnu, gnu_ref, dtype, f"adjoint s{scheme}")


@pytest.mark.parametrize("scheme", [EXPLICIT, BTCS])
def test_checkpoint_stride_does_not_change_the_gradient(ctx, scheme):
    ens = W.mixed_ensemble(6, 40, 700, seed=32)
    steps = 37
    dts, gT = _problem(ens, scheme, steps, 1.0 if scheme == EXPLICIT else 4.0)
    a, ga = _gpu_grads(ctx, scheme, ens, dts, steps, gT, F64, 0)
    for stride in (1, 5, 37, 100):
        b, gb = _gpu_grads(ctx, scheme, ens, dts, steps, gT, F64, stride)
        assert np.array_equal(a, b) and np.array_equal(ga, gb)


@pytest.mark.parametrize("scheme", [EXPLICIT, BTCS])
def test_adjoint_matches_gpu_finite_differences(ctx, scheme):
    """Directional derivative of J = 1/2 |u(T) - target|^2 through the GPU FP64
    forward path against the GPU adjoint (rows kept away from u = 0 kinks)."""
    import torch

    from paper_2601_12204_b300.api import Batch
    x, dx = W.grid(300, W.PERIODIC, 0.0, W.TWO_PI)
    u0 = 0.7 + 0.3 * np.sin(x)
    ens = W.Ensemble(u0, np.zeros(1, np.int64), np.array([300], np.int32),
                     np.array([0], np.int32), np.array([dx]), np.array([0.02]), np.zeros(1),
                     np.array([W.TWO_PI]))
    steps = 50
    dts, gT = _problem(ens, scheme, steps, 1.0 if scheme == EXPLICIT else 5.0)
    target = run_oracle(scheme, ens, dts, steps) - gT
    got, gnu = _gpu_grads(ctx, scheme, ens, dts, steps, gT, F64)

    def J(u, nu):
        b = Batch(F64, [0], [300], [0], [dx], [nu], dts, [steps])
        t = torch.tensor(u, device="cuda")
        ctx.advance(scheme, b, t)
        d = t.cpu().numpy() - target
        return 0.5 * float(d @ d)

    v = np.random.default_rng(3).normal(size=300)
    h = 1e-6
    fd = (J(u0 + h * v, 0.02) - J(u0 - h * v, 0.02)) / (2 * h)
    assert float(got @ v) == pytest.approx(fd, rel=1e-6)
    hn = 1e-7
    fdn = (J(u0, 0.02 + hn) - J(u0, 0.02 - hn)) / (2 * hn)
    assert gnu[0] == pytest.approx(fdn, rel=1e-6)


@pytest.mark.parametrize("scheme", [EXPLICIT, BTCS])
def test_autograd_function(ctx, scheme):
    import torch

    from paper_2601_12204_b300.api import Batch
    from paper_2601_12204_b300.autograd import burgers_solve, misfit_loss
    ens = W.mixed_ensemble(8, 30, 500, seed=33)
    steps = 25
    dts, gT = _problem(ens, scheme, steps, 1.0 if scheme == EXPLICIT else 3.0)
    target_np = run_oracle(scheme, ens, dts, steps) - gT
    ref, gnu_ref = _oracle_grads(scheme, ens, dts, steps, gT)
    batch = Batch.from_ensemble(ens, dts, steps, F64)
    u0 = torch.tensor(ens.u0, device="cuda", requires_grad=True)
    nu = torch.tensor(ens.nus, device="cuda", requires_grad=True)
    uT = burgers_solve(ctx, scheme, batch, u0, nu)
    loss = misfit_loss(uT, torch.tensor(target_np, device="cuda"))
    loss.backward()
    _check(ens, u0.grad.cpu().numpy(), ref, nu.grad.cpu().numpy(), gnu_ref, F64, "autograd")


# Differentiation workload, FP32 against FP64 on every row. The discrete
# gradient is that of a piecewise smooth map (the upwind side switches with
# sign(u_i)), steep near forming shocks. Per row (fp32_gradient_bar): 1e-4,
# plus 4 x (the FP64 gradient's change per unit trajectory deviation when u0
# is rounded to FP32) x (the FP32 trajectory's deviation from the FP64 one);
# 1e-2 for a row whose FP32 trajectory takes another upwind side than the
# FP64 one at some (node, step): its gradient is that of another branch (one
# flipped decision moved a row's gradient by 3.5e-3). Rows above 1e-4 (the
# ones that need their wider bar) must stay rare.
WIDE_ROWS_MAX = 0.02


def _differentiation_problem(scheme):
    B, N = 1024, 2048
    ens = W.fourier_ensemble(B, N, seed=W.DEFAULT_SEED)
    tgt = W.fourier_ensemble(B, N, seed=W.DEFAULT_SEED + 1)
    steps = 2000 if scheme == EXPLICIT else 200
    fac = 1.0 if scheme == EXPLICIT else 10.0
    # one dt per row stable for both runs: the target's u0 (seed + 1) can be
    # larger, and a dt set by the CFL limit of u0 alone can make it diverge
    dts = np.minimum(oracle_dts(ens, fac),
                     oracle_dts(W.Ensemble(tgt.u0, ens.offsets, ens.ns, ens.bcs, ens.dxs, ens.nus,
                                           ens.x0, ens.length), fac))
    return ens, tgt, dts, steps


def _pipeline_grads(ctx, scheme, ens, tgt, dts, steps, dtype, round_u0=False):
    """J = 1/2 |u(T) - target|^2 in one precision: forward of u0 and of the
    target's u0 (seed + 1, same nu, dt, steps), gT = u(T) - target, adjoint.
    round_u0: start from u0 rounded to FP32 (in either precision)."""
    import torch

    from paper_2601_12204_b300.api import Batch
    tdt = torch.float32 if dtype == F32 else torch.float64
    b = Batch.from_ensemble(ens, dts, steps, dtype)
    u0 = torch.tensor(ens.u0, dtype=torch.float64, device="cuda")
    if round_u0:
        u0 = u0.float()
    u0 = u0.to(tdt).contiguous()
    ut = torch.tensor(tgt.u0, dtype=tdt, device="cuda")
    uT = u0.clone()
    ctx.advance(scheme, b, uT)
    ctx.advance(scheme, b, ut)
    gu0 = torch.zeros_like(u0)
    gnu = torch.zeros(ens.count, dtype=torch.float64, device="cuda")
    ctx.adjoint(scheme, b, u0, uT - ut, gu0, gnu)
    torch.cuda.synchronize()
    return gu0.double(), gnu


@pytest.mark.parametrize("scheme", [EXPLICIT, BTCS])
def test_differentiation_1024x2048_all_rows(ctx, scheme):
    """B = 1024 periodic rows x 2048 nodes, 2000 explicit / 200 BTCS steps,
    target from seed + 1. Every row: the FP32 gradient against the GPU FP64
    gradient within the row's bar (1e-4 on well-conditioned rows, see above).
    Sampled rows: the GPU FP64 gradient against the FP64 oracle at 1e-11, the
    FP32 one at the row's bar."""
    import torch

    from paper_2601_12204_b300.api import Batch
    from paper_2601_12204_b300.diagnostics import fp32_gradient_bar, trajectory_stats
    ens, tgt, dts, steps = _differentiation_problem(scheme)
    N = int(ens.ns[0])
    g64, n64 = _pipeline_grads(ctx, scheme, ens, tgt, dts, steps, F64)
    g64r, _ = _pipeline_grads(ctx, scheme, ens, tgt, dts, steps, F64, round_u0=True)
    g32, n32 = _pipeline_grads(ctx, scheme, ens, tgt, dts, steps, F32)
    G64, G32 = g64.view(ens.count, N), g32.view(ens.count, N)
    assert bool(torch.isfinite(G32).all()) and bool(torch.isfinite(n32).all())
    rel = ((G32 - G64).norm(dim=1) / G64.norm(dim=1)).cpu().numpy()
    stats = trajectory_stats(ctx, scheme, Batch.from_ensemble(ens, dts, steps, F64),
                             torch.tensor(ens.u0, dtype=torch.float64, device="cuda"), steps)
    a64, a32 = G64.cpu().numpy(), G32.cpu().numpy()
    bar = fp32_gradient_bar(a64, g64r.view(ens.count, N).cpu().numpy(), stats)
    bad = np.nonzero(rel > bar)[0]
    assert bad.size == 0, [(int(b), float(rel[b]), float(bar[b]), int(stats["flips"][b]))
                           for b in bad[:10]]
    assert np.mean(rel > 1e-4) <= WIDE_ROWS_MAX, f"{int(np.sum(rel > 1e-4))} rows above 1e-4"
    free = stats["flips"] == 0
    nd = (n32 - n64).abs().cpu().numpy()
    na = n64.abs().cpu().numpy()
    assert np.all(nd[free] <= 10 * bar[free] * na[free] + 1e-6 * na.max())
    # sampled rows against the oracle (both precisions of the GPU gradient)
    ids = np.array([0, 511, 1023])
    sub, subt = ens.subset(ids), tgt.subset(ids)
    subt.nus = sub.nus.copy()  # target: same scheme, nu, dt and steps, u0 from seed + 1
    g_sub = run_oracle(scheme, sub, dts[ids], steps) - run_oracle(scheme, subt, dts[ids], steps)
    ref, gnu_ref = _oracle_grads(scheme, sub, dts[ids], steps, g_sub)
    for j, b in enumerate(ids):
        r = ref[j * N:(j + 1) * N]
        assert oracle.rel_l2(a64[b], r) <= 1e-11, f"row {b} FP64"
        assert abs(float(n64[b]) - gnu_ref[j]) <= 1e-10 * abs(gnu_ref[j]) + 1e-13 * np.max(np.abs(gnu_ref))
        assert oracle.rel_l2(a32[b], r) <= bar[b], f"row {b} FP32"


@pytest.mark.parametrize("dtype", [F64, F32])
@pytest.mark.parametrize("bc", [W.PERIODIC, W.DIRICHLET])
def test_explicit_adjoint_exact_rows(ctx, dtype, bc):
    """Rows of exactly a kernel shape's capacity take the exact-row explicit
    adjoint kernel (split-state forward, folds on the global step index):
    oracle parity, and a gradient bitwise independent of the checkpoint
    stride (70 steps: segments that do not line up with the 32-step folds)."""
    ns = [32, 128, 512, 1024, 2048] + ([4096] if dtype == F32 else [])
    parts = []
    for n in ns:
        e = W.fourier_ensemble(2, n, seed=n + 5)
        e.bcs[:] = bc
        parts.append(e)
    counts = np.array([p.count for p in parts])
    lens = np.concatenate([p.ns for p in parts])
    offs = np.zeros(lens.size, np.int64)
    offs[1:] = np.cumsum(lens[:-1])
    cat = lambda k: np.concatenate([getattr(p, k) for p in parts])  # noqa: E731
    ens = W.Ensemble(cat("u0"), offs, lens, cat("bcs"), cat("dxs"), cat("nus"), cat("x0"),
                     cat("length"))
    assert counts.sum() == ens.count
    steps = 70
    dts, gT = _problem(ens, EXPLICIT, steps, 1.0)
    ref, gnu_ref = _oracle_grads(EXPLICIT, ens, dts, steps, gT)
    got, gnu = _gpu_grads(ctx, EXPLICIT, ens, dts, steps, gT, dtype)
    _check(ens, got, ref, gnu, gnu_ref, dtype, f"exact-row adjoint bc{bc}")
    for stride in (1, 7, 32, 70, 100):
        g2, n2 = _gpu_grads(ctx, EXPLICIT, ens, dts, steps, gT, dtype, stride)
        assert np.array_equal(got, g2) and np.array_equal(gnu, n2), f"stride {stride}"


def _long_rows(dtype, bc, salt):
    ns = [1000, 5000, 9000, 70001] + ([3000] if dtype == F64 else [])
    parts = []
    for i, n in enumerate(ns):
        e = W.fourier_ensemble(1, n, seed=n + salt + i)
        e.bcs[:] = bc
        parts.append(e)
    lens = np.concatenate([p.ns for p in parts])
    offs = np.zeros(lens.size, np.int64)
    offs[1:] = np.cumsum(lens[:-1])
    cat = lambda k: np.concatenate([getattr(p, k) for p in parts])  # noqa: E731
    return W.Ensemble(cat("u0"), offs, lens, cat("bcs"), cat("dxs"), cat("nus"), cat("x0"),
                      cat("length"))


@pytest.mark.parametrize("scheme", [EXPLICIT, BTCS])
@pytest.mark.parametrize("dtype", [F64, F32])
@pytest.mark.parametrize("bc", [W.PERIODIC, W.DIRICHLET])
def test_adjoint_long_rows(ctx, scheme, dtype, bc):
    """Rows longer than one CTA holds (FP32 > 4096, FP64 > 2048 nodes) take
    the long-row adjoint (explicit: one step per pass over tiles; BTCS: the
    BTCS plan one step per call and the transposed solves through the
    multi-level solver), beside a short row on the resident kernel in the
    same call: oracle parity with ragged step counts, a gradient bitwise
    independent of the checkpoint stride, and dJ/du0 written over dJ/du(T)."""
    import torch

    from paper_2601_12204_b300.api import Batch
    ens = _long_rows(dtype, bc, 11 if scheme == EXPLICIT else 23)
    steps = (np.array([30, 37, 50, 23, 41]) if scheme == EXPLICIT
             else np.array([9, 12, 7, 10, 5]))[:ens.count]
    dts, gT = _problem(ens, scheme, steps, 1.0 if scheme == EXPLICIT else 4.0)
    ref, gnu_ref = _oracle_grads(scheme, ens, dts, steps, gT)
    got, gnu = _gpu_grads(ctx, scheme, ens, dts, steps, gT, dtype)
    _check(ens, got, ref, gnu, gnu_ref, dtype, f"long-row adjoint s{scheme} bc{bc}",
           mass=_gnu_mass(ens, dts, steps, gT, dtype))
    for stride in (1, 4, 50):
        g2, n2 = _gpu_grads(ctx, scheme, ens, dts, steps, gT, dtype, stride)
        assert np.array_equal(got, g2) and np.array_equal(gnu, n2), f"stride {stride}"
    # dJ/du0 may overwrite dJ/du(T)
    tdt = torch.float32 if dtype == F32 else torch.float64
    b = Batch.from_ensemble(ens, dts, steps, dtype)
    u0 = torch.tensor(ens.u0, dtype=tdt, device="cuda")
    g = torch.tensor(gT, dtype=tdt, device="cuda")
    gn = torch.zeros(ens.count, dtype=torch.float64, device="cuda")
    ctx.adjoint(scheme, b, u0, g, g, gn, 0)
    torch.cuda.synchronize()
    assert np.array_equal(g.cpu().double().numpy(), got)
