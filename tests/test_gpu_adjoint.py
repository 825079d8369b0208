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


def _check(ens, got, ref, gnu, gnu_ref, dtype, what):
    tu, tn, tf = GTOL[dtype]
    floor = tf * float(np.max(np.abs(gnu_ref)))
    for b in range(ens.count):
        o, n = ens.offsets[b], ens.ns[b]
        rel = oracle.rel_l2(got[o:o + n], ref[o:o + n])
        assert rel <= tu, f"{what} row {b} (n={n}, bc={ens.bcs[b]}): dJ/du0 rel L2 {rel:.3e}"
        assert abs(gnu[b] - gnu_ref[b]) <= tn * abs(gnu_ref[b]) + floor, \
            f"{what} row {b}: dJ/dnu {gnu[b]!r} vs {gnu_ref[b]!r}"


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


@pytest.mark.parametrize("scheme", [EXPLICIT, BTCS])
def test_differentiation_1024x2048_sampled(ctx, scheme):
    """B = 1024 periodic rows x 2048 nodes, FP32, 2000 explicit / 200 BTCS steps,
    target from seed + 1: sampled rows against the FP64 oracle gradient."""
    B, N = 1024, 2048
    ens = W.fourier_ensemble(B, N, seed=W.DEFAULT_SEED)
    tgt = W.fourier_ensemble(B, N, seed=W.DEFAULT_SEED + 1)
    steps = 2000 if scheme == EXPLICIT else 200
    # one dt per row stable for both runs: the target's u0 (seed + 1) can be
    # larger, and a dt set by the CFL limit of u0 alone can make it diverge
    dts = np.minimum(oracle_dts(ens, 1.0 if scheme == EXPLICIT else 10.0),
                     oracle_dts(W.Ensemble(tgt.u0, ens.offsets, ens.ns, ens.bcs, ens.dxs, ens.nus,
                                           ens.x0, ens.length), 1.0 if scheme == EXPLICIT else 10.0))
    # gT: the misfit gradient u(T) - target on the sampled rows (oracle forward
    # solves from seed and seed + 1); any seeded field on the other rows (rows are
    # independent, so it does not affect the sampled ones)
    ids = np.array([0, 511, 1023])
    sub, subt = ens.subset(ids), tgt.subset(ids)
    subt.nus = sub.nus.copy()  # target: same scheme, nu, dt and steps, u0 from seed + 1
    g_sub = run_oracle(scheme, sub, dts[ids], steps) - run_oracle(scheme, subt, dts[ids], steps)
    gT = W.rng(99, 0).normal(0.0, 0.1, ens.u0.size)
    for j, b in enumerate(ids):
        gT[ens.offsets[b]:ens.offsets[b] + N] = g_sub[j * N:(j + 1) * N]
    got, gnu = _gpu_grads(ctx, scheme, ens, dts, steps, gT, F32)
    ref, gnu_ref = _oracle_grads(scheme, sub, dts[ids], steps, g_sub)
    for j, b in enumerate(ids):
        o = ens.offsets[b]
        rel = oracle.rel_l2(got[o:o + N], ref[j * N:(j + 1) * N])
        assert rel <= 1e-4, f"row {b}: {rel}"
        assert abs(gnu[b] - gnu_ref[j]) <= 1e-3 * abs(gnu_ref[j]) + 1e-6 * np.max(np.abs(gnu_ref))


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
