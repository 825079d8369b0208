"""GPU parity on the step initial condition of Eq. 20 (Sec. 3.4): a
discontinuous state whose right half is exactly zero, so the upwind tie
H(0) = 0 is taken at every node ahead of the front, and a jump that BTCS must
carry at time steps far above the explicit limit (dt = 5 dx / u_max and
25 dx / u_max). Every scheme, both precisions, both boundary conditions,
elementwise against the FP64 oracle; the explicit and BTCS adjoints on the
same fields against the oracle's discrete adjoints.

Not used: states that fold into a standing shock through u = 0 (for example
1, 0, -1 on thirds of a periodic row). There the node at the shock centre is
an unstable equilibrium of the advective upwind step (it grows by up to
1 + r u_left - 2s per step from any rounding residue), so two correct
implementations diverge: a 1e-12 perturbation of u0 changes the result by
2e-4 after 400 explicit steps on 201 nodes."""
import numpy as np
import pytest

import oracle
from gpu_helpers import (BTCS, CN, EXPLICIT, F32, F64, PICARD, RK4, assert_parity, oracle_dts,
                         run_gpu, run_oracle)
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


def step_ensemble(ns, bcs, pecs):
    """Packed rows of the Eq. 20 step (1 left of x = 1/2, 0 right of it) on
    [0, 1], n nodes each, with nu = u_max dx / Pe for the given cell Peclet
    numbers (Pe = inf: inviscid). Setting nu by the cell Peclet number keeps
    s = nu dt / dx^2 = (dt u_max / dx) / Pe moderate on long rows at the large
    time steps below: the tridiagonal system's condition number grows like
    1 + 4 s, and with it the rounding by which two exact solvers differ."""
    u, offs, dxs, nus = [], [], [], []
    o = 0
    for n, bc, pe in zip(ns, bcs, pecs):
        x, dx = W.grid(int(n), int(bc), 0.0, 1.0)
        u.append(np.where(x < 0.5, 1.0, 0.0))
        offs.append(o)
        dxs.append(dx)
        nus.append(0.0 if np.isinf(pe) else dx / pe)
        o += int(n)
    m = len(ns)
    return W.Ensemble(np.concatenate(u), np.array(offs, np.int64), np.array(ns, np.int32),
                      np.array(bcs, np.int32), np.array(dxs), np.array(nus, np.float64),
                      np.zeros(m), np.ones(m))


PECLET = (np.inf, 20.0, 2.0)


def _rows(lengths):
    ns, bcs, pecs = [], [], []
    for i, n in enumerate(lengths):
        for bc in (W.DIRICHLET, W.PERIODIC):
            for k in range(2):
                ns.append(n)
                bcs.append(bc)
                pecs.append(PECLET[(i + bc + k) % 3])
    return step_ensemble(ns, bcs, pecs)


# rows on the resident paths, ragged ones, the cluster BTCS path (FP32, 20000
# nodes) and the streaming / multi-level paths (70001 nodes)
LONG = [201, 1000, 4097, 20000, 70001]
# Crank-Nicolson and Picard rows stay within one CTA (8192 FP32 / 4096 FP64 nodes)
SHORT = [201, 1000, 4000]

# (scheme, iterations, dt in units of dx / u_max (0: the explicit CFL-0.4 step), steps, lengths)
CASES = [
    (EXPLICIT, 1, 0.0, 400, LONG),
    (RK4, 1, 0.0, 200, LONG),
    (BTCS, 1, 5.0, 30, LONG),
    (BTCS, 1, 25.0, 8, LONG),
    (CN, 1, 5.0, 30, SHORT),
    (PICARD, 3, 5.0, 20, SHORT),
]


@pytest.mark.parametrize("dtype", [F64, F32])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"s{c[0]}i{c[1]}dt{c[2]:g}")
def test_step_ic_parity(ctx, case, dtype):
    scheme, iters, dtf, steps, lengths = case
    ens = _rows(lengths)
    umax = 1.0
    if dtf == 0.0:
        dts = oracle_dts(ens)
    else:
        dts = dtf * ens.dxs / umax
    ref = run_oracle(scheme, ens, dts, steps, iters=iters)
    got = run_gpu(ctx, scheme, ens, dts, steps, dtype, iters=iters)
    assert_parity(ens, got, ref, dtype, f"step IC s{scheme} dt {dtf}")
    if scheme in (BTCS, PICARD):
        # the M-matrix keeps the solution within the range of the data (Sec. 3.4)
        assert got.min() >= -1.0 - 1e-6 and got.max() <= 1.0 + 1e-6


def _adjoint_problem(ens, scheme, steps, dts):
    shifted = ens.subset(np.arange(ens.count))
    for b in range(ens.count):
        o, n = ens.offsets[b], ens.ns[b]
        x, _ = W.grid(int(n), int(ens.bcs[b]), 0.0, 1.0)
        shifted.u0[o:o + n] = np.where(x < 0.4, 1.0, 0.0)
    return run_oracle(scheme, ens, dts, steps) - run_oracle(scheme, shifted, dts, steps)


@pytest.mark.parametrize("dtype", [F64, F32])
@pytest.mark.parametrize("scheme", [EXPLICIT, BTCS])
def test_step_ic_adjoint(ctx, scheme, dtype):
    """dJ/du0 and dJ/dnu through solves from step fields (exact zeros over whole
    regions, so the transposed steps take H(0) = 0 at every node ahead of the
    front) against the oracle's discrete adjoint; J = 1/2 |u(T) - target|^2,
    target from the step moved to x = 0.4."""
    import torch

    from paper_2601_12204_b300.api import Batch
    ns = [201, 1000, 2048]
    rows = [(n, bc) for n in ns for bc in (W.DIRICHLET, W.PERIODIC)]
    ens = step_ensemble([r[0] for r in rows], [r[1] for r in rows],
                        [PECLET[1 + i % 2] for i in range(len(rows))])
    steps = 60 if scheme == EXPLICIT else 20
    dts = oracle_dts(ens) if scheme == EXPLICIT else 5.0 * ens.dxs
    gT = _adjoint_problem(ens, scheme, steps, dts)
    f = oracle.explicit_adjoint if scheme == EXPLICIT else oracle.btcs_adjoint
    tdt = torch.float32 if dtype == F32 else torch.float64
    b = Batch.from_ensemble(ens, dts, steps, dtype)
    u0 = torch.tensor(ens.u0, dtype=tdt, device="cuda")
    g = torch.tensor(gT, dtype=tdt, device="cuda")
    gu0 = torch.zeros_like(u0)
    gnu = torch.zeros(ens.count, dtype=torch.float64, device="cuda")
    ctx.adjoint(scheme, b, u0, g, gu0, gnu)
    torch.cuda.synchronize()
    got, gotn = gu0.cpu().double().numpy(), gnu.cpu().numpy()
    tu, tn = (1e-11, 1e-10) if dtype == F64 else (1e-4, 1e-3)
    refn = []
    for i in range(ens.count):
        o, n = ens.offsets[i], ens.ns[i]
        ref, rn = f(ens.u0[o:o + n], ens.bcs[i], ens.dxs[i], ens.nus[i], dts[i], steps, gT[o:o + n])
        refn.append(rn)
        rel = oracle.rel_l2(got[o:o + n], ref)
        assert rel <= tu, f"row {i} (n={n}, bc={ens.bcs[i]}): dJ/du0 rel L2 {rel:.3e}"
    refn = np.array(refn)
    floor = (1e-13 if dtype == F64 else 1e-6) * float(np.max(np.abs(refn)))
    assert np.all(np.abs(gotn - refn) <= tn * np.abs(refn) + floor)
