"""Shared helpers of the GPU parity tests: run a packed ensemble through the
CUDA library and through the oracle on the same seeded inputs."""
import numpy as np

import oracle
from paper_2601_12204_b300 import _lib as L
from paper_2601_12204_b300.api import Batch

EXPLICIT, BTCS, RK4 = L.BURGERS_EXPLICIT, L.BURGERS_BTCS, L.BURGERS_RK4
CN, PICARD, NEWTON = L.BURGERS_CN, L.BURGERS_PICARD, L.BURGERS_NEWTON
F32, F64 = L.BURGERS_F32, L.BURGERS_F64

# Parity bars. FP64: relative L2 <= 1e-12 per row; elementwise |gpu - oracle|
# <= 1e-11 max|oracle| (rounding of a different but exact-arithmetic-equal
# evaluation order, accumulated over <= a few thousand contractive steps).
# FP32: relative L2 <= 1e-5 per row at t_final against the FP64 oracle;
# elementwise <= 1e-4 max|oracle|.
TOL = {F64: (1e-12, 1e-11), F32: (1e-5, 1e-4)}


def oracle_dts(ens, factor=1.0, cfl=0.4):
    return np.array([oracle.cfl_dt(ens.row(b), ens.dxs[b], ens.nus[b], cfl) * factor
                     for b in range(ens.count)])


def run_gpu(ctx, scheme, ens, dts, nsteps, dtype, u0=None, iters=1):
    import torch
    tdt = torch.float32 if dtype == F32 else torch.float64
    b = Batch.from_ensemble(ens, dts, nsteps, dtype)
    src = ens.u0 if u0 is None else u0
    u = torch.tensor(np.asarray(src, dtype=np.float64), dtype=tdt, device="cuda")
    ctx.advance(scheme, b, u, iters=iters)
    torch.cuda.synchronize()
    return u.cpu().double().numpy()


def run_oracle(scheme, ens, dts, nsteps, threads=0, iters=1):
    steps = np.broadcast_to(np.asarray(nsteps, dtype=np.int64), (ens.count,))
    if scheme in (PICARD, NEWTON):
        f = oracle.picard_batch if scheme == PICARD else oracle.newton_batch
        return f(ens.u0, ens.offsets, ens.ns, ens.bcs, ens.dxs, ens.nus, dts, steps, iters, threads)
    f = {EXPLICIT: oracle.explicit_batch, BTCS: oracle.btcs_batch, RK4: oracle.rk4_batch,
         CN: oracle.cn_batch}[scheme]
    return f(ens.u0, ens.offsets, ens.ns, ens.bcs, ens.dxs, ens.nus, dts, steps, threads)


def assert_parity(ens, got, ref, dtype, what=""):
    tol_rel, tol_abs = TOL[dtype]
    worst = 0.0
    for b in range(ens.count):
        o, n = int(ens.offsets[b]), int(ens.ns[b])
        g, r = got[o:o + n], ref[o:o + n]
        assert np.all(np.isfinite(g)), f"{what} row {b}: non-finite"
        rel = oracle.rel_l2(g, r)
        scale = max(1e-300, float(np.max(np.abs(r))))
        ab = float(np.max(np.abs(g - r))) / scale
        worst = max(worst, rel)
        assert rel <= tol_rel, f"{what} row {b} (n={n}, bc={ens.bcs[b]}): rel L2 {rel:.3e} > {tol_rel}"
        assert ab <= tol_abs, f"{what} row {b} (n={n}): max abs {ab:.3e} > {tol_abs}"
    return worst
