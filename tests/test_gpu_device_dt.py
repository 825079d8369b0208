"""The device-side time step (burgers_cfl_dt_device) and the advance that
reads it on the device (burgers_advance_dt_device): bitwise the host-dt path
(CFL step of Eq. 7-8 brought to the host, then the host-dt advance), which
the parity tests pin to the FP64 oracle."""
import numpy as np
import pytest

from gpu_helpers import BTCS, CN, EXPLICIT, F32, F64, RK4
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


def _concat(parts):
    ns = np.concatenate([p.ns for p in parts])
    offs = np.zeros(ns.size, np.int64)
    offs[1:] = np.cumsum(ns[:-1])
    cat = lambda k: np.concatenate([getattr(p, k) for p in parts])  # noqa: E731
    return W.Ensemble(cat("u0"), offs, ns, cat("bcs"), cat("dxs"), cat("nus"), cat("x0"),
                      cat("length"))


def _one(n, bc, seed):
    x, dx = W.grid(n, bc, 0.0, W.TWO_PI)
    a, phi, nu = W.fourier_coeffs(seed, 96)
    return W.Ensemble(W.fourier_field(x, a, phi), np.zeros(1, np.int64), np.array([n], np.int32),
                      np.array([bc], np.int32), np.array([dx]), np.array([nu]), np.zeros(1),
                      np.array([W.TWO_PI]))


@pytest.mark.parametrize("scheme,factor", [(EXPLICIT, 1.0), (BTCS, 10.0), (RK4, 1.0), (CN, 8.0)])
@pytest.mark.parametrize("dtype", [F64, F32])
def test_device_dt_matches_host_dt(ctx, scheme, factor, dtype):
    import torch
    from paper_2601_12204_b300.api import Batch
    # rows the host path also takes: FP64 implicit rows stay within one CTA
    # (4096 nodes), CN rows are resident only; long rows stream (explicit,
    # RK4) or stay in a cluster (FP32 BTCS)
    wide = dtype == F32 or scheme in (EXPLICIT, RK4)
    ens = W.mixed_ensemble(30, 3, 5000 if wide else 4000, seed=41)
    extra = [20000, 40000] if (scheme in (EXPLICIT, RK4) or (scheme == BTCS and dtype == F32)) else []
    ens = _concat([ens] + [_one(n, bc, seed=n + bc) for n in extra for bc in (0, 1)])
    steps = np.random.default_rng(5).integers(1, 60, ens.count)
    tdt = torch.float32 if dtype == F32 else torch.float64
    u0 = torch.tensor(ens.u0, dtype=tdt, device="cuda")
    probe = Batch.from_ensemble(ens, 1.0, 0, dtype)
    dt_host = ctx.cfl_dt(probe, u0, 0.4)
    b_host = Batch.from_ensemble(ens, dt_host * factor, steps, dtype)
    want = u0.clone()
    ctx.advance(scheme, b_host, want)
    dtd = torch.empty(ens.count, dtype=torch.float64, device="cuda")
    got = u0.clone()
    b_dev = Batch.from_ensemble(ens, 1.0, steps, dtype)  # dt ignored
    ctx.cfl_dt_device(b_dev, got, 0.4, dtd)
    ctx.advance_dt_device(scheme, b_dev, got, dtd, factor)
    torch.cuda.synchronize()
    assert np.array_equal(dtd.cpu().numpy(), dt_host)
    assert torch.equal(got, want)
    # a second call reuses the cached reduction descriptors and plan
    got2 = u0.clone()
    ctx.cfl_dt_device(b_dev, got2, 0.4, dtd)
    ctx.advance_dt_device(scheme, b_dev, got2, dtd, factor)
    torch.cuda.synchronize()
    assert torch.equal(got2, want)


def test_device_dt_rows_without_limit_stay(ctx):
    """u == 0 and nu == 0: no finite CFL limit, dt = -1, row left as it is;
    the other rows advance as with the host path."""
    import torch
    from paper_2601_12204_b300.api import Batch
    ens = W.mixed_ensemble(6, 50, 900, seed=42)
    o, n = int(ens.offsets[2]), int(ens.ns[2])
    ens.u0[o:o + n] = 0.0
    ens.nus[2] = 0.0
    u0 = torch.tensor(ens.u0, device="cuda")
    b = Batch.from_ensemble(ens, 1.0, 25, F64)
    dtd = torch.empty(ens.count, dtype=torch.float64, device="cuda")
    got = u0.clone()
    ctx.cfl_dt_device(b, got, 0.4, dtd)
    ctx.advance_dt_device(EXPLICIT, b, got, dtd, 1.0)
    torch.cuda.synchronize()
    d = dtd.cpu().numpy()
    assert d[2] == -1.0 and np.all(np.delete(d, 2) > 0)
    assert torch.equal(got[o:o + n], u0[o:o + n])
    rest = [i for i in range(ens.count) if i != 2]
    sub = ens.subset(np.array(rest))
    u_sub = torch.tensor(sub.u0, device="cuda")
    bs = Batch.from_ensemble(sub, d[rest], 25, F64)
    ctx.advance(EXPLICIT, bs, u_sub)
    torch.cuda.synchronize()
    for j, i in enumerate(rest):
        oi, ni = int(ens.offsets[i]), int(ens.ns[i])
        oj = int(sub.offsets[j])
        assert torch.equal(got[oi:oi + ni], u_sub[oj:oj + ni])


def test_device_dt_rejections(ctx):
    """Rows for the multi-level solver (FP64 BTCS beyond one CTA), a bad
    factor and a short dt tensor are refused before any work is queued."""
    import torch
    from paper_2601_12204_b300.api import Batch
    e = _one(20000, 0, 3)
    u = torch.tensor(e.u0, device="cuda")
    b = Batch.from_ensemble(e, 1.0, 3, F64)
    dtd = torch.full((1,), 1e-4, dtype=torch.float64, device="cuda")
    before = u.clone()
    with pytest.raises(Exception):
        ctx.advance_dt_device(BTCS, b, u, dtd, 1.0)
    with pytest.raises(Exception):
        ctx.advance_dt_device(EXPLICIT, b, u, dtd, 0.0)
    with pytest.raises(Exception):
        ctx.advance_dt_device(EXPLICIT, b, u, torch.empty(0, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    assert torch.equal(u, before)
