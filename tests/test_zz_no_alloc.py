"""The explicit entry point that allocates no device memory.

burgers_explicit_advance_noalloc is for callers that cannot allocate device
memory while they run (an arena that already owns the GPU's memory, a fixed
footprint service, code called under another allocator's lock). It keeps its
working buffers in a fixed static device array. This file is collected last so
that a failure here cannot hide the results of the other GPU tests; it must
also pass when run alone in a fresh process, where its first call is the one
that looks up the array's device address.
"""
import ctypes

import numpy as np
import pytest

import oracle
from gpu_helpers import F32, F64, TOL, oracle_dts
from paper_2601_12204_b300 import _lib as L
from paper_2601_12204_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _row(n, bc, seed):
    x, dx = W.grid(n, bc, 0.0, W.TWO_PI)
    a, phi, nu = W.fourier_coeffs(seed, 7)
    u0 = W.fourier_field(x, a, phi)
    return W.Ensemble(u0, np.zeros(1, np.int64), np.array([n], np.int32), np.array([bc], np.int32),
                      np.array([dx]), np.array([nu]), np.zeros(1), np.array([W.TWO_PI]))


def test_noalloc_matches_the_allocating_entry_point_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_12204_b300.api import Batch, Context
    lib = L.load()
    ctx = Context(0)
    try:
        for dtype, tdt in ((F32, torch.float32), (F64, torch.float64)):
            # two calls in a row on different rows: the second must not see the
            # first one's leftovers in the shared array
            for n, bc, steps, seed in ((100_000, W.PERIODIC, 150, 1), (70_001, W.DIRICHLET, 97, 2)):
                e = _row(n, bc, seed)
                dts = oracle_dts(e)
                b = Batch.from_ensemble(e, dts, steps, dtype)
                ref = torch.tensor(e.u0, dtype=tdt, device="cuda")
                ctx.explicit_advance(b, ref)
                # place the row at an offset inside a larger buffer
                buf = torch.full((n + 37,), 3.5, dtype=tdt, device="cuda")
                buf[37:] = torch.tensor(e.u0, dtype=tdt, device="cuda")
                inst = L.burgers_instance(37, n, bc, float(e.dxs[0]), float(e.nus[0]),
                                          float(dts[0]), steps)
                stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
                st = lib.burgers_explicit_advance_noalloc(ctypes.byref(inst), dtype,
                                                          ctypes.c_void_p(buf.data_ptr()), stream)
                assert st == L.BURGERS_OK, L.last_error()
                torch.cuda.synchronize()
                got = buf[37:].cpu().double().numpy()
                want = ref.cpu().double().numpy()
                tol_rel, tol_abs = TOL[dtype]
                assert oracle.rel_l2(got, want) <= tol_rel
                assert np.max(np.abs(got - want)) <= tol_abs * np.max(np.abs(want))
                assert torch.all(buf[:37] == 3.5)
        # rows beyond the stated maximum are refused and left untouched
        big = torch.zeros((1 << 20) + 1, dtype=torch.float32, device="cuda")
        inst = L.burgers_instance(0, (1 << 20) + 1, 0, 0.01, 0.01, 1e-4, 5)
        st = lib.burgers_explicit_advance_noalloc(ctypes.byref(inst), F32,
                                                  ctypes.c_void_p(big.data_ptr()), None)
        assert st == L.BURGERS_EINVAL and "limit" in L.last_error()
        assert int(torch.count_nonzero(big)) == 0
    finally:
        ctx.close()
