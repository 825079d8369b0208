"""The explicit entry point that allocates no device memory.

burgers_explicit_advance_noalloc is for callers that cannot allocate device
memory while they run (an arena that already owns the GPU's memory, a fixed
footprint service, code called under another allocator's lock). It keeps its
working buffers in a fixed static device array. This file is collected last so
that a failure here cannot hide the results of the other GPU tests; it must
also pass when run alone in a fresh process, where its first call is the one
that loads the library's module on the device.
"""
import ctypes

import numpy as np
import pytest

import oracle
from gpu_helpers import F32, F64, TOL, oracle_dts
from paper_2601_12204_b300 import _lib as L
from paper_2601_12204_b300 import workloads as W

pytestmark = pytest.mark.gpu

PAD = 37  # the row sits at this offset inside a larger buffer


def _row(n, bc, seed):
    x, dx = W.grid(n, bc, 0.0, W.TWO_PI)
    a, phi, nu = W.fourier_coeffs(seed, 7)
    u0 = W.fourier_field(x, a, phi)
    return W.Ensemble(u0, np.zeros(1, np.int64), np.array([n], np.int32), np.array([bc], np.int32),
                      np.array([dx]), np.array([nu]), np.zeros(1), np.array([W.TWO_PI]))


# (n, bc, steps, seed): two long rows (256-thread windows) and short ones
# (32 x 4 windows, 128 <= n < 4096)
ROWS = [(100_000, W.PERIODIC, 150, 1), (70_001, W.DIRICHLET, 97, 2), (128, W.PERIODIC, 90, 3),
        (1000, W.DIRICHLET, 120, 4), (3000, W.PERIODIC, 75, 5), (3000, W.DIRICHLET, 40, 6)]


def _noalloc(lib, torch, e, dt, steps, dtype, buf):
    inst = L.burgers_instance(PAD, int(e.ns[0]), int(e.bcs[0]), float(e.dxs[0]), float(e.nus[0]),
                              float(dt), int(steps))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.burgers_explicit_advance_noalloc(ctypes.byref(inst), dtype,
                                                ctypes.c_void_p(buf.data_ptr()), stream)


def _check(got, want, dtype):
    tol_rel, tol_abs = TOL[dtype]
    assert oracle.rel_l2(got, want) <= tol_rel
    assert np.max(np.abs(got - want)) <= tol_abs * np.max(np.abs(want))


def test_noalloc_matches_the_oracle_and_the_allocating_entry_point():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = L.load()
    for dtype, tdt in ((F32, torch.float32), (F64, torch.float64)):
        # every buffer exists before the calls, so nothing else allocates in between
        cases = []
        for n, bc, steps, seed in ROWS:
            e = _row(n, bc, seed)
            dt = float(oracle_dts(e)[0])
            buf = torch.full((n + PAD,), 3.5, dtype=tdt, device="cuda")
            buf[PAD:] = torch.tensor(e.u0, dtype=tdt, device="cuda")
            ref = oracle.explicit(e.u0, int(bc), float(e.dxs[0]), float(e.nus[0]), dt, steps)
            cases.append((e, dt, steps, buf, ref))
        torch.cuda.synchronize()
        # calls in a row on different rows, before any context exists in this
        # test: none may see an earlier call's leftovers in the shared array.
        # The first long-row and short-row calls load their kernels (lazy module
        # loading may place their code in device memory); after them the device's
        # free memory must not change
        first = [0, 2]
        for i in first:
            e, dt, steps, buf, ref = cases[i]
            assert _noalloc(lib, torch, e, dt, steps, dtype, buf) == L.BURGERS_OK, L.last_error()
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        for i, (e, dt, steps, buf, ref) in enumerate(cases):
            if i not in first:
                assert _noalloc(lib, torch, e, dt, steps, dtype, buf) == L.BURGERS_OK, L.last_error()
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, f"free device memory changed by {free0 - free1} bytes"
        for e, dt, steps, buf, ref in cases:
            assert torch.all(buf[:PAD] == 3.5)
            _check(buf[PAD:].cpu().double().numpy(), ref, dtype)
    # against the allocating entry point (same rows and steps)
    from paper_2601_12204_b300.api import Batch, Context
    ctx = Context(0)
    try:
        for dtype, tdt in ((F32, torch.float32), (F64, torch.float64)):
            for n, bc, steps, seed in ROWS:
                e = _row(n, bc, seed)
                dts = oracle_dts(e)
                b = Batch.from_ensemble(e, dts, steps, dtype)
                want = torch.tensor(e.u0, dtype=tdt, device="cuda")
                ctx.explicit_advance(b, want)
                buf = torch.full((n + PAD,), 3.5, dtype=tdt, device="cuda")
                buf[PAD:] = torch.tensor(e.u0, dtype=tdt, device="cuda")
                assert _noalloc(lib, torch, e, dts[0], steps, dtype, buf) == L.BURGERS_OK
                torch.cuda.synchronize()
                _check(buf[PAD:].cpu().double().numpy(), want.cpu().double().numpy(), dtype)
        # rows beyond the stated maximum are refused and left untouched
        big = torch.zeros((1 << 20) + 1, dtype=torch.float32, device="cuda")
        inst = L.burgers_instance(0, (1 << 20) + 1, 0, 0.01, 0.01, 1e-4, 5)
        st = lib.burgers_explicit_advance_noalloc(ctypes.byref(inst), F32,
                                                  ctypes.c_void_p(big.data_ptr()), None)
        assert st == L.BURGERS_EINVAL and "limit" in L.last_error()
        assert int(torch.count_nonzero(big)) == 0
    finally:
        ctx.close()
