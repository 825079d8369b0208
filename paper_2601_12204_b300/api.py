"""Python front end of libburgers: batches, a context wrapper, torch tensors.

PyTorch provides device memory and streams; every solver step runs in the
library's CUDA kernels. Tensors are passed by pointer on the current torch
stream of their device.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np

from . import _lib as L

DTYPES = {L.BURGERS_F32: np.float32, L.BURGERS_F64: np.float64}


def _torch():
    import torch
    return torch


class Batch:
    """A packed batch of rows (mirror of burgers_batch)."""

    def __init__(self, dtype: int, offsets, ns, bcs, dxs, nus, dts, nsteps):
        offsets = np.asarray(offsets, dtype=np.int64).ravel()
        count = offsets.size
        arr = np.zeros(count, dtype=L.INSTANCE_DTYPE)
        arr["offset"] = offsets
        arr["n"] = np.broadcast_to(np.asarray(ns, dtype=np.int32), (count,))
        arr["bc"] = np.broadcast_to(np.asarray(bcs, dtype=np.int32), (count,))
        arr["dx"] = np.broadcast_to(np.asarray(dxs, dtype=np.float64), (count,))
        arr["nu"] = np.broadcast_to(np.asarray(nus, dtype=np.float64), (count,))
        arr["dt"] = np.broadcast_to(np.asarray(dts, dtype=np.float64), (count,))
        arr["nsteps"] = np.broadcast_to(np.asarray(nsteps, dtype=np.int64), (count,))
        self.arr = np.ascontiguousarray(arr)
        self.dtype = int(dtype)
        self._c = L.burgers_batch(self.dtype, 0, count, self.arr.ctypes.data)

    @classmethod
    def from_ensemble(cls, ens, dts, nsteps, dtype: int = L.BURGERS_F32) -> "Batch":
        return cls(dtype, ens.offsets, ens.ns, ens.bcs, ens.dxs, ens.nus, dts, nsteps)

    @property
    def count(self) -> int:
        return int(self.arr.size)

    @property
    def span(self) -> int:
        if self.count == 0:
            return 0
        return int(np.max(self.arr["offset"] + self.arr["n"]))

    def ref(self):
        return ctypes.byref(self._c)

    def with_fields(self, **kw) -> "Batch":
        a = self.arr
        f = {k: a[k] for k in ("offset", "n", "bc", "dx", "nu", "dt", "nsteps")}
        f.update(kw)
        return Batch(kw.get("dtype", self.dtype), f["offset"], f["n"], f["bc"], f["dx"], f["nu"],
                     f["dt"], f["nsteps"])


class Context:
    """Owns a burgers_ctx on one CUDA device."""

    def __init__(self, device: int = 0):
        self._lib = L.load()
        h = ctypes.c_void_p()
        L.check(self._lib.burgers_ctx_create(int(device), ctypes.byref(h)), "burgers_ctx_create")
        self.h = h
        self.device = int(device)

    def close(self) -> None:
        if getattr(self, "h", None) is not None and self.h.value:
            self._lib.burgers_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- helpers ----------------------------------------------------------
    def _stream(self, stream, t=None):
        if stream is not None:
            return ctypes.c_void_p(int(stream))
        torch = _torch()
        dev = t.device if t is not None else torch.device("cuda", self.device)
        return ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)

    def _check_tensor(self, t, batch: Batch, dtype: Optional[int] = None):
        torch = _torch()
        want = {L.BURGERS_F32: torch.float32, L.BURGERS_F64: torch.float64}[
            batch.dtype if dtype is None else dtype]
        if not t.is_cuda or t.device.index != self.device:
            raise ValueError("tensor must live on the context's CUDA device")
        if t.dtype != want:
            raise ValueError(f"tensor dtype {t.dtype} does not match batch dtype {want}")
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if t.numel() < batch.span:
            raise ValueError("tensor is smaller than the batch span")
        return ctypes.c_void_p(t.data_ptr())

    # -- entry points -------------------------------------------------------
    def set(self, option: int, value: int) -> None:
        L.check(self._lib.burgers_ctx_set(self.h, int(option), int(value)), "burgers_ctx_set")

    def get(self, key: int) -> int:
        v = ctypes.c_int64(0)
        L.check(self._lib.burgers_ctx_get(self.h, int(key), ctypes.byref(v)), "burgers_ctx_get")
        return int(v.value)

    def launch_count(self) -> int:
        return int(self._lib.burgers_launch_count(self.h))

    def device_error(self, clear: bool = False) -> int:
        """The context's device error word (blocking); bit 0: a bounded wait
        inside a kernel gave up."""
        v = ctypes.c_int32(0)
        L.check(self._lib.burgers_device_error(self.h, ctypes.byref(v), int(bool(clear))),
                "burgers_device_error")
        return int(v.value)

    def explicit_advance(self, batch: Batch, u, stream=None) -> None:
        p = self._check_tensor(u, batch)
        L.check(self._lib.burgers_explicit_advance(self.h, batch.ref(), p, self._stream(stream, u)),
                "burgers_explicit_advance")

    def btcs_advance(self, batch: Batch, u, stream=None) -> None:
        p = self._check_tensor(u, batch)
        L.check(self._lib.burgers_btcs_advance(self.h, batch.ref(), p, self._stream(stream, u)),
                "burgers_btcs_advance")

    def rk4_advance(self, batch: Batch, u, stream=None) -> None:
        """Classical RK4 in time (Eq. 22) on the explicit step's operator."""
        p = self._check_tensor(u, batch)
        L.check(self._lib.burgers_rk4_advance(self.h, batch.ref(), p, self._stream(stream, u)),
                "burgers_rk4_advance")

    def cn_advance(self, batch: Batch, u, stream=None) -> None:
        """Crank-Nicolson with lagged upwind coefficients (resident rows)."""
        p = self._check_tensor(u, batch)
        L.check(self._lib.burgers_cn_advance(self.h, batch.ref(), p, self._stream(stream, u)),
                "burgers_cn_advance")

    def picard_advance(self, batch: Batch, u, iters: int, stream=None) -> None:
        """Implicit upwind step, `iters` Picard iterations per step (resident rows)."""
        p = self._check_tensor(u, batch)
        L.check(self._lib.burgers_picard_advance(self.h, batch.ref(), p, int(iters),
                                                 self._stream(stream, u)),
                "burgers_picard_advance")

    def newton_advance(self, batch: Batch, u, iters: int, stream=None) -> None:
        """Eq. 11 implicit step, `iters` Newton iterations per step (resident rows)."""
        p = self._check_tensor(u, batch)
        L.check(self._lib.burgers_newton_advance(self.h, batch.ref(), p, int(iters),
                                                 self._stream(stream, u)),
                "burgers_newton_advance")

    def advance(self, scheme: int, batch: Batch, u, stream=None, iters: int = 1) -> None:
        if scheme == L.BURGERS_EXPLICIT:
            self.explicit_advance(batch, u, stream)
        elif scheme == L.BURGERS_RK4:
            self.rk4_advance(batch, u, stream)
        elif scheme == L.BURGERS_BTCS:
            self.btcs_advance(batch, u, stream)
        elif scheme == L.BURGERS_CN:
            self.cn_advance(batch, u, stream)
        elif scheme == L.BURGERS_PICARD:
            self.picard_advance(batch, u, iters, stream)
        elif scheme == L.BURGERS_NEWTON:
            self.newton_advance(batch, u, iters, stream)
        else:
            raise ValueError(f"unknown scheme {scheme}")

    def cfl_dt(self, batch: Batch, u, cfl: float = 0.4, stream=None) -> np.ndarray:
        p = self._check_tensor(u, batch)
        out = np.zeros(batch.count, dtype=np.float64)
        L.check(self._lib.burgers_cfl_dt(self.h, batch.ref(), p, float(cfl),
                                         out.ctypes.data_as(ctypes.c_void_p),
                                         self._stream(stream, u)), "burgers_cfl_dt")
        return out

    def _check_dt(self, dt, batch: Batch) -> ctypes.c_void_p:
        torch = _torch()
        if (not dt.is_cuda or dt.dtype != torch.float64 or not dt.is_contiguous()
                or dt.numel() < batch.count):
            raise ValueError("dt must be a contiguous CUDA float64 tensor with one entry per row")
        return ctypes.c_void_p(dt.data_ptr())

    def cfl_dt_device(self, batch: Batch, u, cfl: float, dt, stream=None) -> None:
        """dt[b] = cfl * min(dx/max|u_b|, dx^2/(2 nu_b)) on the device, asynchronously
        (dt: CUDA float64 tensor, one entry per row; -1 where no limit is finite)."""
        p = self._check_tensor(u, batch)
        L.check(self._lib.burgers_cfl_dt_device(self.h, batch.ref(), p, float(cfl),
                                                self._check_dt(dt, batch),
                                                self._stream(stream, u)), "burgers_cfl_dt_device")

    def advance_dt_device(self, scheme: int, batch: Batch, u, dt, factor: float = 1.0,
                          iters: int = 1, stream=None) -> None:
        """Advances every row by its nsteps steps with dt_b = factor * dt[b] read on
        the device (the batch's dt is ignored); no host synchronisation."""
        p = self._check_tensor(u, batch)
        L.check(self._lib.burgers_advance_dt_device(self.h, int(scheme), batch.ref(), p,
                                                    self._check_dt(dt, batch), float(factor),
                                                    int(iters), self._stream(stream, u)),
                "burgers_advance_dt_device")

    def fma_peak(self, dtype: int = L.BURGERS_F32) -> float:
        """Measured FMA issue rate of the device (lane-FMAs per second) for dtype,
        at the clock the GPU runs during the call."""
        out = ctypes.c_double(0.0)
        L.check(self._lib.burgers_fma_peak(self.h, int(dtype), ctypes.byref(out)),
                "burgers_fma_peak")
        return float(out.value)

    def rel_l2(self, batch: Batch, u, ref, stream=None):
        torch = _torch()
        p = self._check_tensor(u, batch)
        rdt = L.BURGERS_F64 if ref.dtype == torch.float64 else L.BURGERS_F32
        q = self._check_tensor(ref, batch, rdt)
        rel = np.zeros(batch.count)
        rms = np.zeros(batch.count)
        L.check(self._lib.burgers_rel_l2(self.h, batch.ref(), p, q, rdt,
                                         rel.ctypes.data_as(ctypes.c_void_p),
                                         rms.ctypes.data_as(ctypes.c_void_p),
                                         self._stream(stream, u)), "burgers_rel_l2")
        return rel, rms

    def adjoint(self, scheme: int, batch: Batch, u0, gT, gu0, gnu, ckpt_stride: int = 0,
                stream=None) -> None:
        """dJ/du0 into gu0 and dJ/dnu (FP64, one per row) into gnu, given gT = dJ/du(T)."""
        torch = _torch()
        a = self._check_tensor(u0, batch)
        g = self._check_tensor(gT, batch)
        o = self._check_tensor(gu0, batch)
        if (not gnu.is_cuda or gnu.dtype != torch.float64 or gnu.numel() < batch.count
                or not gnu.is_contiguous()):
            raise ValueError("gnu must be a contiguous CUDA float64 tensor with one entry per row")
        L.check(self._lib.burgers_adjoint(self.h, int(scheme), batch.ref(), a, g, o,
                                          ctypes.c_void_p(gnu.data_ptr()), int(ckpt_stride),
                                          self._stream(stream, u0)), "burgers_adjoint")

    def autotune(self, scheme: int, batch: Batch, u, probe_steps: int = 50, stream=None) -> int:
        """Times the kernel shapes of the batch's capacity classes on a copy of
        its rows and keeps the fastest; returns the number of classes tuned."""
        p = self._check_tensor(u, batch)
        n = ctypes.c_int32(0)
        L.check(self._lib.burgers_autotune(self.h, int(scheme), batch.ref(), p, int(probe_steps),
                                           ctypes.byref(n), self._stream(stream, u)),
                "burgers_autotune")
        return int(n.value)

    def tune_save(self, path: str) -> None:
        L.check(self._lib.burgers_tune_save(self.h, str(path).encode()), "burgers_tune_save")

    def tune_load(self, path: str) -> None:
        L.check(self._lib.burgers_tune_load(self.h, str(path).encode()), "burgers_tune_load")

    def solve_host(self, scheme: int, batch: Batch, u_host, stream=None) -> None:
        """In-place solve of a host buffer (numpy array or CPU tensor)."""
        if isinstance(u_host, np.ndarray):
            if u_host.dtype != DTYPES[batch.dtype] or not u_host.flags.c_contiguous:
                raise ValueError("host array dtype/contiguity mismatch")
            ptr = u_host.ctypes.data
            n = u_host.size
        else:
            torch = _torch()
            want = torch.float32 if batch.dtype == L.BURGERS_F32 else torch.float64
            if u_host.is_cuda or u_host.dtype != want or not u_host.is_contiguous():
                raise ValueError("host tensor dtype/device/contiguity mismatch")
            ptr = u_host.data_ptr()
            n = u_host.numel()
        if n < batch.span:
            raise ValueError("host buffer is smaller than the batch span")
        L.check(self._lib.burgers_solve_host(self.h, int(scheme), batch.ref(), ctypes.c_void_p(ptr),
                                             self._stream(stream)), "burgers_solve_host")


class Server:
    """Continuous-batching server over a Context (burgers_serve_*)."""

    def __init__(self, ctx: Context, dtype: int = L.BURGERS_F32, hbm_budget: int = 0,
                 slice_steps: int = 256, max_active: int = 0, slice_timeout_s: float = 60.0):
        self._lib = ctx._lib
        self.ctx = ctx
        self.dtype = int(dtype)
        self.np_dtype = DTYPES[self.dtype]
        cfg = L.burgers_serve_cfg(self.dtype, 0, int(max_active), int(hbm_budget),
                                  int(slice_steps), float(slice_timeout_s))
        h = ctypes.c_void_p()
        L.check(self._lib.burgers_serve_create(ctx.h, ctypes.byref(cfg), ctypes.byref(h)),
                "burgers_serve_create")
        self.h = h

    def submit(self, scheme: int, bc: int, u0, dx: float, nu: float, dt: float, nsteps: int) -> int:
        a = np.ascontiguousarray(u0, dtype=self.np_dtype)
        rq = L.burgers_request(int(scheme), int(bc), int(a.size), 0, float(dx), float(nu), float(dt),
                               int(nsteps), a.ctypes.data)
        t = ctypes.c_uint64(0)
        L.check(self._lib.burgers_serve_submit(self.h, ctypes.byref(rq), ctypes.byref(t)),
                "burgers_serve_submit")
        return int(t.value)

    def _submit_ptr(self, scheme: int, bc: int, n: int, u0_ptr: int, dx: float, nu: float,
                    dt: float, nsteps: int) -> int:
        """submit() from a raw host pointer to n values of the server dtype."""
        rq = L.burgers_request(int(scheme), int(bc), int(n), 0, float(dx), float(nu), float(dt),
                               int(nsteps), int(u0_ptr))
        t = ctypes.c_uint64(0)
        L.check(self._lib.burgers_serve_submit(self.h, ctypes.byref(rq), ctypes.byref(t)),
                "burgers_serve_submit")
        return int(t.value)

    def submit_timed(self, reqs, t_arrive):
        """Replays a trace from native code: reqs is a ctypes array of
        burgers_request, t_arrive the arrival times in seconds after the call
        (float64). Blocks until every request is submitted; returns the
        tickets (uint64) and each submission's lateness in seconds."""
        n = len(reqs)
        ta = np.ascontiguousarray(t_arrive, dtype=np.float64)
        if ta.size != n:
            raise ValueError("one arrival time per request")
        tickets = np.zeros(n, dtype=np.uint64)
        late = np.zeros(n, dtype=np.float64)
        L.check(self._lib.burgers_serve_submit_timed(
            self.h, ctypes.cast(reqs, ctypes.c_void_p), ta.ctypes.data, ctypes.c_int64(n),
            tickets.ctypes.data, late.ctypes.data), "burgers_serve_submit_timed")
        return tickets, late

    def _result(self, fn, ticket, n, *extra):
        out = np.empty(n, dtype=self.np_dtype)
        st = L.burgers_req_stats()
        rc = fn(self.h, ctypes.c_uint64(ticket), *extra, out.ctypes.data, ctypes.byref(st))
        return rc, out, st

    def poll(self, ticket: int, n: int):
        """(status, result or None, stats); status EAGAIN while running."""
        rc, out, st = self._result(self._lib.burgers_serve_poll, ticket, n)
        return rc, (out if rc == L.BURGERS_OK else None), st

    def poll_stats(self, ticket: int):
        """(status, stats) without the result (it is dropped with the ticket);
        status EAGAIN while running."""
        st = L.burgers_req_stats()
        rc = self._lib.burgers_serve_poll(self.h, ctypes.c_uint64(ticket), None, ctypes.byref(st))
        return rc, st

    def wait(self, ticket: int, n: int, timeout_s: float = 60.0):
        rc, out, st = self._result(self._lib.burgers_serve_wait, ticket, n,
                                   ctypes.c_double(timeout_s))
        return rc, (out if rc == L.BURGERS_OK else None), st

    def wait_any(self, timeout_s: float = 1.0):
        """Ticket of the next finished request, or None on timeout."""
        t = ctypes.c_uint64(0)
        rc = self._lib.burgers_serve_wait_any(self.h, float(timeout_s), ctypes.byref(t))
        return int(t.value) if rc == L.BURGERS_OK else None

    def cancel(self, ticket: int) -> int:
        return int(self._lib.burgers_serve_cancel(self.h, ctypes.c_uint64(ticket)))

    def stats(self) -> dict:
        s = L.burgers_serve_stats()
        L.check(self._lib.burgers_serve_get_stats(self.h, ctypes.byref(s)), "burgers_serve_get_stats")
        return {k: getattr(s, k) for k, _ in s._fields_}

    def close(self) -> int:
        if getattr(self, "h", None) is not None and self.h.value:
            rc = int(self._lib.burgers_serve_destroy(self.h))
            self.h = None
            return rc
        return 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
