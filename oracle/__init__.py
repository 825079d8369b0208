"""Plain FP64 CPU oracle for the 1D viscous Burgers solvers (arXiv 2601.12204).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The CUDA product path neither imports it nor shares any code with it;
the two meet only in the seeded input generators, which hold none of the
method's arithmetic.

The numerics live in ``burgers_oracle.c`` (explicit step Eq. 21 with the
upwind side chosen per Sec. 2.2; lagged-coefficient BTCS of Sec. 2.4 / Eq. 23
solved by Thomas, or by Sherman-Morrison around Thomas for the periodic
system of Eq. 18; CFL time step Eq. 7-8; discrete adjoints; Kahan norms).
``cole_hopf.py`` holds the analytic references (Sec. 2.6) and the inviscid
characteristics solution.

Parity status: every function is pinned by the CPU tests (dense LU, linear
limits, Cole-Hopf convergence, invariants, finite differences); none is
"parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "burgers_oracle.c")
_HDR = os.path.join(_HERE, "burgers_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

PERIODIC = 0
DIRICHLET = 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math) if it is stale."""
    stale = force or not os.path.exists(_LIB)
    if not stale:
        t = os.path.getmtime(_LIB)
        stale = t < os.path.getmtime(_SRC) or t < os.path.getmtime(_HDR)
    if stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        d, i64, i32, c = ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.c_int
        P = ctypes.c_void_p
        lib.or_cfl_dt.restype = d
        lib.or_cfl_dt.argtypes = [P, i64, d, d, d]
        for name in ("or_explicit", "or_btcs", "or_rk4", "or_cn"):
            f = getattr(lib, name)
            f.restype = c
            f.argtypes = [P, i64, i32, d, d, d, i64]
        lib.or_btcs_system.restype = c
        lib.or_btcs_system.argtypes = [P, i64, i32, d, d, P, P, P, P]
        lib.or_thomas.restype = c
        lib.or_thomas.argtypes = [i64, P, P, P, P, P]
        lib.or_cyclic.restype = c
        lib.or_cyclic.argtypes = [i64, P, P, P, P, P]
        for name in ("or_picard", "or_newton"):
            f = getattr(lib, name)
            f.restype = c
            f.argtypes = [P, i64, i32, d, d, d, i64, c]
        lib.or_newton_residual.restype = c
        lib.or_newton_residual.argtypes = [P, P, i64, i32, d, d, d, P]
        for name in ("or_picard_batch", "or_newton_batch"):
            f = getattr(lib, name)
            f.restype = c
            f.argtypes = [P, i64, P, P, P, P, P, P, P, c, c]
        for name in ("or_explicit_batch", "or_btcs_batch", "or_rk4_batch", "or_cn_batch"):
            f = getattr(lib, name)
            f.restype = c
            f.argtypes = [P, i64, P, P, P, P, P, P, P, c]
        for name in ("or_explicit_adjoint", "or_btcs_adjoint"):
            f = getattr(lib, name)
            f.restype = c
            f.argtypes = [P, i64, i32, d, d, d, i64, P, P, P]
        lib.or_rel_l2.restype = d
        lib.or_rel_l2.argtypes = [P, P, i64]
        lib.or_rms.restype = d
        lib.or_rms.argtypes = [P, P, i64]
        lib.or_max_threads.restype = c
        lib.or_max_threads.argtypes = []
        _lib = lib
        return lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def max_threads() -> int:
    return int(_load().or_max_threads())


def cfl_dt(u0, dx: float, nu: float, cfl: float = 0.4) -> float:
    """Eq. 7-8: dt = cfl * min(dx / max|u0|, dx^2 / (2 nu))."""
    u = _f64(u0)
    dt = _load().or_cfl_dt(_p(u), u.size, float(dx), float(nu), float(cfl))
    if dt <= 0:
        raise ValueError("no finite CFL limit (u0 == 0 and nu == 0)")
    return float(dt)


def explicit(u0, bc: int, dx: float, nu: float, dt: float, nsteps: int) -> np.ndarray:
    """Forward-Euler upwind/central solve (Eq. 21), returns u(nsteps*dt)."""
    u = _f64(u0).copy()
    _check(_load().or_explicit(_p(u), u.size, int(bc), dx, nu, dt, int(nsteps)), "explicit")
    return u


def rk4(u0, bc: int, dx: float, nu: float, dt: float, nsteps: int) -> np.ndarray:
    """Classical fourth-order Runge-Kutta (Eq. 22) on the operator of Eq. 21."""
    u = _f64(u0).copy()
    _check(_load().or_rk4(_p(u), u.size, int(bc), dx, nu, dt, int(nsteps)), "rk4")
    return u


def cn(u0, bc: int, dx: float, nu: float, dt: float, nsteps: int) -> np.ndarray:
    """Crank-Nicolson with the convecting velocity lagged at u^n (upwind side by sign)."""
    u = _f64(u0).copy()
    _check(_load().or_cn(_p(u), u.size, int(bc), dx, nu, dt, int(nsteps)), "cn")
    return u


def picard(u0, bc: int, dx: float, nu: float, dt: float, nsteps: int, iters: int) -> np.ndarray:
    """`iters` Picard iterations A(w) w' = u^n per step (iters = 1: lagged BTCS)."""
    u = _f64(u0).copy()
    _check(_load().or_picard(_p(u), u.size, int(bc), dx, nu, dt, int(nsteps), int(iters)), "picard")
    return u


def newton(u0, bc: int, dx: float, nu: float, dt: float, nsteps: int, iters: int) -> np.ndarray:
    """`iters` Newton-Raphson iterations per step on the residual of Eq. 11."""
    u = _f64(u0).copy()
    _check(_load().or_newton(_p(u), u.size, int(bc), dx, nu, dt, int(nsteps), int(iters)), "newton")
    return u


def newton_residual(w, un, bc: int, dx: float, nu: float, dt: float) -> np.ndarray:
    """F(w) of Eq. 11 for the step from un (zero at Dirichlet ends)."""
    w, un = _f64(w), _f64(un)
    f = np.empty_like(w)
    _check(_load().or_newton_residual(_p(w), _p(un), w.size, int(bc), dx, nu, dt, _p(f)),
           "newton_residual")
    return f


def btcs(u0, bc: int, dx: float, nu: float, dt: float, nsteps: int) -> np.ndarray:
    """Lagged-coefficient upwind BTCS solve (Sec. 2.4, Eq. 23)."""
    u = _f64(u0).copy()
    _check(_load().or_btcs(_p(u), u.size, int(bc), dx, nu, dt, int(nsteps)), "btcs")
    return u


def btcs_system(un, bc: int, r: float, s: float):
    """(l, d, c, rhs) of the system one BTCS step solves; see burgers_oracle.c."""
    u = _f64(un)
    n = u.size
    m = n if bc == PERIODIC else n - 2
    l, d, c, rhs = (np.zeros(m) for _ in range(4))
    _check(_load().or_btcs_system(_p(u), n, int(bc), r, s, _p(l), _p(d), _p(c), _p(rhs)),
           "btcs_system")
    return l, d, c, rhs


def thomas(l, d, c, rhs) -> np.ndarray:
    l, d, c, rhs = map(_f64, (l, d, c, rhs))
    x = np.zeros_like(rhs)
    _check(_load().or_thomas(rhs.size, _p(l), _p(d), _p(c), _p(rhs), _p(x)), "thomas")
    return x


def cyclic(l, d, c, rhs) -> np.ndarray:
    l, d, c, rhs = map(_f64, (l, d, c, rhs))
    x = np.zeros_like(rhs)
    _check(_load().or_cyclic(rhs.size, _p(l), _p(d), _p(c), _p(rhs), _p(x)), "cyclic")
    return x


def _batch_arrays(offsets, ns, bcs, dxs, nus, dts, nsteps):
    return (np.ascontiguousarray(offsets, dtype=np.int64),
            np.ascontiguousarray(ns, dtype=np.int32),
            np.ascontiguousarray(bcs, dtype=np.int32),
            _f64(dxs), _f64(nus), _f64(dts),
            np.ascontiguousarray(nsteps, dtype=np.int64))


def _run_batch(fn, name, u, offsets, ns, bcs, dxs, nus, dts, nsteps, threads):
    u = _f64(u).copy()
    arrs = _batch_arrays(offsets, ns, bcs, dxs, nus, dts, nsteps)
    count = arrs[0].size
    for a in arrs:
        if a.size != count:
            raise ValueError("batch arrays differ in length")
    _check(fn(_p(u), count, *[_p(a) for a in arrs], int(threads)), name)
    return u


def explicit_batch(u, offsets, ns, bcs, dxs, nus, dts, nsteps, threads: int = 0) -> np.ndarray:
    """Independent explicit solves of a packed batch (one thread per instance)."""
    return _run_batch(_load().or_explicit_batch, "explicit_batch", u, offsets, ns, bcs,
                      dxs, nus, dts, nsteps, threads)


def rk4_batch(u, offsets, ns, bcs, dxs, nus, dts, nsteps, threads: int = 0) -> np.ndarray:
    """Independent RK4 solves of a packed batch (one thread per instance)."""
    return _run_batch(_load().or_rk4_batch, "rk4_batch", u, offsets, ns, bcs,
                      dxs, nus, dts, nsteps, threads)


def cn_batch(u, offsets, ns, bcs, dxs, nus, dts, nsteps, threads: int = 0) -> np.ndarray:
    """Independent Crank-Nicolson solves of a packed batch."""
    return _run_batch(_load().or_cn_batch, "cn_batch", u, offsets, ns, bcs,
                      dxs, nus, dts, nsteps, threads)


def _run_batch_iter(fn, name, u, offsets, ns, bcs, dxs, nus, dts, nsteps, iters, threads):
    u = _f64(u).copy()
    arrs = _batch_arrays(offsets, ns, bcs, dxs, nus, dts, nsteps)
    count = arrs[0].size
    for a in arrs:
        if a.size != count:
            raise ValueError("batch arrays differ in length")
    _check(fn(_p(u), count, *[_p(a) for a in arrs], int(iters), int(threads)), name)
    return u


def picard_batch(u, offsets, ns, bcs, dxs, nus, dts, nsteps, iters, threads: int = 0):
    """Independent Picard-iterated implicit solves of a packed batch."""
    return _run_batch_iter(_load().or_picard_batch, "picard_batch", u, offsets, ns, bcs, dxs,
                           nus, dts, nsteps, iters, threads)


def newton_batch(u, offsets, ns, bcs, dxs, nus, dts, nsteps, iters, threads: int = 0):
    """Independent Newton (Eq. 10-15) solves of a packed batch."""
    return _run_batch_iter(_load().or_newton_batch, "newton_batch", u, offsets, ns, bcs, dxs,
                           nus, dts, nsteps, iters, threads)


def btcs_batch(u, offsets, ns, bcs, dxs, nus, dts, nsteps, threads: int = 0) -> np.ndarray:
    """Independent BTCS solves of a packed batch (one thread per instance)."""
    return _run_batch(_load().or_btcs_batch, "btcs_batch", u, offsets, ns, bcs,
                      dxs, nus, dts, nsteps, threads)


def explicit_adjoint(u0, bc, dx, nu, dt, nsteps, gT):
    """(dJ/du0, dJ/dnu) of the explicit solve given gT = dJ/du(T)."""
    u = _f64(u0)
    g = _f64(gT)
    gu0 = np.zeros_like(u)
    gnu = ctypes.c_double(0.0)
    _check(_load().or_explicit_adjoint(_p(u), u.size, int(bc), dx, nu, dt, int(nsteps),
                                       _p(g), _p(gu0), ctypes.byref(gnu)), "explicit_adjoint")
    return gu0, float(gnu.value)


def btcs_adjoint(u0, bc, dx, nu, dt, nsteps, gT):
    """(dJ/du0, dJ/dnu) of the BTCS solve given gT = dJ/du(T)."""
    u = _f64(u0)
    g = _f64(gT)
    gu0 = np.zeros_like(u)
    gnu = ctypes.c_double(0.0)
    _check(_load().or_btcs_adjoint(_p(u), u.size, int(bc), dx, nu, dt, int(nsteps),
                                   _p(g), _p(gu0), ctypes.byref(gnu)), "btcs_adjoint")
    return gu0, float(gnu.value)


def rel_l2(u, ref) -> float:
    """||u - ref||_2 / ||ref||_2 with compensated sums."""
    a, b = _f64(u), _f64(ref)
    if a.size != b.size:
        raise ValueError("size mismatch")
    return float(_load().or_rel_l2(_p(a), _p(b), a.size))


def rms(u, ref) -> float:
    """sqrt(mean((u - ref)^2)): the 'L2' of the paper's nomenclature."""
    a, b = _f64(u), _f64(ref)
    if a.size != b.size:
        raise ValueError("size mismatch")
    return float(_load().or_rms(_p(a), _p(b), a.size))
