"""Seeded synthetic Burgers workloads shared by the CUDA path and the oracle.

This module only draws inputs: grids, initial fields, viscosities, request
traces. It holds none of the solvers' arithmetic (no time step rule, no
stencil, no solve), so both sides of a parity test can take their inputs from
here without sharing any of the method.

Random draws use numpy's PCG64 seeded with ``(seed, stream)``, where the
stream is the instance index, so a subset of an ensemble reproduces exactly
the same instances as the full ensemble.

Workloads (the paper's own runs use N = 201 and a sine or step initial
condition, Sec. 2.5-2.6 and Sec. 3; the ensembles below are synthetic stand-ins
of the same family at production sizes):

* ``plain_sine``        Dirichlet on [-1, 1], u0 = -sin(pi x) (Eq. 19 with the
                        sign flipped), nu = 0.01/pi, t_final = 1/pi.
* ``fourier_ensemble``  periodic on [0, 2 pi), u0 = sum_{k=1..8} a_k sin(k x +
                        phi_k), a_k ~ Normal(0, variance 1/k), phi_k ~ U[0, 2 pi),
                        nu log-uniform in [1e-3, 1e-1].
* ``large_grid``        periodic on [0, 2 pi), u0 = sin x + 0.5 + Normal(0,
                        variance 0.01) per node, nu = 1e-3.
* ``serving_trace``     Poisson arrivals; per request N log-uniform in
                        [2^8, 2^16], scheme and BC 50/50, steps uniform in
                        [100, 5000], random-Fourier u0, nu log-uniform.
* ``step_ic``           Eq. 20: u0 = 1 for x < L/2, else 0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PERIODIC = 0
DIRICHLET = 1
EXPLICIT = 0
BTCS = 1
TWO_PI = 2.0 * math.pi
DEFAULT_SEED = 12204


def rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(seed), int(stream)]))


def grid(n: int, bc: int, x0: float, length: float):
    """Node coordinates and spacing. Periodic: n distinct nodes, dx = L/n.
    Dirichlet: n nodes including both ends, dx = L/(n-1)."""
    if bc == PERIODIC:
        dx = length / n
    else:
        dx = length / (n - 1)
    x = x0 + dx * np.arange(n, dtype=np.float64)
    return x, dx


@dataclass
class Ensemble:
    """A packed batch: row b occupies u0[offsets[b] : offsets[b] + ns[b]]."""
    u0: np.ndarray
    offsets: np.ndarray
    ns: np.ndarray
    bcs: np.ndarray
    dxs: np.ndarray
    nus: np.ndarray
    x0: np.ndarray
    length: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def count(self) -> int:
        return int(self.offsets.size)

    def row(self, b: int) -> np.ndarray:
        o = int(self.offsets[b])
        return self.u0[o:o + int(self.ns[b])]

    def subset(self, ids) -> "Ensemble":
        ids = np.asarray(ids, dtype=np.int64)
        ns = self.ns[ids]
        offs = np.zeros(ids.size, dtype=np.int64)
        offs[1:] = np.cumsum(ns[:-1])
        u0 = np.concatenate([self.row(int(b)) for b in ids]) if ids.size else np.zeros(0)
        meta = dict(self.meta)
        meta["ids"] = ids
        for k in ("a", "phi"):
            if k in meta:
                meta[k] = meta[k][ids]
        return Ensemble(u0, offs, ns.copy(), self.bcs[ids].copy(), self.dxs[ids].copy(),
                        self.nus[ids].copy(), self.x0[ids].copy(), self.length[ids].copy(), meta)


def plain_sine(n: int = 256):
    """u0 = -sin(pi x) on [-1, 1], Dirichlet u(+-1) = 0, nu = 0.01/pi, t_f = 1/pi."""
    x, dx = grid(n, DIRICHLET, -1.0, 2.0)
    u0 = -np.sin(math.pi * x)
    u0[0] = 0.0
    u0[-1] = 0.0
    return Ensemble(u0, np.zeros(1, np.int64), np.array([n], np.int32),
                    np.array([DIRICHLET], np.int32), np.array([dx]),
                    np.array([0.01 / math.pi]), np.array([-1.0]), np.array([2.0]),
                    {"t_final": 1.0 / math.pi, "x": x})


def fourier_coeffs(seed: int, stream: int, kmax: int = 8):
    g = rng(seed, stream)
    k = np.arange(1, kmax + 1, dtype=np.float64)
    a = g.normal(0.0, 1.0, kmax) / np.sqrt(k)
    phi = g.uniform(0.0, TWO_PI, kmax)
    lognu = g.uniform(math.log(1e-3), math.log(1e-1))
    return a, phi, math.exp(lognu)


def fourier_field(x: np.ndarray, a: np.ndarray, phi: np.ndarray) -> np.ndarray:
    out = np.zeros_like(x)
    for j in range(a.size):
        out += a[j] * np.sin((j + 1) * x + phi[j])
    return out


def fourier_ensemble(count: int, n: int, seed: int = DEFAULT_SEED, ids=None,
                     dtype=np.float64) -> Ensemble:
    """Periodic random-Fourier ensemble on [0, 2 pi) (row b from stream b)."""
    ids = np.arange(count, dtype=np.int64) if ids is None else np.asarray(ids, np.int64)
    m = ids.size
    x, dx = grid(n, PERIODIC, 0.0, TWO_PI)
    u0 = np.empty((m, n), dtype=np.float64)
    A = np.empty((m, 8))
    P = np.empty((m, 8))
    nus = np.empty(m)
    for j, b in enumerate(ids):
        a, phi, nu = fourier_coeffs(seed, int(b))
        A[j], P[j], nus[j] = a, phi, nu
        u0[j] = fourier_field(x, a, phi)
    return Ensemble(u0.reshape(-1).astype(dtype, copy=False), np.arange(m, dtype=np.int64) * n,
                    np.full(m, n, np.int32), np.full(m, PERIODIC, np.int32),
                    np.full(m, dx), nus, np.zeros(m), np.full(m, TWO_PI),
                    {"a": A, "phi": P, "ids": ids, "seed": seed})


def large_grid(n: int = 1 << 24, seed: int = DEFAULT_SEED) -> Ensemble:
    """u0 = sin x + 0.5 + noise (std 0.1) on a periodic [0, 2 pi) grid, nu = 1e-3."""
    x, dx = grid(n, PERIODIC, 0.0, TWO_PI)
    g = rng(seed, 1 << 40)
    u0 = np.sin(x) + 0.5 + g.normal(0.0, 0.1, n)
    return Ensemble(u0, np.zeros(1, np.int64), np.array([n], np.int32),
                    np.array([PERIODIC], np.int32), np.array([dx]), np.array([1e-3]),
                    np.zeros(1), np.array([TWO_PI]), {"seed": seed})


def step_ic(n: int, bc: int = DIRICHLET, length: float = 1.0) -> Ensemble:
    """Eq. 20: u0 = 1 for x < L/2, 0 otherwise."""
    x, dx = grid(n, bc, 0.0, length)
    u0 = np.where(x < 0.5 * length, 1.0, 0.0)
    return Ensemble(u0, np.zeros(1, np.int64), np.array([n], np.int32), np.array([bc], np.int32),
                    np.array([dx]), np.array([0.0]), np.zeros(1), np.array([length]), {"x": x})


def step_ensemble(count: int, n: int, bc: int = DIRICHLET, seed: int = DEFAULT_SEED,
                  length: float = 1.0) -> Ensemble:
    """The step-IC shock workload (Eq. 20, Sec. 3.4): every row starts from
    u0 = 1 for x < L/2, 0 otherwise, on [0, L]; nu log-uniform in [1e-5, 1e-3]
    from stream b (cell Peclet numbers u dx / nu from about 0.2 to 24 at
    n = 4096 on [0, 1], from resolved to under-resolved fronts)."""
    x, dx = grid(n, bc, 0.0, length)
    row = np.where(x < 0.5 * length, 1.0, 0.0)
    nus = np.array([math.exp(rng(seed, b).uniform(math.log(1e-5), math.log(1e-3)))
                    for b in range(count)])
    return Ensemble(np.tile(row, count), np.arange(count, dtype=np.int64) * n,
                    np.full(count, n, np.int32), np.full(count, bc, np.int32),
                    np.full(count, dx), nus, np.zeros(count), np.full(count, length), {"seed": seed})


def mixed_ensemble(count: int, nmin: int, nmax: int, seed: int = DEFAULT_SEED,
                   bc_mix: bool = True) -> Ensemble:
    """Ragged batch: n log-uniform in [nmin, nmax], periodic/Dirichlet mixed,
    random-Fourier u0 (Dirichlet rows span [0, 2 pi] so u0(0) = u0(2 pi))."""
    rows, ns, bcs, dxs, nus = [], [], [], [], []
    for b in range(count):
        g = rng(seed, (1 << 32) + b)
        n = int(round(math.exp(g.uniform(math.log(nmin), math.log(nmax)))))
        bc = int(g.integers(0, 2)) if bc_mix else PERIODIC
        a, phi, nu = fourier_coeffs(seed, (1 << 33) + b)
        x, dx = grid(n, bc, 0.0, TWO_PI)
        rows.append(fourier_field(x, a, phi))
        ns.append(n); bcs.append(bc); dxs.append(dx); nus.append(nu)
    ns = np.array(ns, np.int32)
    offs = np.zeros(count, np.int64)
    offs[1:] = np.cumsum(ns[:-1])
    return Ensemble(np.concatenate(rows), offs, ns, np.array(bcs, np.int32), np.array(dxs),
                    np.array(nus), np.zeros(count), np.full(count, TWO_PI), {"seed": seed})


@dataclass
class Request:
    rid: int
    t_arrive: float
    scheme: int
    bc: int
    n: int
    nsteps: int
    nu: float
    dx: float
    u0: np.ndarray
    a: np.ndarray = None
    phi: np.ndarray = None


def serving_trace(rate: float = 20000.0, duration: float = 10.0, seed: int = DEFAULT_SEED,
                  nmin: int = 1 << 8, nmax: int = 1 << 16, smin: int = 100, smax: int = 5000,
                  max_requests: int | None = None, with_u0: bool = True):
    """Poisson arrival trace of mixed Burgers requests."""
    g = rng(seed, 1 << 41)
    t = 0.0
    out = []
    rid = 0
    while True:
        t += g.exponential(1.0 / rate)
        if t >= duration:
            break
        if max_requests is not None and rid >= max_requests:
            break
        n = int(round(math.exp(g.uniform(math.log(nmin), math.log(nmax)))))
        scheme = int(g.integers(0, 2))
        bc = int(g.integers(0, 2))
        nsteps = int(g.integers(smin, smax + 1))
        a, phi, nu = fourier_coeffs(seed, (1 << 34) + rid)
        x, dx = grid(n, bc, 0.0, TWO_PI)
        u0 = fourier_field(x, a, phi) if with_u0 else None
        out.append(Request(rid, t, scheme, bc, n, nsteps, nu, dx, u0, a, phi))
        rid += 1
    return out


def fourier_rows_torch(reqs, device, dtype, chunk: int = 1 << 24):
    """Packs the random-Fourier initial fields of `reqs` (Requests with their
    coefficients) into one device tensor, evaluated with torch on `device`.
    Returns (tensor, offsets). Same recipe as fourier_field on each request's
    grid (periodic: dx = 2 pi/n, Dirichlet: dx = 2 pi/(n-1))."""
    import torch
    ns = np.array([q.n for q in reqs], dtype=np.int64)
    offs = np.zeros(ns.size, dtype=np.int64)
    offs[1:] = np.cumsum(ns[:-1])
    total = int(ns.sum())
    out = torch.empty(total, dtype=dtype, device=device)
    A = torch.tensor(np.stack([q.a for q in reqs]), dtype=torch.float64, device=device)
    P = torch.tensor(np.stack([q.phi for q in reqs]), dtype=torch.float64, device=device)
    dxs = torch.tensor([q.dx for q in reqs], dtype=torch.float64, device=device)
    row_of = torch.repeat_interleave(torch.arange(ns.size, device=device),
                                     torch.tensor(ns, device=device))
    start = torch.tensor(offs, device=device)
    k = torch.arange(1, A.shape[1] + 1, dtype=torch.float64, device=device)
    for lo in range(0, total, chunk):
        hi = min(total, lo + chunk)
        r = row_of[lo:hi]
        i = torch.arange(lo, hi, device=device) - start[r]
        x = i.to(torch.float64) * dxs[r]
        u = torch.sum(A[r] * torch.sin(k[None, :] * x[:, None] + P[r]), dim=1)
        out[lo:hi] = u.to(dtype)
    return out, offs
