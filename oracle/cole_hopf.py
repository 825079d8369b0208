"""Analytic references for the viscous and inviscid Burgers equation (Eq. 1).

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).

* ``hopf``: the Cole-Hopf transformation that Sec. 2.6 uses as the analytic
  reference. On the infinite line, with U0(y) = int_0^y u0,

      u(x, t) = int ((x - y)/t) exp(-G/(2 nu)) dy / int exp(-G/(2 nu)) dy,
      G(y; x, t) = (x - y)^2 / (2 t) + U0(y).

  Evaluated with a trapezoid rule on a window around the characteristic foot,
  shifted by min G (log-sum-exp) so nothing underflows, and refined by
  halving the step until two successive answers agree.
* ``characteristics``: the inviscid (nu = 0) solution u = u0(x - u t) before
  the first shock time, solved per point by safeguarded Newton iteration.

Profiles carry both u0 and its antiderivative U0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Callable

import numpy as np


@dataclass
class Profile:
    u0: Callable[[np.ndarray], np.ndarray]
    U0: Callable[[np.ndarray], np.ndarray]
    umax: float
    du0: Callable[[np.ndarray], np.ndarray] | None = None


def sine(amp: float, k: float) -> Profile:
    """u0 = amp sin(k x), U0 = amp (1 - cos k x) / k (Eq. 19 for amp=1, k=pi)."""
    return Profile(lambda x: amp * np.sin(k * x),
                   lambda x: amp * (1.0 - np.cos(k * x)) / k,
                   abs(amp),
                   lambda x: amp * k * np.cos(k * x))


def fourier(a, phi, shift: float = 0.0) -> Profile:
    """u0 = shift + sum_k a_k sin(k x + phi_k), k = 1..len(a)."""
    a = np.asarray(a, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    ks = np.arange(1, a.size + 1, dtype=np.float64)

    def u0(x):
        x = np.asarray(x, dtype=np.float64)
        return shift + np.sum(a[:, None] * np.sin(ks[:, None] * x.ravel()[None, :] + phi[:, None]),
                              axis=0).reshape(x.shape)

    def U0(x):
        x = np.asarray(x, dtype=np.float64)
        t = a[:, None] * (np.cos(phi[:, None]) - np.cos(ks[:, None] * x.ravel()[None, :] + phi[:, None]))
        return shift * x + np.sum(t / ks[:, None], axis=0).reshape(x.shape)

    def du0(x):
        x = np.asarray(x, dtype=np.float64)
        return np.sum((a * ks)[:, None] * np.cos(ks[:, None] * x.ravel()[None, :] + phi[:, None]),
                      axis=0).reshape(x.shape)

    return Profile(u0, U0, abs(shift) + float(np.sum(np.abs(a))), du0)


def _log_cosh(z):
    z = np.abs(z)
    return z + np.log1p(np.exp(-2.0 * z)) - math.log(2.0)


def tanh_shock(U: float, nu: float) -> Profile:
    """Steady viscous shock u0 = -U tanh(U x / (2 nu)), U0 = -2 nu log cosh(.)."""
    return Profile(lambda x: -U * np.tanh(U * np.asarray(x) / (2.0 * nu)),
                   lambda x: -2.0 * nu * _log_cosh(U * np.asarray(x) / (2.0 * nu)),
                   abs(U))


def hopf(profile: Profile, x, t: float, nu: float, rtol: float = 1e-12,
         max_halvings: int = 14) -> np.ndarray:
    """Cole-Hopf solution u(x, t) for nu > 0, t > 0 (see module docstring)."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    if t <= 0:
        return profile.u0(x)
    # window: beyond |x - y| = 3 t umax + delta the weight is below exp(-delta^2/(4 nu t))
    half = 3.0 * t * profile.umax + 20.0 * math.sqrt(nu * t) + 1e-12
    # first step: resolve both the heat kernel and the exp(-U0/2nu) scale
    h = min(math.sqrt(nu * t), nu / max(profile.umax, 1e-300)) / 4.0
    out = None
    for _ in range(max_halvings):
        m = int(math.ceil(2.0 * half / h))
        if m % 2:
            m += 1
        offs = np.linspace(-half, half, m + 1)
        w = np.full(m + 1, 1.0)
        w[0] = w[-1] = 0.5
        res = np.empty_like(x)
        chunk = max(1, int(4_000_000 // (m + 1)))
        for s in range(0, x.size, chunk):
            xs = x[s:s + chunk]
            y = xs[:, None] + offs[None, :]
            G = (xs[:, None] - y) ** 2 / (2.0 * t) + profile.U0(y)
            G -= G.min(axis=1, keepdims=True)
            e = np.exp(-G / (2.0 * nu)) * w[None, :]
            res[s:s + chunk] = np.sum(((xs[:, None] - y) / t) * e, axis=1) / np.sum(e, axis=1)
        if out is not None:
            scale = max(float(np.max(np.abs(res))), 1e-300)
            if float(np.max(np.abs(res - out))) <= rtol * scale:
                return res
        out = res
        h *= 0.5
    return out


def characteristics(profile: Profile, x, t: float, iters: int = 100) -> np.ndarray:
    """Inviscid solution u = u0(x - u t) for t below the first shock time."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    u = profile.u0(x)
    for _ in range(iters):
        xi = x - u * t
        f = u - profile.u0(xi)
        df = 1.0 + t * profile.du0(xi)
        step = f / df
        u = u - step
        if float(np.max(np.abs(step))) < 1e-15 * max(1.0, float(np.max(np.abs(u)))):
            break
    return u
