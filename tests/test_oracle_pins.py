"""Pins of the FP64 CPU oracle against things the paper and the mathematics fix.

None of these compares the oracle with itself: each check is a closed form, a
library routine on a special case, an invariant, an independent analytic
solution, or a finite difference.
"""
import math

import numpy as np
import pytest

from oracle import cole_hopf as CH
from paper_2601_12204_b300 import workloads as W

P, D = W.PERIODIC, W.DIRICHLET


def dense_from_tridiag(l, d, c, cyclic):
    n = d.size
    A = np.diag(d)
    for i in range(n):
        if i > 0:
            A[i, i - 1] = l[i]
        if i < n - 1:
            A[i, i + 1] = c[i]
    if cyclic:
        A[0, n - 1] = l[0]
        A[n - 1, 0] = c[n - 1]
    return A


# --------------------------------------------------------------------------
# Tridiagonal and cyclic solvers vs dense LU (numpy.linalg.solve).
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [3, 4, 5, 7, 16, 33, 64])
@pytest.mark.parametrize("cyclic", [False, True])
def test_solvers_match_dense_lu(orc, n, cyclic):
    g = np.random.default_rng(100 + n)
    for trial in range(4):
        l = -g.uniform(0, 3, n)
        c = -g.uniform(0, 3, n)
        d = 1.0 + np.abs(l) + np.abs(c) + g.uniform(0, 0.5, n)
        rhs = g.normal(size=n)
        A = dense_from_tridiag(l, d, c, cyclic)
        ref = np.linalg.solve(A, rhs)
        x = orc.cyclic(l, d, c, rhs) if cyclic else orc.thomas(l, d, c, rhs)
        assert np.max(np.abs(x - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("bc", [P, D])
@pytest.mark.parametrize("n", [3, 5, 17, 64])
def test_btcs_system_is_m_matrix_and_solves_dense(orc, bc, n):
    """Assembled BTCS rows (Eq. 23): off-diagonals <= 0, diagonal margin exactly
    1 (rows sum to one), and one step equals the dense solve of that system."""
    g = np.random.default_rng(7 * n + bc)
    u = g.normal(size=n)
    r, s = 2.3, 1.7
    l, d, c, rhs = orc.btcs_system(u, bc, r, s)
    cyc = bc == P
    A = dense_from_tridiag(l, d, c, cyc)
    offd = A - np.diag(np.diag(A))
    assert np.all(offd <= 0)
    if cyc:
        np.testing.assert_allclose(A.sum(axis=1), 1.0, rtol=0, atol=1e-14)
    x_dense = np.linalg.solve(A, rhs)
    dx = 0.1
    dt = r * dx
    nu = s * dx * dx / dt
    x = orc.btcs(u, bc, dx, nu, dt, 1)
    got = x if cyc else x[1:-1]
    assert np.max(np.abs(got - x_dense)) <= 1e-13 * max(1.0, np.max(np.abs(x_dense)))
    if not cyc:
        assert x[0] == u[0] and x[-1] == u[-1]


# --------------------------------------------------------------------------
# Closed-form linear limits (von Neumann amplification factors).
# --------------------------------------------------------------------------
def _periodic(n, L=2 * math.pi):
    return W.grid(n, P, 0.0, L)


def rk4_factor(z):
    """Amplification of classical RK4 (Eq. 22) for du/dt = (z/dt) u: the
    degree-4 Taylor polynomial of exp(z)."""
    return 1 + z + z**2 / 2 + z**3 / 6 + z**4 / 24


@pytest.mark.parametrize("scheme", ["explicit", "btcs", "rk4"])
def test_small_amplitude_is_heat_equation(orc, scheme):
    n, k, eps = 64, 3, 1e-9
    x, dx = _periodic(n)
    nu = 0.3
    dt = 0.4 * dx * dx / (2 * nu)
    if scheme == "btcs":
        dt *= 10
    s = nu * dt / dx**2
    steps = 40
    u = eps * np.sin(k * x)
    out = getattr(orc, scheme)(u, P, dx, nu, dt, steps)
    sn2 = math.sin(k * dx / 2) ** 2
    if scheme == "rk4":
        g = rk4_factor(-4 * s * sn2)
    else:
        g = 1 - 4 * s * sn2 if scheme == "explicit" else 1 / (1 + 4 * s * sn2)
    expect = eps * g**steps * np.sin(k * x)
    assert np.max(np.abs(out - expect)) <= 1e-6 * eps


@pytest.mark.parametrize("scheme", ["explicit", "btcs", "rk4"])
@pytest.mark.parametrize("c0", [0.7, -0.7])
def test_linear_advection_upwind_side(orc, scheme, c0):
    """u = c + eps w: the perturbation obeys the linear upwind scheme whose
    side is selected by sign(c) (Sec. 2.2); a wrong side or sign fails."""
    n, k, eps = 48, 2, 1e-7
    x, dx = _periodic(n)
    nu = 0.02
    dt = 0.4 * min(dx / abs(c0), dx * dx / (2 * nu))
    if scheme == "btcs":
        dt *= 4
    r, s = dt / dx, nu * dt / dx**2
    steps = 30
    u0 = c0 + eps * np.sin(k * x)
    out = getattr(orc, scheme)(u0, P, dx, nu, dt, steps)
    e = np.exp(1j * k * dx)
    if c0 > 0:
        conv = r * c0 * (1 - 1 / e)
    else:
        conv = r * c0 * (e - 1)
    diff = 4 * s * math.sin(k * dx / 2) ** 2
    if scheme == "rk4":
        g = rk4_factor(-conv - diff)
    else:
        g = 1 - conv - diff if scheme == "explicit" else 1 / (1 + conv + diff)
    expect = c0 + eps * np.imag(g**steps * np.exp(1j * k * x))
    assert np.max(np.abs(out - expect)) <= 2e-3 * eps


@pytest.mark.parametrize("scheme", ["explicit", "btcs", "rk4"])
@pytest.mark.parametrize("bc", [P, D])
def test_constant_state_is_fixed_point(orc, scheme, bc):
    n = 37
    for cval in (0.0, 1.25, -0.8):
        u = np.full(n, cval)
        out = getattr(orc, scheme)(u, bc, 0.05, 0.01, 0.01, 25)
        assert np.max(np.abs(out - cval)) <= 1e-14 * max(1, abs(cval))


# --------------------------------------------------------------------------
# Invariants.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("bc", [P, D])
def test_max_principle_explicit_under_cfl(orc, bc):
    e = W.fourier_ensemble(6, 200, seed=3)
    for b in range(e.count):
        u0 = e.row(b).copy()
        dx, nu = e.dxs[b], e.nus[b]
        dt = 0.4 * min(dx / np.max(np.abs(u0)), dx * dx / (2 * nu))
        u = u0
        lo, hi = u0.min(), u0.max()
        for _ in range(20):
            u = orc.explicit(u, bc, dx, nu, dt, 10)
            assert u.min() >= lo - 1e-13 and u.max() <= hi + 1e-13


@pytest.mark.parametrize("bc", [P, D])
def test_btcs_bounded_for_large_steps(orc, bc):
    """Sec. 3.4: the implicit solver stays stable at dt = 5 dx / u_max on a step IC
    (M-matrix: the solution stays within the range of the data)."""
    e = W.step_ic(128, bc)
    dx = e.dxs[0]
    for nu, factor in ((1e-3, 5.0), (1e-2, 5.0), (0.0, 25.0)):
        dt = factor * dx / 1.0
        u = orc.btcs(e.u0, bc, dx, nu, dt, 60)
        assert u.min() >= -1e-13 and u.max() <= 1 + 1e-13


def test_explicit_beyond_cfl_oscillates(orc):
    """Sec. 3.1: beyond the diffusive limit (s = 0.6 > 1/2) the explicit scheme
    amplifies the grid-scale mode; BTCS at the same step does not."""
    n = 64
    x, dx = _periodic(n)
    nu = 0.1
    dt = 1.2 * dx * dx / (2 * nu)
    g = np.random.default_rng(1)
    u0 = 0.01 * np.sin(x) + 1e-6 * g.normal(size=n)
    ue = orc.explicit(u0, P, dx, nu, dt, 60)
    ub = orc.btcs(u0, P, dx, nu, dt, 300)
    # the grid-scale mode grows by |1 - 4 s| = 1.4 per step
    assert not np.all(np.isfinite(ue)) or np.max(np.abs(ue)) > 100 * np.max(np.abs(u0))
    assert np.max(np.abs(ub)) <= np.max(np.abs(u0))


@pytest.mark.parametrize("scheme", ["explicit", "btcs", "rk4"])
def test_mirror_symmetry(orc, scheme):
    """u0(x) -> -u0(-x) maps solutions to mirrored solutions; the odd IC of
    the plain sine case (u0 = -sin(pi x), Dirichlet) stays odd: u_i = -u_{N-1-i}."""
    e = W.plain_sine(101)
    dx, nu = e.dxs[0], e.nus[0]
    dt = 0.004
    out = getattr(orc, scheme)(e.u0, D, dx, nu, dt, 60)
    assert np.max(np.abs(out + out[::-1])) <= 1e-14


@pytest.mark.parametrize("scheme", ["explicit", "btcs", "rk4"])
def test_shift_equivariance_periodic(orc, scheme):
    e = W.fourier_ensemble(1, 96, seed=11)
    u0, dx, nu = e.u0, e.dxs[0], e.nus[0]
    dt = 0.4 * min(dx / np.max(np.abs(u0)), dx * dx / (2 * nu))
    base = getattr(orc, scheme)(u0, P, dx, nu, dt, 50)
    for sh in (1, 17, 95):
        got = getattr(orc, scheme)(np.roll(u0, sh), P, dx, nu, dt, 50)
        assert np.max(np.abs(got - np.roll(base, sh))) <= 1e-13


@pytest.mark.parametrize("scheme", ["explicit", "btcs", "rk4"])
def test_batch_matches_single(orc, scheme):
    e = W.mixed_ensemble(9, 5, 80, seed=5)
    dts = np.array([0.4 * min(e.dxs[b] / np.max(np.abs(e.row(b))), e.dxs[b] ** 2 / (2 * e.nus[b]))
                    for b in range(e.count)])
    steps = np.arange(e.count) * 3 + 1
    fb = getattr(orc, scheme + "_batch")
    out = fb(e.u0, e.offsets, e.ns, e.bcs, e.dxs, e.nus, dts, steps, threads=3)
    for b in range(e.count):
        one = getattr(orc, scheme)(e.row(b), e.bcs[b], e.dxs[b], e.nus[b], dts[b], steps[b])
        o = e.offsets[b]
        assert np.array_equal(out[o:o + e.ns[b]], one)


# --------------------------------------------------------------------------
# CFL time step (Eq. 7-8) and norms.
# --------------------------------------------------------------------------
def test_cfl_dt_closed_form(orc):
    u = np.array([0.5, -2.0, 1.0])
    assert orc.cfl_dt(u, 0.1, 0.0, 0.4) == pytest.approx(0.4 * 0.1 / 2.0, rel=1e-15)
    assert orc.cfl_dt(u, 0.1, 1.0, 0.4) == pytest.approx(0.4 * 0.01 / 2.0, rel=1e-15)
    assert orc.cfl_dt(np.zeros(4), 0.2, 0.5, 1.0) == pytest.approx(0.04, rel=1e-15)
    with pytest.raises(ValueError):
        orc.cfl_dt(np.zeros(4), 0.1, 0.0, 0.4)


def test_norms_against_exact_sums(orc):
    g = np.random.default_rng(2)
    ref = g.normal(size=10001)
    u = ref + 1e-3 * g.normal(size=ref.size)
    num = math.fsum((u - ref) ** 2)
    den = math.fsum(ref**2)
    assert orc.rel_l2(u, ref) == pytest.approx(math.sqrt(num / den), rel=1e-14)
    assert orc.rel_l2(ref * (1 + 2.0**-20), ref) == pytest.approx(2.0**-20, rel=1e-12)
    assert orc.rms(ref + 0.25, ref) == pytest.approx(0.25, rel=1e-13)
    assert orc.rel_l2(ref, ref) == 0.0


# --------------------------------------------------------------------------
# Analytic references: Cole-Hopf (Sec. 2.6) and the inviscid limit.
# --------------------------------------------------------------------------
def test_hopf_reproduces_stationary_shock():
    U, nu = 1.0, 0.05
    prof = CH.tanh_shock(U, nu)
    x = np.linspace(-0.7, 0.7, 29)
    got = CH.hopf(prof, x, 0.4, nu)
    assert np.max(np.abs(got - prof.u0(x))) <= 1e-10


def test_hopf_small_amplitude_is_heat_kernel():
    eps, k, nu, t = 1e-7, 2.0, 0.1, 0.7
    x = np.linspace(0, 2 * math.pi, 23)
    got = CH.hopf(CH.sine(eps, k), x, t, nu)
    expect = eps * math.exp(-nu * k * k * t) * np.sin(k * x)
    assert np.max(np.abs(got - expect)) <= 1e-6 * eps


def test_hopf_matches_mpmath_quadrature():
    """Independent arbitrary-precision evaluation of the Hopf integrals for the
    configuration-1 data u0 = -sin(pi x), nu = 0.01/pi, t = 1/pi."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    nu, t = 0.01 / math.pi, 1.0 / math.pi
    prof = CH.sine(-1.0, math.pi)
    xs = [-0.5, -0.05, 0.02, 0.3]
    got = CH.hopf(prof, np.array(xs), t, nu)
    for xv, gv in zip(xs, got):
        X = mp.mpf(xv)

        def G(y):
            return (X - y) ** 2 / (2 * t) + (mp.cos(mp.pi * y) - 1) / mp.pi

        y0 = X - 3
        y1 = X + 3
        pts = [y0] + [X + mp.mpf(j) / 40 for j in range(-80, 81)] + [y1]
        gmin = min(G(p) for p in pts)
        num = mp.quad(lambda y: (X - y) / t * mp.exp(-(G(y) - gmin) / (2 * nu)), pts)
        den = mp.quad(lambda y: mp.exp(-(G(y) - gmin) / (2 * nu)), pts)
        assert abs(float(num / den) - gv) <= 1e-9


def _order(errs, ns):
    return [math.log(errs[i] / errs[i + 1]) / math.log(ns[i + 1] / ns[i]) for i in range(len(ns) - 1)]


@pytest.mark.parametrize("scheme", ["explicit", "btcs", "rk4"])
def test_first_order_convergence_to_cole_hopf(orc, scheme):
    """Smooth regime (t < shock time 1): error vs Cole-Hopf falls at order ~1
    (upwind convection + forward/backward Euler with dt ~ dx), not the O(dx^2)
    the paper claims."""
    nu, t = 0.05, 0.5
    prof = CH.sine(1.0, 1.0)
    ns = [64, 128, 256, 512]
    errs = []
    for n in ns:
        x, dx = _periodic(n)
        dt0 = 0.4 * min(dx / 1.0, dx * dx / (2 * nu))
        if scheme == "btcs":
            dt0 *= 2
        steps = math.ceil(t / dt0)
        dt = t / steps
        u = getattr(orc, scheme)(prof.u0(x), P, dx, nu, dt, steps)
        errs.append(orc.rms(u, CH.hopf(prof, x, t, nu)))
    orders = _order(errs, ns)
    assert all(0.8 <= o <= 1.25 for o in orders), (errs, orders)


def test_rk4_is_fourth_order_in_time(orc):
    """Eq. 22 on a fixed grid: halving dt cuts the error against a much finer
    time step by ~2^4 (a wrong stage weight or stage offset drops the order),
    while forward Euler on the same problem gains only ~2^1. u > 0 everywhere,
    so the upwind side never switches and the semi-discrete operator is smooth."""
    n, nu, t = 64, 0.05, 0.2
    x, dx = _periodic(n)
    u0 = 1.0 + 0.3 * np.sin(x) + 0.1 * np.cos(3 * x)
    ref = orc.rk4(u0, P, dx, nu, t / 4096, 4096)
    for scheme, lo, hi in (("rk4", 13.0, 19.0), ("explicit", 1.7, 2.3)):
        errs = []
        for steps in (64, 128, 256):
            out = getattr(orc, scheme)(u0, P, dx, nu, t / steps, steps)
            errs.append(np.max(np.abs(out - ref)))
        ratios = [errs[i] / errs[i + 1] for i in range(2)]
        assert all(lo <= q <= hi for q in ratios), (scheme, errs, ratios)


def test_rk4_dirichlet_ends_held(orc):
    e = W.plain_sine(64)
    u0 = e.u0.copy()
    u0[0], u0[-1] = 0.3, -0.2
    out = orc.rk4(u0, D, e.dxs[0], e.nus[0], 0.004, 40)
    assert out[0] == 0.3 and out[-1] == -0.2


def test_inviscid_limit_converges_to_characteristics(orc):
    prof = CH.fourier([0.2], [0.0], shift=0.5)
    t = 2.0  # shock time 1/0.2 = 5
    ns = [64, 128, 256, 512]
    errs = []
    for n in ns:
        x, dx = _periodic(n)
        dt0 = 0.4 * dx / 0.7
        steps = math.ceil(t / dt0)
        u = orc.explicit(prof.u0(x), P, dx, 0.0, t / steps, steps)
        errs.append(orc.rms(u, CH.characteristics(prof, x, t)))
    orders = _order(errs, ns)
    assert all(0.8 <= o <= 1.25 for o in orders), (errs, orders)


def test_dirichlet_steady_shock_converges(orc):
    U, nu, t = 1.0, 0.05, 0.5
    prof = CH.tanh_shock(U, nu)
    ns = [65, 129, 257]
    errs = []
    for n in ns:
        x, dx = W.grid(n, D, -1.0, 2.0)
        dt0 = 0.4 * min(dx / U, dx * dx / (2 * nu))
        steps = math.ceil(t / dt0)
        u = orc.explicit(prof.u0(x), D, dx, nu, t / steps, steps)
        errs.append(orc.rms(u, prof.u0(x)))
    orders = _order(errs, [n - 1 for n in ns])
    assert all(0.7 <= o <= 1.3 for o in orders), (errs, orders)


# --------------------------------------------------------------------------
# Adjoints vs central finite differences of the forward oracle.
# --------------------------------------------------------------------------
def _loss_and_fd(orc, scheme, u0, bc, dx, nu, dt, steps, target, v, h):
    fwd = getattr(orc, scheme)

    def J(u, nu_):
        return 0.5 * math.fsum(((fwd(u, bc, dx, nu_, dt, steps) - target) ** 2).tolist())

    d_u = (J(u0 + h * v, nu) - J(u0 - h * v, nu)) / (2 * h)
    hn = 1e-6 * nu
    d_nu = (J(u0, nu + hn) - J(u0, nu - hn)) / (2 * hn)
    return d_u, d_nu


@pytest.mark.parametrize("scheme", ["explicit", "btcs"])
@pytest.mark.parametrize("bc", [P, D])
@pytest.mark.parametrize("shift", [0.6, -0.6, 0.0])
def test_adjoint_matches_central_differences(orc, scheme, bc, shift):
    n = 40
    x, dx = W.grid(n, bc, 0.0, 2 * math.pi)
    nu = 0.05
    u0 = shift + 0.3 * np.sin(x) + 0.05 * np.cos(3 * x)
    dt = 0.4 * min(dx / np.max(np.abs(u0)), dx * dx / (2 * nu))
    if scheme == "btcs":
        dt *= 5
    steps = 25
    fwd = getattr(orc, scheme)
    target = fwd(u0 + 0.1 * np.cos(2 * x), bc, dx, nu, dt, steps)
    uT = fwd(u0, bc, dx, nu, dt, steps)
    gu0, gnu = getattr(orc, scheme + "_adjoint")(u0, bc, dx, nu, dt, steps, uT - target)
    g = np.random.default_rng(9)
    for _ in range(3):
        v = g.normal(size=n)
        d_u, d_nu = _loss_and_fd(orc, scheme, u0, bc, dx, nu, dt, steps, target, v, 1e-6)
        assert float(gu0 @ v) == pytest.approx(d_u, rel=2e-6, abs=1e-10)
    assert gnu == pytest.approx(d_nu, rel=2e-6, abs=1e-10)


# --------------------------------------------------------------------------
# Further implicit variants: Crank-Nicolson (lagged upwind), Picard-iterated
# implicit upwind, Newton-Raphson on the residual of Eq. 11.
# --------------------------------------------------------------------------
def test_cn_heat_and_advection_limits(orc):
    """Small perturbations obey the linear CN scheme: amplification
    (1 - z/2)/(1 + z/2) with z the upwind/central eigenvalue (both signs of
    the convecting velocity)."""
    n, k, eps = 48, 2, 1e-7
    x, dx = _periodic(n)
    nu = 0.02
    for c0 in (0.0, 0.7, -0.7):
        amp = eps if c0 == 0.0 else eps
        dt = 0.4 * (dx * dx / (2 * nu) if c0 == 0.0 else min(dx / abs(c0), dx * dx / (2 * nu))) * 5
        r, s = dt / dx, nu * dt / dx**2
        steps = 30
        out = orc.cn(c0 + amp * np.sin(k * x), P, dx, nu, dt, steps)
        e = np.exp(1j * k * dx)
        conv = 0.0 if c0 == 0.0 else (r * c0 * (1 - 1 / e) if c0 > 0 else r * c0 * (e - 1))
        z = conv + 4 * s * math.sin(k * dx / 2) ** 2
        g = (1 - z / 2) / (1 + z / 2)
        expect = c0 + amp * np.imag(g**steps * np.exp(1j * k * x))
        assert np.max(np.abs(out - expect)) <= 2e-3 * amp, c0


def test_cn_second_order_in_time_for_heat(orc):
    """In the heat limit CN converges at second order in dt to the
    semi-discrete solution exp(-4 nu sin^2(k dx/2)/dx^2 t); BTCS at first."""
    n, k, eps, nu, t = 32, 3, 1e-9, 0.2, 0.5
    x, dx = _periodic(n)
    lam = 4 * nu * math.sin(k * dx / 2) ** 2 / dx**2
    exact = eps * math.exp(-lam * t) * np.sin(k * x)
    for scheme, lo, hi in (("cn", 3.6, 4.4), ("btcs", 1.7, 2.3)):
        errs = []
        for steps in (40, 80, 160):
            out = getattr(orc, scheme)(eps * np.sin(k * x), P, dx, nu, t / steps, steps)
            errs.append(np.max(np.abs(out - exact)))
        ratios = [errs[i] / errs[i + 1] for i in range(2)]
        assert all(lo <= q <= hi for q in ratios), (scheme, errs, ratios)


@pytest.mark.parametrize("scheme", ["cn"])
@pytest.mark.parametrize("bc", [P, D])
def test_cn_invariants(orc, scheme, bc):
    for cval in (0.0, 1.25, -0.8):
        out = orc.cn(np.full(37, cval), bc, 0.05, 0.01, 0.01, 25)
        assert np.max(np.abs(out - cval)) <= 1e-14 * max(1, abs(cval))
    e = W.plain_sine(101)
    out = orc.cn(e.u0, D, e.dxs[0], e.nus[0], 0.004, 60)
    assert np.max(np.abs(out + out[::-1])) <= 1e-14 and out[0] == 0.0 and out[-1] == 0.0


@pytest.mark.parametrize("bc", [P, D])
def test_picard_one_iteration_is_btcs(orc, bc):
    e = W.mixed_ensemble(4, 20, 200, seed=3)
    for b in range(e.count):
        u0, dx, nu = e.row(b), e.dxs[b], e.nus[b]
        dt = 5 * orc.cfl_dt(u0, dx, nu)
        assert np.array_equal(orc.picard(u0, bc, dx, nu, dt, 7, 1), orc.btcs(u0, bc, dx, nu, dt, 7))


def _upwind_implicit_residual(w, un, dx, nu, dt, bc):
    """w_i + r (w_i+ (w_i - w_{i-1}) + w_i- (w_{i+1} - w_i)) - s (w_{i+1} - 2 w_i + w_{i-1}) - un_i."""
    r, s = dt / dx, nu * dt / dx**2
    wm, wp = np.roll(w, 1), np.roll(w, -1)
    res = w + r * (np.maximum(w, 0) * (w - wm) + np.minimum(w, 0) * (wp - w)) \
        - s * (wp - 2 * w + wm) - un
    if bc == D:
        res[0] = res[-1] = 0.0
    return res


@pytest.mark.parametrize("bc", [P, D])
def test_picard_converges_to_the_implicit_upwind_equation(orc, bc):
    """Iterating the lagged solve reaches the fixed point of the fully implicit
    upwind equation; the iterates contract geometrically."""
    x, dx = _periodic(64)
    u0 = 0.2 + 0.8 * np.sin(x)
    nu = 0.02
    dt = 3 * orc.cfl_dt(u0, dx, nu)
    prev, diffs = None, []
    for it in range(1, 9):
        w = orc.picard(u0, bc, dx, nu, dt, 1, it)
        if prev is not None:
            diffs.append(np.max(np.abs(w - prev)))
        prev = w
    assert all(diffs[i + 1] < 0.7 * diffs[i] for i in range(len(diffs) - 1) if diffs[i] > 1e-14)
    w = orc.picard(u0, bc, dx, nu, dt, 1, 60)
    assert np.max(np.abs(_upwind_implicit_residual(w, u0, dx, nu, dt, bc))) <= 1e-13


def test_newton_linear_limits_are_central_implicit(orc):
    """Small perturbations of a constant state obey the implicit scheme with
    CENTRAL convection of Eq. 11: amplification 1/(1 + i r c sin(k dx) +
    4 s sin^2(k dx/2)) (an upwind or sign-flipped convection fails)."""
    n, k, eps = 48, 2, 1e-8
    x, dx = _periodic(n)
    nu = 0.02
    for c0 in (0.0, 0.6, -0.6):
        dt = 0.01
        r, s = dt / dx, nu * dt / dx**2
        steps = 25
        out = orc.newton(c0 + eps * np.sin(k * x), P, dx, nu, dt, steps, 3)
        g = 1 / (1 + 1j * r * c0 * math.sin(k * dx) + 4 * s * math.sin(k * dx / 2) ** 2)
        expect = c0 + eps * np.imag(g**steps * np.exp(1j * k * x))
        assert np.max(np.abs(out - expect)) <= 1e-4 * eps, c0


@pytest.mark.parametrize("bc", [P, D])
def test_newton_converges_quadratically(orc, bc):
    """||F(w_{k+1})|| <= C ||F(w_k)||^2 for the residual of Eq. 11: the
    Jacobian matches F (a wrong entry, e.g. the sign Eq. 15 prints for the
    diffusive part, gives linear convergence)."""
    x, dx = _periodic(96)
    u0 = 0.3 + 0.9 * np.sin(x) + 0.2 * np.cos(2 * x)
    nu, dt = 0.03, 0.02
    norms = []
    for it in range(1, 6):
        w = orc.newton(u0, bc, dx, nu, dt, 1, it)
        norms.append(np.max(np.abs(orc.newton_residual(w, u0, bc, dx, nu, dt))))
    f0 = np.max(np.abs(orc.newton_residual(u0, u0, bc, dx, nu, dt)))
    seq = [f0] + norms
    assert seq[-1] <= 1e-13
    for a, b in zip(seq, seq[1:]):
        if b > 1e-12:
            assert b <= 10.0 * a * a, seq


@pytest.mark.parametrize("scheme", ["cn", "picard", "newton"])
def test_implicit_variants_batch_matches_single(orc, scheme):
    e = W.mixed_ensemble(7, 5, 80, seed=6)
    dts = np.array([2 * orc.cfl_dt(e.row(b), e.dxs[b], e.nus[b]) for b in range(e.count)])
    steps = np.arange(e.count) + 2
    if scheme == "cn":
        out = orc.cn_batch(e.u0, e.offsets, e.ns, e.bcs, e.dxs, e.nus, dts, steps, threads=3)
        one = lambda b: orc.cn(e.row(b), e.bcs[b], e.dxs[b], e.nus[b], dts[b], steps[b])  # noqa: E731
    else:
        fb = getattr(orc, scheme + "_batch")
        out = fb(e.u0, e.offsets, e.ns, e.bcs, e.dxs, e.nus, dts, steps, 3, threads=3)
        f1 = getattr(orc, scheme)
        one = lambda b: f1(e.row(b), e.bcs[b], e.dxs[b], e.nus[b], dts[b], steps[b], 3)  # noqa: E731
    for b in range(e.count):
        o = e.offsets[b]
        assert np.array_equal(out[o:o + e.ns[b]], one(b))
