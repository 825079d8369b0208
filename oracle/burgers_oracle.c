/*
 * burgers_oracle.c -- plain, slow, FP64 CPU oracle of the 1D viscous Burgers
 * solvers of "Explicit and Implicit Finite Difference Solvers Implemented in
 * JAX for Shock Wave Physics" (arXiv 2601.12204).
 *
 * TEST INFRASTRUCTURE. It exists so that the CUDA path can be checked against
 * something written independently from the paper. Only tests, the smoke check
 * and the benchmark's CPU-baseline leg may load it; the CUDA library never
 * calls, links or includes it, and nothing here was derived from that library.
 *
 * Everything is double precision, straight loops in the order the method
 * states them, no blocking and no reordering:
 *
 *   explicit step   Eq. 21 (the signs of Eq. 21; Eq. 5/6/9 carry a sign typo in
 *                   the Laplacian), with the upwind side chosen by the sign of
 *                   u_i as Sec. 2.2 describes: backward difference for u_i > 0,
 *                   forward difference for u_i < 0.
 *   CN step         Crank-Nicolson (named in Sec. 2.2) with the convecting
 *                   velocity lagged at u^n, upwind side by its sign.
 *   Picard / Newton the implicit upwind equation iterated to convergence by
 *                   Picard; Newton-Raphson on the residual of Eq. 11 (central
 *                   convection), Eq. 10-15.
 *   RK4 step        Eq. 22: classical fourth-order Runge-Kutta on the spatial
 *                   operator of Eq. 21, stage by stage.
 *   BTCS step       Sec. 2.4 / Eq. 23: all spatial terms at t^{n+1}; the
 *                   convecting velocity is lagged (one Picard linearisation per
 *                   step, coefficients from u^n) and the upwind side is chosen
 *                   by the sign of u^n_i. Dirichlet: tridiagonal system on the
 *                   n-2 interior unknowns (Thomas). Periodic: cyclic system,
 *                   Sherman-Morrison around two Thomas solves.
 *   CFL time step   Eq. 7-8 with safety factor cfl: dt = cfl * min(dx/max|u|,
 *                   dx^2/(2 nu)).
 *   adjoints        transpose of the Jacobian of each step, applied in reverse
 *                   over a stored trajectory (reverse-mode differentiation,
 *                   Sec. 2.7.1 / 2.7.3).
 *   norms           relative L2 and RMS (Nomenclature "L2", Sec. 2.7.4) with
 *                   Kahan-compensated sums.
 *
 * Parity of every function here is pinned by the CPU tests against dense LU,
 * closed-form linear limits, Cole-Hopf, invariants and finite differences.
 */
#include "burgers_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_PERIODIC = 0, OR_DIRICHLET = 1 };

static double pos_part(double a) { return a > 0.0 ? a : 0.0; } /* a+ */
static double neg_part(double a) { return a < 0.0 ? a : 0.0; } /* a- */
static double heaviside(double a) { return a > 0.0 ? 1.0 : 0.0; } /* H(0) = 0 */

static int bad_common(int64_t n, int bc, double dx, double nu, double dt, int64_t nsteps) {
  if (n < 3) return 1;
  if (bc != OR_PERIODIC && bc != OR_DIRICHLET) return 1;
  if (!(dx > 0.0) || !(nu >= 0.0) || !(dt > 0.0) || nsteps < 0) return 1;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Eq. 7-8: combined convective and diffusive CFL limit.                     */
/* ------------------------------------------------------------------------ */
double or_cfl_dt(const double* u, int64_t n, double dx, double nu, double cfl) {
  double umax = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double a = fabs(u[i]);
    if (a > umax) umax = a;
  }
  double dt_conv = (umax > 0.0) ? dx / umax : INFINITY;
  double dt_diff = (nu > 0.0) ? dx * dx / (2.0 * nu) : INFINITY;
  double dt = dt_conv < dt_diff ? dt_conv : dt_diff;
  if (isinf(dt)) return -1.0;
  return cfl * dt;
}

/* ------------------------------------------------------------------------ */
/* Explicit forward-Euler upwind/central step, Eq. 21 + Sec. 2.2.            */
/* ------------------------------------------------------------------------ */
static void explicit_step(const double* u, double* v, int64_t n, int bc, double r, double s) {
  for (int64_t i = 0; i < n; ++i) {
    if (bc == OR_DIRICHLET && (i == 0 || i == n - 1)) {
      v[i] = u[i]; /* Eq. 16-17: boundary values held */
      continue;
    }
    int64_t im = (i == 0) ? n - 1 : i - 1; /* Eq. 18: periodic wrap */
    int64_t ip = (i == n - 1) ? 0 : i + 1;
    double a = u[i]; /* convecting velocity u_i^n */
    double convection = pos_part(a) * (u[i] - u[im]) + neg_part(a) * (u[ip] - u[i]);
    double diffusion = u[ip] - 2.0 * u[i] + u[im];
    v[i] = u[i] - r * convection + s * diffusion;
  }
}

int or_explicit(double* u, int64_t n, int bc, double dx, double nu, double dt, int64_t nsteps) {
  if (!u || bad_common(n, bc, dx, nu, dt, nsteps)) return -1;
  double r = dt / dx, s = nu * dt / (dx * dx);
  double* v = (double*)malloc(sizeof(double) * (size_t)n);
  if (!v) return -2;
  for (int64_t k = 0; k < nsteps; ++k) {
    explicit_step(u, v, n, bc, r, s);
    memcpy(u, v, sizeof(double) * (size_t)n);
  }
  free(v);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Tridiagonal solvers.                                                      */
/* Row i:  l[i] x[i-1] + d[i] x[i] + c[i] x[i+1] = rhs[i].                    */
/* ------------------------------------------------------------------------ */

/* Textbook Thomas algorithm (no pivoting); l[0] and c[m-1] are ignored. */
int or_thomas(int64_t m, const double* l, const double* d, const double* c,
              const double* rhs, double* x) {
  if (m < 1) return -1;
  double* cp = (double*)malloc(sizeof(double) * (size_t)m);
  double* rp = (double*)malloc(sizeof(double) * (size_t)m);
  if (!cp || !rp) { free(cp); free(rp); return -2; }
  cp[0] = (m > 1 ? c[0] : 0.0) / d[0];
  rp[0] = rhs[0] / d[0];
  for (int64_t i = 1; i < m; ++i) {
    double piv = d[i] - l[i] * cp[i - 1];
    cp[i] = (i < m - 1 ? c[i] : 0.0) / piv;
    rp[i] = (rhs[i] - l[i] * rp[i - 1]) / piv;
  }
  x[m - 1] = rp[m - 1];
  for (int64_t i = m - 2; i >= 0; --i) x[i] = rp[i] - cp[i] * x[i + 1];
  free(cp);
  free(rp);
  return 0;
}

/*
 * Cyclic tridiagonal system: l[0] is the corner A[0][n-1], c[n-1] the corner
 * A[n-1][0]. Sherman-Morrison: A = T + u v^T with gamma = -d[0],
 *   u = (gamma, 0, ..., 0, c[n-1]),  v = (1, 0, ..., 0, l[0]/gamma),
 *   T = A without corners, T[0][0] = d[0] - gamma,
 *   T[n-1][n-1] = d[n-1] - c[n-1] l[0] / gamma,
 * then x = y - (v.y)/(1 + v.z) z with T y = rhs and T z = u.
 */
int or_cyclic(int64_t n, const double* l, const double* d, const double* c,
              const double* rhs, double* x) {
  if (n < 3) return -1;
  double gamma = -d[0];
  double* dt = (double*)malloc(sizeof(double) * (size_t)n);
  double* uu = (double*)malloc(sizeof(double) * (size_t)n);
  double* y = (double*)malloc(sizeof(double) * (size_t)n);
  double* z = (double*)malloc(sizeof(double) * (size_t)n);
  if (!dt || !uu || !y || !z) { free(dt); free(uu); free(y); free(z); return -2; }
  for (int64_t i = 0; i < n; ++i) { dt[i] = d[i]; uu[i] = 0.0; }
  dt[0] = d[0] - gamma;
  dt[n - 1] = d[n - 1] - c[n - 1] * l[0] / gamma;
  uu[0] = gamma;
  uu[n - 1] = c[n - 1];
  int rc = or_thomas(n, l, dt, c, rhs, y);
  if (rc == 0) rc = or_thomas(n, l, dt, c, uu, z);
  if (rc == 0) {
    double vy = y[0] + (l[0] / gamma) * y[n - 1];
    double vz = z[0] + (l[0] / gamma) * z[n - 1];
    double fac = vy / (1.0 + vz);
    for (int64_t i = 0; i < n; ++i) x[i] = y[i] - fac * z[i];
  }
  free(dt); free(uu); free(y); free(z);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* BTCS with lagged (Picard) upwind coefficients, Sec. 2.4 and Eq. 23.       */
/* Implicit equation for node i, convecting velocity a = u_i^n:              */
/*   x_i + r[a+ (x_i - x_{i-1}) + a- (x_{i+1} - x_i)]                         */
/*       - s (x_{i+1} - 2 x_i + x_{i-1}) = u_i^n                              */
/* ------------------------------------------------------------------------ */
static void btcs_row(double a, double r, double s, double* l, double* d, double* c) {
  *l = -r * pos_part(a) - s;
  *d = 1.0 + r * pos_part(a) - r * neg_part(a) + 2.0 * s;
  *c = r * neg_part(a) - s;
}

/*
 * Writes the linear system that one BTCS step solves.
 * Periodic: n rows, l[0] / c[n-1] are the corners.
 * Dirichlet: n-2 rows for the interior nodes 1..n-2; the known boundary
 * values are moved to the right-hand side; l[0] and c[n-3] are set to 0.
 */
int or_btcs_system(const double* un, int64_t n, int bc, double r, double s,
                   double* l, double* d, double* c, double* rhs) {
  if (n < 3) return -1;
  if (bc == OR_PERIODIC) {
    for (int64_t i = 0; i < n; ++i) {
      btcs_row(un[i], r, s, &l[i], &d[i], &c[i]);
      rhs[i] = un[i];
    }
    return 0;
  }
  if (bc != OR_DIRICHLET) return -1;
  int64_t m = n - 2;
  for (int64_t j = 0; j < m; ++j) {
    int64_t i = j + 1;
    btcs_row(un[i], r, s, &l[j], &d[j], &c[j]);
    rhs[j] = un[i];
  }
  rhs[0] -= l[0] * un[0];
  rhs[m - 1] -= c[m - 1] * un[n - 1];
  l[0] = 0.0;
  c[m - 1] = 0.0;
  return 0;
}

typedef struct {
  double *l, *d, *c, *rhs, *x;
} work5;

static int work_alloc(work5* w, int64_t n) {
  size_t b = sizeof(double) * (size_t)n;
  w->l = (double*)malloc(b); w->d = (double*)malloc(b); w->c = (double*)malloc(b);
  w->rhs = (double*)malloc(b); w->x = (double*)malloc(b);
  if (!w->l || !w->d || !w->c || !w->rhs || !w->x) return -2;
  return 0;
}
static void work_free(work5* w) {
  free(w->l); free(w->d); free(w->c); free(w->rhs); free(w->x);
}

static int btcs_step(double* u, int64_t n, int bc, double r, double s, work5* w) {
  int rc = or_btcs_system(u, n, bc, r, s, w->l, w->d, w->c, w->rhs);
  if (rc) return rc;
  if (bc == OR_PERIODIC) {
    rc = or_cyclic(n, w->l, w->d, w->c, w->rhs, w->x);
    if (rc) return rc;
    memcpy(u, w->x, sizeof(double) * (size_t)n);
  } else {
    rc = or_thomas(n - 2, w->l, w->d, w->c, w->rhs, w->x);
    if (rc) return rc;
    memcpy(u + 1, w->x, sizeof(double) * (size_t)(n - 2));
  }
  return 0;
}

int or_btcs(double* u, int64_t n, int bc, double dx, double nu, double dt, int64_t nsteps) {
  if (!u || bad_common(n, bc, dx, nu, dt, nsteps)) return -1;
  double r = dt / dx, s = nu * dt / (dx * dx);
  work5 w;
  int rc = work_alloc(&w, n);
  for (int64_t k = 0; rc == 0 && k < nsteps; ++k) rc = btcs_step(u, n, bc, r, s, &w);
  work_free(&w);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Further implicit variants (the paper names Crank-Nicolson, Sec. 2.2, and   */
/* Newton-Raphson on the residual of Eq. 11, Eq. 10-15).                      */
/* Each step solves tridiagonal systems (cyclic when periodic) with the        */
/* solvers above; Dirichlet end values are held and moved to the right-hand  */
/* side of the interior system.                                               */
/* ------------------------------------------------------------------------ */

/* Solves the n-row system (l, d, c, rhs) for the new state x: periodic rows  */
/* as a cyclic system; Dirichlet rows 1..n-2 with x[0], x[n-1] known (their   */
/* couplings moved to the right-hand side). l, d, c, rhs are clobbered.       */
static int solve_rows(int64_t n, int bc, double* l, double* d, double* c, double* rhs,
                      double* x, double* tmp) {
  if (bc == OR_PERIODIC) {
    int rc = or_cyclic(n, l, d, c, rhs, tmp);
    if (rc == 0) memcpy(x, tmp, sizeof(double) * (size_t)n);
    return rc;
  }
  int64_t m = n - 2;
  rhs[1] -= l[1] * x[0];
  rhs[n - 2] -= c[n - 2] * x[n - 1];
  l[1] = 0.0;
  c[n - 2] = 0.0;
  int rc = or_thomas(m, l + 1, d + 1, c + 1, rhs + 1, tmp);
  if (rc == 0) memcpy(x + 1, tmp, sizeof(double) * (size_t)m);
  return rc;
}

/* Crank-Nicolson with the convecting velocity lagged at u^n (upwind side by  */
/* its sign, as for BTCS): with L(a) the upwind/central operator of Eq. 21,   */
/*   (I - dt/2 L(u^n)) u^{n+1} = (I + dt/2 L(u^n)) u^n,                        */
/* i.e. BTCS rows with r/2, s/2 and the right-hand side u^n plus half the     */
/* forward-Euler increment of u^n.                                            */
int or_cn(double* u, int64_t n, int bc, double dx, double nu, double dt, int64_t nsteps) {
  if (!u || bad_common(n, bc, dx, nu, dt, nsteps)) return -1;
  double r = dt / dx, s = nu * dt / (dx * dx);
  double* buf = (double*)malloc(sizeof(double) * (size_t)n * 6);
  if (!buf) return -2;
  double *l = buf, *d = buf + n, *c = buf + 2 * n, *rhs = buf + 3 * n, *half = buf + 4 * n,
         *tmp = buf + 5 * n;
  int rc = 0;
  for (int64_t k = 0; rc == 0 && k < nsteps; ++k) {
    explicit_step(u, half, n, bc, 0.5 * r, 0.5 * s); /* u^n + dt/2 L(u^n) u^n */
    for (int64_t i = 0; i < n; ++i) {
      btcs_row(u[i], 0.5 * r, 0.5 * s, &l[i], &d[i], &c[i]);
      rhs[i] = half[i];
    }
    rc = solve_rows(n, bc, l, d, c, rhs, u, tmp);
  }
  free(buf);
  return rc;
}

/* Picard iteration on the implicit upwind equation: iterate                  */
/*   A(w) w' = u^n,  w^0 = u^n,                                                */
/* `iters` times per step (A as in BTCS, coefficients from the latest iterate); */
/* iters = 1 is the lagged BTCS step.                                          */
int or_picard(double* u, int64_t n, int bc, double dx, double nu, double dt, int64_t nsteps,
              int iters) {
  if (!u || bad_common(n, bc, dx, nu, dt, nsteps) || iters < 1) return -1;
  double r = dt / dx, s = nu * dt / (dx * dx);
  double* buf = (double*)malloc(sizeof(double) * (size_t)n * 6);
  if (!buf) return -2;
  double *l = buf, *d = buf + n, *c = buf + 2 * n, *rhs = buf + 3 * n, *w = buf + 4 * n,
         *tmp = buf + 5 * n;
  int rc = 0;
  for (int64_t k = 0; rc == 0 && k < nsteps; ++k) {
    memcpy(w, u, sizeof(double) * (size_t)n);
    for (int it = 0; rc == 0 && it < iters; ++it) {
      for (int64_t i = 0; i < n; ++i) {
        btcs_row(w[i], r, s, &l[i], &d[i], &c[i]);
        rhs[i] = u[i];
      }
      rc = solve_rows(n, bc, l, d, c, rhs, w, tmp);
    }
    memcpy(u, w, sizeof(double) * (size_t)n);
  }
  free(buf);
  return rc;
}

/* Residual of Eq. 11 (central convection, all terms at the new level) at    */
/* node i, for a periodic row or an interior Dirichlet node.                   */
static double newton_residual(const double* w, const double* un, int64_t n, int64_t i, double r,
                              double s) {
  int64_t im = (i == 0) ? n - 1 : i - 1;
  int64_t ip = (i == n - 1) ? 0 : i + 1;
  return w[i] - un[i] + 0.5 * r * w[i] * (w[ip] - w[im]) - s * (w[ip] - 2.0 * w[i] + w[im]);
}

/* Newton-Raphson on F(w) = 0, F of Eq. 11 (Eq. 10-14), `iters` iterations per */
/* step from w^0 = u^n. The Jacobian follows from Eq. 11 (Eq. 15 prints only   */
/* a sub-diagonal entry, with a garbled sign on its diffusive part):           */
/*   dF_i/dw_{i-1} = -r/2 w_i - s,  dF_i/dw_i = 1 + r/2 (w_{i+1} - w_{i-1}) + 2s, */
/*   dF_i/dw_{i+1} = r/2 w_i - s.                                              */
/* Dirichlet end values are held (zero Newton update there).                   */
int or_newton(double* u, int64_t n, int bc, double dx, double nu, double dt, int64_t nsteps,
              int iters) {
  if (!u || bad_common(n, bc, dx, nu, dt, nsteps) || iters < 1) return -1;
  double r = dt / dx, s = nu * dt / (dx * dx);
  double* buf = (double*)malloc(sizeof(double) * (size_t)n * 7);
  if (!buf) return -2;
  double *l = buf, *d = buf + n, *c = buf + 2 * n, *rhs = buf + 3 * n, *w = buf + 4 * n,
         *du = buf + 5 * n, *tmp = buf + 6 * n;
  int rc = 0;
  for (int64_t k = 0; rc == 0 && k < nsteps; ++k) {
    memcpy(w, u, sizeof(double) * (size_t)n);
    for (int it = 0; rc == 0 && it < iters; ++it) {
      for (int64_t i = 0; i < n; ++i) {
        int64_t im = (i == 0) ? n - 1 : i - 1;
        int64_t ip = (i == n - 1) ? 0 : i + 1;
        l[i] = -0.5 * r * w[i] - s;
        d[i] = 1.0 + 0.5 * r * (w[ip] - w[im]) + 2.0 * s;
        c[i] = 0.5 * r * w[i] - s;
        rhs[i] = -newton_residual(w, u, n, i, r, s);
      }
      du[0] = 0.0;
      du[n - 1] = 0.0;
      rc = solve_rows(n, bc, l, d, c, rhs, du, tmp);
      for (int64_t i = 0; i < n; ++i) w[i] += du[i];
    }
    memcpy(u, w, sizeof(double) * (size_t)n);
  }
  free(buf);
  return rc;
}

/* Residual of Eq. 11 for the whole row (Dirichlet ends report 0).            */
int or_newton_residual(const double* w, const double* un, int64_t n, int bc, double dx,
                       double nu, double dt, double* f) {
  if (!w || !un || !f || bad_common(n, bc, dx, nu, dt, 0)) return -1;
  double r = dt / dx, s = nu * dt / (dx * dx);
  for (int64_t i = 0; i < n; ++i)
    f[i] = (bc == OR_DIRICHLET && (i == 0 || i == n - 1)) ? 0.0
                                                          : newton_residual(w, un, n, i, r, s);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Batched drivers: independent instances, one OpenMP thread per instance.   */
/* ------------------------------------------------------------------------ */
int or_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Classical fourth-order Runge-Kutta in time, Eq. 22, on the semi-discrete  */
/* operator of Eq. 21 (upwind side by the sign of u_i, Sec. 2.2):            */
/*   F(u)_i = -(a+ (u_i - u_{i-1}) + a- (u_{i+1} - u_i))/dx                   */
/*            + nu (u_{i+1} - 2 u_i + u_{i-1})/dx^2,     a = u_i,             */
/* F = 0 at held Dirichlet ends.                                             */
/*   k1 = F(u^n), k2 = F(u^n + dt/2 k1), k3 = F(u^n + dt/2 k2),              */
/*   k4 = F(u^n + dt k3),  u^{n+1} = u^n + dt/6 (k1 + 2 k2 + 2 k3 + k4).      */
/* ------------------------------------------------------------------------ */
static void burgers_rhs(const double* u, double* f, int64_t n, int bc, double dx, double nu) {
  for (int64_t i = 0; i < n; ++i) {
    if (bc == OR_DIRICHLET && (i == 0 || i == n - 1)) {
      f[i] = 0.0;
      continue;
    }
    int64_t im = (i == 0) ? n - 1 : i - 1;
    int64_t ip = (i == n - 1) ? 0 : i + 1;
    double a = u[i];
    double convection = (pos_part(a) * (u[i] - u[im]) + neg_part(a) * (u[ip] - u[i])) / dx;
    double diffusion = nu * (u[ip] - 2.0 * u[i] + u[im]) / (dx * dx);
    f[i] = -convection + diffusion;
  }
}

int or_rk4(double* u, int64_t n, int bc, double dx, double nu, double dt, int64_t nsteps) {
  if (!u || bad_common(n, bc, dx, nu, dt, nsteps)) return -1;
  double* k1 = (double*)malloc(sizeof(double) * (size_t)n * 5);
  if (!k1) return -2;
  double* k2 = k1 + n;
  double* k3 = k2 + n;
  double* k4 = k3 + n;
  double* w = k4 + n;
  for (int64_t k = 0; k < nsteps; ++k) {
    burgers_rhs(u, k1, n, bc, dx, nu);
    for (int64_t i = 0; i < n; ++i) w[i] = u[i] + 0.5 * dt * k1[i];
    burgers_rhs(w, k2, n, bc, dx, nu);
    for (int64_t i = 0; i < n; ++i) w[i] = u[i] + 0.5 * dt * k2[i];
    burgers_rhs(w, k3, n, bc, dx, nu);
    for (int64_t i = 0; i < n; ++i) w[i] = u[i] + dt * k3[i];
    burgers_rhs(w, k4, n, bc, dx, nu);
    for (int64_t i = 0; i < n; ++i)
      u[i] = u[i] + dt / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
  }
  free(k1);
  return 0;
}

typedef int (*stepper_fn)(double*, int64_t, int, double, double, double, int64_t);

static int run_batch(stepper_fn f, double* u, int64_t count, const int64_t* offset,
                     const int32_t* n, const int32_t* bc, const double* dx, const double* nu,
                     const double* dt, const int64_t* nsteps, int nthreads) {
  int err = 0;
#ifdef _OPENMP
  if (nthreads < 1) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) reduction(| : err)
#endif
  for (int64_t b = 0; b < count; ++b) {
    int rc = f(u + offset[b], n[b], bc[b], dx[b], nu[b], dt[b], nsteps[b]);
    if (rc) err |= 1;
  }
  (void)nthreads;
  return err ? -1 : 0;
}

int or_explicit_batch(double* u, int64_t count, const int64_t* offset, const int32_t* n,
                      const int32_t* bc, const double* dx, const double* nu, const double* dt,
                      const int64_t* nsteps, int nthreads) {
  return run_batch(or_explicit, u, count, offset, n, bc, dx, nu, dt, nsteps, nthreads);
}

int or_rk4_batch(double* u, int64_t count, const int64_t* offset, const int32_t* n,
                 const int32_t* bc, const double* dx, const double* nu, const double* dt,
                 const int64_t* nsteps, int nthreads) {
  return run_batch(or_rk4, u, count, offset, n, bc, dx, nu, dt, nsteps, nthreads);
}

int or_cn_batch(double* u, int64_t count, const int64_t* offset, const int32_t* n,
                const int32_t* bc, const double* dx, const double* nu, const double* dt,
                const int64_t* nsteps, int nthreads) {
  return run_batch(or_cn, u, count, offset, n, bc, dx, nu, dt, nsteps, nthreads);
}

typedef int (*iter_fn)(double*, int64_t, int, double, double, double, int64_t, int);

static int run_batch_iter(iter_fn f, double* u, int64_t count, const int64_t* offset,
                          const int32_t* n, const int32_t* bc, const double* dx, const double* nu,
                          const double* dt, const int64_t* nsteps, int iters, int nthreads) {
  int err = 0;
#ifdef _OPENMP
  if (nthreads < 1) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) reduction(| : err)
#endif
  for (int64_t b = 0; b < count; ++b) {
    int rc = f(u + offset[b], n[b], bc[b], dx[b], nu[b], dt[b], nsteps[b], iters);
    if (rc) err |= 1;
  }
  (void)nthreads;
  return err ? -1 : 0;
}

int or_picard_batch(double* u, int64_t count, const int64_t* offset, const int32_t* n,
                    const int32_t* bc, const double* dx, const double* nu, const double* dt,
                    const int64_t* nsteps, int iters, int nthreads) {
  return run_batch_iter(or_picard, u, count, offset, n, bc, dx, nu, dt, nsteps, iters, nthreads);
}

int or_newton_batch(double* u, int64_t count, const int64_t* offset, const int32_t* n,
                    const int32_t* bc, const double* dx, const double* nu, const double* dt,
                    const int64_t* nsteps, int iters, int nthreads) {
  return run_batch_iter(or_newton, u, count, offset, n, bc, dx, nu, dt, nsteps, iters, nthreads);
}

int or_btcs_batch(double* u, int64_t count, const int64_t* offset, const int32_t* n,
                  const int32_t* bc, const double* dx, const double* nu, const double* dt,
                  const int64_t* nsteps, int nthreads) {
  return run_batch(or_btcs, u, count, offset, n, bc, dx, nu, dt, nsteps, nthreads);
}

/* ------------------------------------------------------------------------ */
/* Adjoints (reverse mode over a stored trajectory).                          */
/* gT = dJ/du(T); outputs gu0 = dJ/du(0) and gnu = dJ/dnu, with dt, dx and    */
/* nsteps held constant. At a = 0 the derivative of a+ is taken as 0 and that */
/* of a- as 1 (H(0) = 0).                                                     */
/* ------------------------------------------------------------------------ */
int or_explicit_adjoint(const double* u0, int64_t n, int bc, double dx, double nu, double dt,
                        int64_t nsteps, const double* gT, double* gu0, double* gnu) {
  if (!u0 || !gT || !gu0 || !gnu || bad_common(n, bc, dx, nu, dt, nsteps)) return -1;
  double r = dt / dx, s = nu * dt / (dx * dx), ds_dnu = dt / (dx * dx);
  size_t nb = sizeof(double) * (size_t)n;
  double* traj = (double*)malloc(nb * (size_t)(nsteps + 1));
  double* lam = (double*)malloc(nb);
  double* nl = (double*)malloc(nb);
  if (!traj || !lam || !nl) { free(traj); free(lam); free(nl); return -2; }
  memcpy(traj, u0, nb);
  for (int64_t k = 0; k < nsteps; ++k) explicit_step(traj + k * n, traj + (k + 1) * n, n, bc, r, s);
  memcpy(lam, gT, nb);
  double g = 0.0;
  for (int64_t k = nsteps - 1; k >= 0; --k) {
    const double* u = traj + k * n;
    for (int64_t i = 0; i < n; ++i) nl[i] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      if (bc == OR_DIRICHLET && (i == 0 || i == n - 1)) {
        nl[i] += lam[i]; /* held value: identity */
        continue;
      }
      int64_t im = (i == 0) ? n - 1 : i - 1;
      int64_t ip = (i == n - 1) ? 0 : i + 1;
      double a = u[i], H = heaviside(a);
      double dl = u[i] - u[im], dr = u[ip] - u[i];
      /* partial derivatives of v_i = explicit update at node i */
      double dv_dim = r * pos_part(a) + s;
      double dv_dip = -r * neg_part(a) + s;
      double dv_dii = 1.0 - r * (H * dl + (1.0 - H) * dr + pos_part(a) - neg_part(a)) - 2.0 * s;
      nl[i] += lam[i] * dv_dii;
      nl[im] += lam[i] * dv_dim;
      nl[ip] += lam[i] * dv_dip;
      g += lam[i] * ds_dnu * (u[ip] - 2.0 * u[i] + u[im]);
    }
    memcpy(lam, nl, nb);
  }
  memcpy(gu0, lam, nb);
  *gnu = g;
  free(traj); free(lam); free(nl);
  return 0;
}

int or_btcs_adjoint(const double* u0, int64_t n, int bc, double dx, double nu, double dt,
                    int64_t nsteps, const double* gT, double* gu0, double* gnu) {
  if (!u0 || !gT || !gu0 || !gnu || bad_common(n, bc, dx, nu, dt, nsteps)) return -1;
  double r = dt / dx, s = nu * dt / (dx * dx), ds_dnu = dt / (dx * dx);
  size_t nb = sizeof(double) * (size_t)n;
  double* traj = (double*)malloc(nb * (size_t)(nsteps + 1));
  double* lam = (double*)malloc(nb);
  double* nl = (double*)malloc(nb);
  double *al = (double*)malloc(nb), *ad = (double*)malloc(nb), *ac = (double*)malloc(nb);
  double *tl = (double*)malloc(nb), *tc = (double*)malloc(nb), *mu = (double*)malloc(nb);
  work5 w;
  int rc = work_alloc(&w, n);
  if (!traj || !lam || !nl || !al || !ad || !ac || !tl || !tc || !mu) rc = -2;
  if (rc == 0) {
    memcpy(traj, u0, nb);
    for (int64_t k = 0; rc == 0 && k < nsteps; ++k) {
      memcpy(traj + (k + 1) * n, traj + k * n, nb);
      rc = btcs_step(traj + (k + 1) * n, n, bc, r, s, &w);
    }
  }
  if (rc == 0) {
    memcpy(lam, gT, nb);
    double g = 0.0;
    for (int64_t k = nsteps - 1; k >= 0 && rc == 0; --k) {
      const double* un = traj + k * n;        /* coefficients lagged from u^n */
      const double* x = traj + (k + 1) * n;   /* u^{n+1} */
      if (bc == OR_PERIODIC) {
        for (int64_t i = 0; i < n; ++i) btcs_row(un[i], r, s, &al[i], &ad[i], &ac[i]);
        /* A^T: sub-diagonal of row i is c[i-1], super-diagonal is l[i+1];
           corners: A^T[0][n-1] = c[n-1], A^T[n-1][0] = l[0]. */
        for (int64_t i = 0; i < n; ++i) {
          tl[i] = ac[(i + n - 1) % n];
          tc[i] = al[(i + 1) % n];
        }
        rc = or_cyclic(n, tl, ad, tc, lam, mu);
        if (rc) break;
        for (int64_t i = 0; i < n; ++i) {
          int64_t im = (i + n - 1) % n, ip = (i + 1) % n;
          double H = heaviside(un[i]);
          /* d(A x)_i / d a_i with x = u^{n+1} held fixed */
          double drow = r * (-H * x[im] + (2.0 * H - 1.0) * x[i] + (1.0 - H) * x[ip]);
          nl[i] = mu[i] - mu[i] * drow;
          g += mu[i] * ds_dnu * (x[ip] - 2.0 * x[i] + x[im]);
        }
      } else {
        int64_t m = n - 2;
        for (int64_t j = 0; j < m; ++j) btcs_row(un[j + 1], r, s, &al[j], &ad[j], &ac[j]);
        for (int64_t j = 0; j < m; ++j) {
          tl[j] = (j > 0) ? ac[j - 1] : 0.0;
          tc[j] = (j < m - 1) ? al[j + 1] : 0.0;
        }
        rc = or_thomas(m, tl, ad, tc, lam + 1, mu);
        if (rc) break;
        for (int64_t j = 0; j < m; ++j) {
          int64_t i = j + 1;
          double H = heaviside(un[i]);
          double drow = r * (-H * x[i - 1] + (2.0 * H - 1.0) * x[i] + (1.0 - H) * x[i + 1]);
          nl[i] = mu[j] - mu[j] * drow;
          g += mu[j] * ds_dnu * (x[i + 1] - 2.0 * x[i] + x[i - 1]);
        }
        /* boundary values: held (identity) and moved to the right-hand side
           of the first / last interior rows with coefficients -l_1, -c_{n-2} */
        nl[0] = lam[0] - al[0] * mu[0];
        nl[n - 1] = lam[n - 1] - ac[m - 1] * mu[m - 1];
      }
      memcpy(lam, nl, nb);
    }
    if (rc == 0) {
      memcpy(gu0, lam, nb);
      *gnu = g;
    }
  }
  work_free(&w);
  free(traj); free(lam); free(nl); free(al); free(ad); free(ac); free(tl); free(tc); free(mu);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Norms with Kahan-compensated sums.                                         */
/* ------------------------------------------------------------------------ */
static double kahan_sum_sq_diff(const double* a, const double* b, int64_t n) {
  double sum = 0.0, comp = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double e = b ? (a[i] - b[i]) : a[i];
    double y = e * e - comp;
    double t = sum + y;
    comp = (t - sum) - y;
    sum = t;
  }
  return sum;
}

double or_rel_l2(const double* u, const double* ref, int64_t n) {
  double num = kahan_sum_sq_diff(u, ref, n);
  double den = kahan_sum_sq_diff(ref, NULL, n);
  if (den == 0.0) return num == 0.0 ? 0.0 : INFINITY;
  return sqrt(num / den);
}

double or_rms(const double* u, const double* ref, int64_t n) {
  if (n < 1) return 0.0;
  return sqrt(kahan_sum_sq_diff(u, ref, n) / (double)n);
}
