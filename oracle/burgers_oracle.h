/*
 * burgers_oracle.h -- prototypes of the plain FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this code. The product path (the
 * CUDA library) shares no code, header, table or helper with it.
 *
 * Conventions (all arrays are double, row-major, one instance per call unless
 * the name ends in _batch):
 *   bc = 0  periodic   (Eq. 18): n distinct nodes, node n wraps to node 0.
 *   bc = 1  Dirichlet  (Eq. 16-17): n nodes including both ends; u[0] = a and
 *                       u[n-1] = b are held at their initial values.
 *   r = dt/dx, s = nu*dt/dx^2 (the two CFL numbers of Eq. 7-8).
 * Return codes: 0 ok, -1 invalid argument, -2 allocation failure.
 */
#ifndef BURGERS_ORACLE_H
#define BURGERS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

double or_cfl_dt(const double* u, int64_t n, double dx, double nu, double cfl);

int or_explicit(double* u, int64_t n, int bc, double dx, double nu, double dt, int64_t nsteps);
int or_btcs(double* u, int64_t n, int bc, double dx, double nu, double dt, int64_t nsteps);
int or_rk4(double* u, int64_t n, int bc, double dx, double nu, double dt, int64_t nsteps);
int or_cn(double* u, int64_t n, int bc, double dx, double nu, double dt, int64_t nsteps);
int or_picard(double* u, int64_t n, int bc, double dx, double nu, double dt, int64_t nsteps,
              int iters);
int or_newton(double* u, int64_t n, int bc, double dx, double nu, double dt, int64_t nsteps,
              int iters);
int or_newton_residual(const double* w, const double* un, int64_t n, int bc, double dx,
                       double nu, double dt, double* f);

int or_btcs_system(const double* un, int64_t n, int bc, double r, double s,
                   double* l, double* d, double* c, double* rhs);
int or_thomas(int64_t m, const double* l, const double* d, const double* c,
              const double* rhs, double* x);
int or_cyclic(int64_t n, const double* l, const double* d, const double* c,
              const double* rhs, double* x);

int or_explicit_batch(double* u, int64_t count, const int64_t* offset, const int32_t* n,
                      const int32_t* bc, const double* dx, const double* nu, const double* dt,
                      const int64_t* nsteps, int nthreads);
int or_rk4_batch(double* u, int64_t count, const int64_t* offset, const int32_t* n,
                 const int32_t* bc, const double* dx, const double* nu, const double* dt,
                 const int64_t* nsteps, int nthreads);
int or_cn_batch(double* u, int64_t count, const int64_t* offset, const int32_t* n,
                const int32_t* bc, const double* dx, const double* nu, const double* dt,
                const int64_t* nsteps, int nthreads);
int or_picard_batch(double* u, int64_t count, const int64_t* offset, const int32_t* n,
                    const int32_t* bc, const double* dx, const double* nu, const double* dt,
                    const int64_t* nsteps, int iters, int nthreads);
int or_newton_batch(double* u, int64_t count, const int64_t* offset, const int32_t* n,
                    const int32_t* bc, const double* dx, const double* nu, const double* dt,
                    const int64_t* nsteps, int iters, int nthreads);
int or_btcs_batch(double* u, int64_t count, const int64_t* offset, const int32_t* n,
                  const int32_t* bc, const double* dx, const double* nu, const double* dt,
                  const int64_t* nsteps, int nthreads);

int or_explicit_adjoint(const double* u0, int64_t n, int bc, double dx, double nu, double dt,
                        int64_t nsteps, const double* gT, double* gu0, double* gnu);
int or_btcs_adjoint(const double* u0, int64_t n, int bc, double dx, double nu, double dt,
                    int64_t nsteps, const double* gT, double* gu0, double* gnu);

double or_rel_l2(const double* u, const double* ref, int64_t n);
double or_rms(const double* u, const double* ref, int64_t n);

int or_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
