// adjoint.cu -- hand-written discrete adjoints of the explicit and BTCS solves
// (reverse-mode differentiation of the solution with respect to the initial
// state and the viscosity, Sec. 2.7.1 / 2.7.3).
//
// Given gT = dJ/du(T) the kernels return dJ/du(0) and dJ/dnu, holding dt, dx
// and the step count fixed. One CTA owns one row (the resident register
// layout of the forward kernels: thread t holds C consecutive nodes).
//
// Checkpointing: the forward pass stores u every k steps (k = ceil(sqrt(nsteps))
// by default); the reverse pass walks the segments backwards, recomputes the
// k+1 states of a segment into a per-row buffer and applies the transposed
// step Jacobians to lambda, held in registers, from the last state to the first.
// Memory per row: (ceil(nsteps/k) + k + 1) * n values.
//
// Explicit step (Eq. 21, upwind side by sign, H(0) = 0):
//   lambda_i <- (1 - 2s - r (H_i dl_i + (1-H_i) dr_i + |u_i|)) lambda_i
//             + (s + r u_{i+1}^+) lambda_{i+1} + (s - r u_{i-1}^-) lambda_{i-1}
//   dJ/dnu  += (dt/dx^2) sum_i lambda_i (u_{i+1} - 2u_i + u_{i-1})
// BTCS step A(u^n) u^{n+1} = u^n:
//   mu = A^{-T} lambda   (transposed rows: sub c_{i-1}, diag d_i, super l_{i+1},
//                         corners c_{n-1}, l_0; the same partitioned cyclic solver)
//   lambda_i <- mu_i - mu_i r (-H_i x_{i-1} + (2H_i - 1) x_i + (1 - H_i) x_{i+1}),
//   dJ/dnu  += (dt/dx^2) sum_i mu_i (x_{i+1} - 2x_i + x_{i-1}),   x = u^{n+1}.
// Dirichlet end nodes are identity rows: they pass lambda through (plus what
// their neighbours' updates send them) and add nothing to dJ/dnu.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "adjoint.h"
#include "btcs_common.cuh"
#include "common.cuh"
#include "kernels.h"
#include "api_internal.h"

namespace burgers {

template <typename T, int NT>
struct Xch {
  T first[2][NT], last[2][NT], wl[2], wr[2];
};

// dJ/dnu partial sums of the FP32 kernels between folds into the FP64 total:
// Kahan summation over at most SPLIT_FOLD reverse steps, then s - c added in
// FP64 (the fold schedule is the global reverse-step count, so the sum does
// not depend on the checkpoint stride). One FP64 conversion and add per step
// and thread would keep B300's FP64 pipe, which runs at a small fraction of
// the FP32 rate, busy through the whole reverse sweep.
struct NuSum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ void fold(double& acc) {
    acc += double(s) - double(c);
    s = 0.f;
    c = 0.f;
  }
};

// The same on packed pairs (two partial sums per thread).
struct NuSum2 {
  float2 s = make_float2(0.f, 0.f), c = make_float2(0.f, 0.f);
  __device__ __forceinline__ void add(float2 x) {
    const float2 y = sub2(x, c);
    const float2 t = add2(s, y);
    c = sub2(sub2(t, s), y);
    s = t;
  }
  __device__ __forceinline__ void fold(double& acc) {
    acc += (double(s.x) - double(c.x)) + (double(s.y) - double(c.y));
    s = make_float2(0.f, 0.f);
    c = make_float2(0.f, 0.f);
  }
};

// Publishes this thread's end nodes of v; after the barrier, returns the
// value left of node `base` (wrap: node n-1 for thread 0), right of node
// base+C-1 and the periodic right neighbour of node n-1 (node 0).
template <typename T, int NT, int C>
__device__ __forceinline__ void xch_publish(const T (&v)[C], int jstar, Xch<T, NT>& x, int p) {
  const int tid = threadIdx.x;
  x.first[p][tid] = v[0];
  x.last[p][tid] = v[C - 1];
  if (jstar >= 0 && jstar < C) {
    T sel = v[0];
#pragma unroll
    for (int j = 1; j < C; ++j)
      if (j == jstar) sel = v[j];
    x.wl[p] = sel;
  }
  if (tid == 0) x.wr[p] = v[0];
}
template <typename T, int NT>
__device__ __forceinline__ void xch_read(const Xch<T, NT>& x, int p, T& left, T& right, T& wrapR) {
  const int tid = threadIdx.x;
  left = tid > 0 ? x.last[p][tid - 1] : x.wl[p];
  right = tid + 1 < NT ? x.first[p][tid + 1] : x.wr[p];
  wrapR = x.wr[p];
}

// neighbours of node j of this thread: ul, ur (periodic wrap at node n-1)
template <typename T, int C>
__device__ __forceinline__ void nbrs(const T (&v)[C], int j, int jstar, T left, T right, T wrapR,
                                     T& ul, T& ur) {
  ul = j > 0 ? v[j - 1] : left;
  ur = j + 1 < C ? v[j + 1] : right;
  if (j == jstar) ur = wrapR;
}

// one explicit forward step of the resident layout (generic, padding aware)
template <typename T, int NT, int C>
__device__ __forceinline__ void fwd_explicit_step(T (&v)[C], T (&lo)[C], int n, int base, bool per,
                                                  T r, T h, T s, Xch<T, NT>& xs, int& p) {
  const int jstar = n - 1 - base;
  xch_publish<T, NT, C>(v, jstar, xs, p);
  __syncthreads();
  T left, right, wr;
  xch_read<T, NT>(xs, p, left, right, wr);
  p ^= 1;
  T prev = left;
#pragma unroll
  for (int j = 0; j < C; ++j) {
    const int gi = base + j;
    T ul = prev, ur = j + 1 < C ? v[j + 1] : right;
    if (j == jstar) ur = wr;
    const T cur = v[j];
    const T lo0 = lo[j];
    T nv = explicit_update(cur, ul, ur, r, h, s, lo[j]);
    const bool keep = gi >= n || (!per && (gi == 0 || gi == n - 1));
    if (keep) { nv = cur; lo[j] = lo0; }
    prev = cur;
    v[j] = nv;
  }
}

// BTCS rows (lagged coefficients of node values a) and their transpose.
template <typename T>
__device__ __forceinline__ void btcs_coef(T a, T r, T s, T& l, T& d, T& c) {
  const T ra = r * a;
  l = -s - tmax(ra, T(0));
  c = tmin(ra, T(0)) - s;
  d = T(1) + T(2) * s + tabs(ra);
}

// generic resident cyclic / plain tridiagonal solve of this CTA's row: rows
// from rowfn(j, l, d, c, rhs); solution into x. Uses sm (three barriers).
template <typename T, int NT, int C, typename RowFn>
__device__ __forceinline__ void resident_solve(T (&x)[C], T (&ah)[C], T (&ch)[C], RowFn&& rowfn,
                                               int n, bool cyc, BtcsShared<T, NT>& sm) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int base = tid * C;
  const int tl = (n - 1) / C;
  const int je = base < n ? (n - 1 - base < C - 1 ? n - 1 - base : C - 1) : -1;
  T e_ch, e_ah, e_dh;
  chunk_forward<T, C>(x, ah, ch, je, rowfn, e_ch, e_ah, e_dh);
  chunk_backward<T, C>(x, ah, ch, je);
  sm.rd[sk(tid)] = x[0];
  sm.ra[sk(tid)] = ah[0];
  sm.rg[sk(tid)] = ch[0];
  __syncthreads();
  T A = T(0), B = T(1), Cc = T(0), D = T(0);
  if (tid <= tl) {
    const int nx = (tid == tl) ? 0 : tid + 1;
    A = e_ah;
    B = T(1) - e_ch * sm.ra[sk(nx)];
    Cc = -e_ch * sm.rg[sk(nx)];
    D = tfma(-e_ch, sm.rd[sk(nx)], e_dh);
  }
  const int si = sk(tid);
  sm.A[si] = A; sm.B[si] = B; sm.Cc[si] = Cc; sm.D[si] = D; sm.U[si] = T(0);
  __syncthreads();
  if (warp == NT / 32 - 1) {  // the last warp (warp 0 also carries the row's first node)
    if (cyc) reduced_solve<T, NT, true>(sm, tl, lane);
    else reduced_solve<T, NT, false>(sm, tl, lane);
  }
  __syncthreads();
  if (tid <= tl) {
    T L = T(0);
    if (tid > 0) L = sm.X[sk(tid - 1)];
    else if (cyc) L = sm.X[sk(tl)];
    const T Xt = sm.X[sk(tid)];
#pragma unroll
    for (int j = 0; j < C; ++j) x[j] = tfma(-ch[j], Xt, tfma(-ah[j], L, x[j]));
  }
}

// one BTCS forward step of the resident layout (generic), in the increment
// form of the forward kernel: A(u^n) delta = Delta(u^n), u += delta.
template <typename T, int NT, int C>
__device__ __forceinline__ void fwd_btcs_step(T (&v)[C], T (&lo)[C], int n, int base, bool per,
                                              T r, T s, BtcsShared<T, NT>& sm,
                                              Xch<T, NT>& xs, int& p) {
  const int jstar = n - 1 - base;
  xch_publish<T, NT, C>(v, jstar, xs, p);
  __syncthreads();
  T left, right, wr;
  xch_read<T, NT>(xs, p, left, right, wr);
  p ^= 1;
  T ah[C], ch[C], x[C];
  auto rows = [&](int j, T& l, T& d, T& c, T& rhs) {
    const int gi = base + j;
    T ul, ur;
    nbrs<T, C>(v, j, jstar, left, right, wr, ul, ur);
    btcs_coef(v[j], r, s, l, d, c);
    rhs = tfma(l, v[j] - ul, -c * (ur - v[j]));  // explicit increment from the same coefficients
    if (!per && (gi == 0 || gi == n - 1)) { l = T(0); c = T(0); d = T(1); rhs = T(0); }
  };
  resident_solve<T, NT, C>(x, ah, ch, rows, n, per, sm);
#pragma unroll
  for (int j = 0; j < C; ++j)
    if (base + j < n) v[j] = comp_add(v[j], x[j], lo[j]);
}

template <typename T, int NT>
struct AdjShared {
  BtcsShared<T, NT> bt;
  Xch<T, NT> xa, xb;
  double red[NT / 32];
};

template <typename T, int NT, int C, int SCHEME>
__global__ void __launch_bounds__(NT) k_adjoint(const T* __restrict__ u0, const T* gT,
                                                T* gu0, double* __restrict__ gnu,
                                                const RowDesc* __restrict__ rows,
                                                const AdjRow* __restrict__ arows, int count,
                                                int* __restrict__ counter, T* __restrict__ ws) {
  __shared__ AdjShared<T, NT> sm;
  __shared__ int s_item;
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= count) return;
    const RowDesc rd = rows[item];
    const AdjRow ar = arows[item];
    const int n = rd.n, base = tid * C, jstar = n - 1 - base;
    const bool per = rd.bc == BC_PERIODIC;
    const T r = T(rd.r), s = T(rd.s), h = T(0.5 * rd.r);
    const int64_t ns = rd.nsteps, k = ar.stride;
    // Stored states use the kernel's own layout, element (j, thread) at
    // j * NT + tid of a CAP-value slot, so that every store and load of a
    // warp is one contiguous line. Checkpoints: ar.nckpt slots (FP32: each
    // followed by a slot of Kahan terms); segment states: k + 1 slots.
    constexpr int CAP = NT * C;
    constexpr int CKW = Kahan<T>::on ? 2 : 1;
    T* ck = ws + ar.ckpt;
    T* sg = ws + ar.seg;
    int p = 0;
    T v[C], lo[C];
#pragma unroll
    for (int j = 0; j < C; ++j) {
      v[j] = base + j < n ? u0[rd.offset + base + j] : T(0);
      lo[j] = T(0);
    }
    // ---- forward pass with checkpoints every k steps
    for (int64_t st = 0; st < ns; ++st) {
      if (st % k == 0) {
        T* dst = ck + (st / k) * CAP * CKW;
#pragma unroll
        for (int j = 0; j < C; ++j) {
          dst[j * NT + tid] = v[j];
          if constexpr (Kahan<T>::on) dst[CAP + j * NT + tid] = lo[j];
        }
      }
      if (st + 1 == ns) break;  // the last state is not needed
      if constexpr (SCHEME == 0) fwd_explicit_step<T, NT, C>(v, lo, n, base, per, r, h, s, sm.xa, p);
      else fwd_btcs_step<T, NT, C>(v, lo, n, base, per, r, s, sm.bt, sm.xa, p);
    }
    // ---- reverse pass. lambda advances in increment form, lambda' = lambda +
    // dlam (explicit: the transposed stencil minus lambda; BTCS: mu - lambda
    // from the increment form of the transposed solve, minus the coefficient
    // term); FP32 keeps a split state, lambda = lam + lamd with lamd the
    // increments since the last fold, folded every SPLIT_FOLD reverse steps.
    constexpr bool SPLIT = Kahan<T>::on;
    T lam[C], lamd[C];
#pragma unroll
    for (int j = 0; j < C; ++j) {
      lam[j] = base + j < n ? gT[rd.offset + base + j] : T(0);
      lamd[j] = T(0);
    }
    int64_t nrev = 0;
    double gacc = 0.0;
    NuSum nus;  // FP32: this fold block's dJ/dnu partial sum
    const int64_t nseg = ns > 0 ? (ns + k - 1) / k : 0;
    for (int64_t sgi = nseg - 1; sgi >= 0; --sgi) {
      const int64_t s0 = sgi * k;
      const int64_t s1 = (s0 + k < ns) ? s0 + k : ns;
      // recompute the states s0 .. s1 (BTCS needs u^{s+1}; explicit only u^s)
      const T* src = ck + sgi * CAP * CKW;
#pragma unroll
      for (int j = 0; j < C; ++j) {
        v[j] = base + j < n ? src[j * NT + tid] : T(0);
        if constexpr (Kahan<T>::on) lo[j] = base + j < n ? src[CAP + j * NT + tid] : T(0);
      }
      const int64_t last = SCHEME == 0 ? s1 - 1 : s1;
      for (int64_t st = s0; st <= last; ++st) {
        T* dst = sg + (st - s0) * CAP;
#pragma unroll
        for (int j = 0; j < C; ++j) dst[j * NT + tid] = v[j];
        if (st == last) break;
        if constexpr (SCHEME == 0) fwd_explicit_step<T, NT, C>(v, lo, n, base, per, r, h, s, sm.xa, p);
        else fwd_btcs_step<T, NT, C>(v, lo, n, base, per, r, s, sm.bt, sm.xa, p);
      }
      // reverse through the segment; the state of the next (earlier) step is
      // loaded while this one computes, and BTCS takes u^{s+1} from the
      // previous iteration's u^s
      T vn[C], vx[C];
      {
        const T* us = sg + (s1 - 1 - s0) * CAP;
#pragma unroll
        for (int j = 0; j < C; ++j) vn[j] = base + j < n ? us[j * NT + tid] : T(0);
        if constexpr (SCHEME == 1) {
          const T* ux = sg + (s1 - s0) * CAP;  // u^{s1}
#pragma unroll
          for (int j = 0; j < C; ++j) vx[j] = base + j < n ? ux[j * NT + tid] : T(0);
        }
      }
      for (int64_t st = s1 - 1; st >= s0; --st) {
#pragma unroll
        for (int j = 0; j < C; ++j) v[j] = vn[j];
        if (st > s0) {
          const T* us = sg + (st - 1 - s0) * CAP;
#pragma unroll
          for (int j = 0; j < C; ++j) vn[j] = base + j < n ? us[j * NT + tid] : T(0);
        }
        T part = T(0);
        T w[C];  // lambda of this step
#pragma unroll
        for (int j = 0; j < C; ++j) w[j] = SPLIT ? lam[j] + lamd[j] : lam[j];
        if constexpr (SCHEME == 0) {
          // transposed explicit step
          xch_publish<T, NT, C>(v, jstar, sm.xa, p);
          xch_publish<T, NT, C>(w, jstar, sm.xb, p);
          __syncthreads();
          T ul0, ur0, uw, ll0, lr0, lw;
          xch_read<T, NT>(sm.xa, p, ul0, ur0, uw);
          xch_read<T, NT>(sm.xb, p, ll0, lr0, lw);
          p ^= 1;
#pragma unroll
          for (int j = 0; j < C; ++j) {
            const int gi = base + j;
            T ul, ur, ll, lr;
            nbrs<T, C>(v, j, jstar, ul0, ur0, uw, ul, ur);
            nbrs<T, C>(w, j, jstar, ll0, lr0, lw, ll, lr);
            const T u = v[j];
            const bool upI = per || (gi > 0 && gi < n - 1);
            const bool upR = per || (gi + 1 < n - 1);
            const bool upL = per || (gi - 1 > 0);
            const T dl = u - ul, dr = ur - u;
            // 1 - diagonal of the step's Jacobian
            const T cI = upI ? tfma(r, (u > T(0) ? dl : dr) + tabs(u), T(2) * s) : T(0);
            T inc = -cI * w[j];
            if (upR) inc = tfma(tfma(r, tmax(ur, T(0)), s), lr, inc);
            if (upL) inc = tfma(tfma(-r, tmin(ul, T(0)), s), ll, inc);
            if (upI) part = tfma(w[j], dr - dl, part);
            if (gi >= n) inc = T(0);
            if constexpr (SPLIT) lamd[j] += inc;
            else lam[j] = w[j] + inc;
          }
        } else {
          // transposed BTCS step in increment form: with mu = lam + nu,
          // A^T nu = lam - A^T lam, whose right-hand side is minus the
          // off-identity part of the transposed rows applied to lam; then
          // lam' = mu - mu drow = lam + (nu - mu drow)
          xch_publish<T, NT, C>(v, jstar, sm.xa, p);
          xch_publish<T, NT, C>(w, jstar, sm.xb, p);
          __syncthreads();
          T ul0, ur0, uw, ll0, lr0, lw;
          xch_read<T, NT>(sm.xa, p, ul0, ur0, uw);
          xch_read<T, NT>(sm.xb, p, ll0, lr0, lw);
          p ^= 1;
          T nu[C], ah[C], ch[C];
          auto trows = [&](int j, T& l, T& d, T& c, T& rhs) {
            const int gi = base + j;
            T ul, ur, ll, lr;
            nbrs<T, C>(v, j, jstar, ul0, ur0, uw, ul, ur);
            nbrs<T, C>(w, j, jstar, ll0, lr0, lw, ll, lr);
            T l0, d0, c0, lm, dm, cm, lp, dp, cp;
            btcs_coef(v[j], r, s, l0, d0, c0);
            btcs_coef(ul, r, s, lm, dm, cm);
            btcs_coef(ur, r, s, lp, dp, cp);
            const bool bI = !per && (gi == 0 || gi == n - 1);
            const bool bL = !per && (gi - 1 == 0);       // row i-1 is an identity row
            const bool bR = !per && (gi + 1 == n - 1);   // row i+1 is an identity row
            l = (bL || (!per && gi == 0)) ? T(0) : cm;   // sub-diagonal: c_{i-1}
            c = (bR || (!per && gi == n - 1)) ? T(0) : lp;  // super-diagonal: l_{i+1}
            d = bI ? T(1) : d0;
            const T dm1 = bI ? T(0) : tfma(r, tabs(v[j]), T(2) * s);  // d - 1
            rhs = -tfma(l, ll, tfma(c, lr, dm1 * w[j]));
          };
          resident_solve<T, NT, C>(nu, ah, ch, trows, n, per, sm.bt);
          T (&xv)[C] = vx;  // x = u^{s+1}
          // its neighbours across the chunk edges, read from the stored state
          // (the values an exchange of xv would give, without its barrier)
          T xl0, xr0, xw;
          {
            const T* ux = sg + (st + 1 - s0) * CAP;
            const int tn = (n - 1) / C, jn = (n - 1) - tn * C;
            xw = ux[0];
            xl0 = tid > 0 ? ux[(C - 1) * NT + tid - 1] : ux[jn * NT + tn];
            xr0 = tid + 1 < NT ? ux[tid + 1] : xw;
          }
#pragma unroll
          for (int j = 0; j < C; ++j) {
            const int gi = base + j;
            T xl, xr;
            nbrs<T, C>(xv, j, jstar, xl0, xr0, xw, xl, xr);
            const bool bI = !per && (gi == 0 || gi == n - 1);
            const T H = v[j] > T(0) ? T(1) : T(0);
            const T drow = r * (-H * xl + (T(2) * H - T(1)) * xv[j] + (T(1) - H) * xr);
            const T mu = w[j] + nu[j];
            T inc = bI ? nu[j] : tfma(-mu, drow, nu[j]);
            if (!bI && gi < n) part = tfma(mu, xr - T(2) * xv[j] + xl, part);
            if (gi >= n) inc = T(0);
            if constexpr (SPLIT) lamd[j] += inc;
            else lam[j] = w[j] + inc;
          }
#pragma unroll
          for (int j = 0; j < C; ++j) vx[j] = v[j];  // u^s is the next step's u^{s+1}
        }
        if constexpr (SPLIT) nus.add(part);
        else gacc += double(part);
        if constexpr (SPLIT) {
          if (++nrev % SPLIT_FOLD == 0) {
#pragma unroll
            for (int j = 0; j < C; ++j) {
              const T t = lam[j] + lamd[j];
              lamd[j] = lamd[j] - (t - lam[j]);
              lam[j] = t;
            }
            nus.fold(gacc);
          }
        }
      }
    }
    if constexpr (SPLIT) nus.fold(gacc);
    // ---- outputs
#pragma unroll
    for (int j = 0; j < C; ++j)
      if (base + j < n) gu0[rd.offset + base + j] = SPLIT ? lam[j] + lamd[j] : lam[j];
    // block reduction of the nu gradient (FP64)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) gacc += __shfl_xor_sync(FULL_MASK, gacc, o);
    if ((tid & 31) == 0) sm.red[tid >> 5] = gacc;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < NT / 32; ++w) t += sm.red[w];
      gnu[ar.out_index] = t * rd.ds_dnu;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Explicit scheme, rows of exactly NT*C nodes. Same adjoint as k_adjoint
// (forward pass with checkpoints every k steps, per segment a recompute that
// stores the states, then the transposed steps backwards through them), with
// the forward step of k_explicit_resident: FP32 evaluates the split state
// u = uh + d and folds d into uh after every step whose global index + 1 is a
// multiple of SPLIT_FOLD, so the checkpoint pass and every recompute follow
// the same rounding and give the main kernel's trajectory; FP64 updates in
// place. Neighbour values move branch-free (shuffles inside a warp, one
// predicated shared-memory store per warp edge and one barrier per exchange,
// u and lambda together in the reverse step), and the boundary cases of
// Dirichlet rows are the handful of nodes next to the row's ends.
template <typename T, int NT>
struct AdjFastShared {
  static constexpr int NW = NT / 32;
  T slot[2][2][2][NW];  // [parity][0: first of a warp, 1: last][quantity][warp]
  double red[NW];
};

// Exchanges K quantities' chunk-edge values: left[k] = value of quantity k
// at the node before this thread's first, right[k] after its last (periodic
// wrap through the first and last warp).
template <typename T, int NT, int K>
__device__ __forceinline__ void adj_xch(const T (&first)[K], const T (&last)[K], int p,
                                        AdjFastShared<T, NT>& sh, T (&left)[K], T (&right)[K]) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    left[k] = shfl(last[k], (lane + 31) & 31);
    right[k] = shfl(first[k], (lane + 1) & 31);
  }
  if constexpr (NW > 1) {
    const bool lo_lane = lane == 0;
#pragma unroll
    for (int k = 0; k < K; ++k)
      st_shared_if(&sh.slot[p][lo_lane ? 0 : 1][k][warp], lo_lane ? first[k] : last[k],
                   lo_lane || lane == 31);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const T lv = sh.slot[p][1][k][(warp + NW - 1) % NW];
      const T rv = sh.slot[p][0][k][(warp + 1) % NW];
      left[k] = lane == 0 ? lv : left[k];
      right[k] = lane == 31 ? rv : right[k];
    }
  }
}

// One forward step (Eq. 21) of the global step index `st`.
template <typename T, int NT, int C, int BCT>
__device__ __forceinline__ void adj_fwd_step(T (&v)[C], T (&d)[C], int64_t st, int& p, T r, T h,
                                             T s, AdjFastShared<T, NT>& sh) {
  constexpr bool SPLIT = Kahan<T>::on;
  const int tid = threadIdx.x;
  auto w = [&](int j) -> T { return SPLIT ? v[j] + d[j] : v[j]; };
  T fl[1] = {w(0)}, la[1] = {w(C - 1)}, L[1], R[1];
  adj_xch<T, NT, 1>(fl, la, p, sh, L, R);
  p ^= 1;
  T wl = L[0], wc = fl[0];
#pragma unroll
  for (int j = 0; j < C; ++j) {
    const T wr = (j + 1 < C) ? w(j + 1) : R[0];
    bool keep = false;
    if constexpr (BCT == BC_DIRICHLET) keep = (j == 0 && tid == 0) || (j == C - 1 && tid == NT - 1);
    if constexpr (SPLIT) {
      const T dn = explicit_increment(wc, wl, wr, r, h, s, d[j]);
      if (!keep) d[j] = dn;
    } else {
      const T nv = explicit_increment(wc, wl, wr, r, h, s, wc);
      if (!keep) v[j] = nv;
    }
    wl = wc;
    wc = wr;
  }
  if constexpr (SPLIT) {
    if ((st + 1) % SPLIT_FOLD == 0) {
#pragma unroll
      for (int j = 0; j < C; ++j) {
        const T t = v[j] + d[j];
        d[j] = d[j] - (t - v[j]);
        v[j] = t;
      }
    }
  }
}

template <typename T, int NT, int C, int BCT>
__device__ __forceinline__ void adj_explicit_exact_row(const T* __restrict__ u0, const T* gT,
                                                       T* gu0, double* __restrict__ gnu,
                                                       const RowDesc& rd, const AdjRow& ar,
                                                       T* __restrict__ ws,
                                                       AdjFastShared<T, NT>& sh) {
  constexpr bool SPLIT = Kahan<T>::on;
  constexpr int CAP = NT * C, CKW = SPLIT ? 2 : 1;
  const int tid = threadIdx.x, base = tid * C;
  const T r = T(rd.r), s = T(rd.s), h = T(0.5 * rd.r);
  const int64_t ns = rd.nsteps, k = ar.stride;
  T* ck = ws + ar.ckpt;
  T* sg = ws + ar.seg;
  int p = 0;
  T v[C], d[C];
#pragma unroll
  for (int j = 0; j < C; ++j) {
    v[j] = u0[rd.offset + base + j];
    d[j] = T(0);
  }
  // ---- forward pass with checkpoints every k steps
  for (int64_t st = 0; st < ns; ++st) {
    if (st % k == 0) {
      T* dst = ck + (st / k) * CAP * CKW;
#pragma unroll
      for (int j = 0; j < C; ++j) {
        dst[j * NT + tid] = v[j];
        if constexpr (SPLIT) dst[CAP + j * NT + tid] = d[j];
      }
    }
    if (st + 1 == ns) break;  // the last state is not needed
    adj_fwd_step<T, NT, C, BCT>(v, d, st, p, r, h, s, sh);
  }
  // ---- reverse pass. lambda advances in increment form, lambda' = lambda +
  // dlam with dlam = -(2s + r(H dl + (1-H) dr + |u|)) lambda + (s + r u_{i+1}^+)
  // lambda_{i+1} + (s - r u_{i-1}^-) lambda_{i-1}; FP32 keeps it as a split
  // state (lh, the value at the last fold, plus ld, the increments summed
  // since), evaluates the transposed stencil on lh + ld and folds ld into lh
  // every SPLIT_FOLD reverse steps, so the rounding of lambda + dlam is not
  // accumulated over the steps (plain FP32 accumulation drifts by ~6e-5 of
  // the gradient over 2000 steps).
  T lam[C], lamd[C];
#pragma unroll
  for (int j = 0; j < C; ++j) {
    lam[j] = gT[rd.offset + base + j];
    lamd[j] = T(0);
  }
  double gacc = 0.0;
  NuSum nus;  // FP32: this fold block's dJ/dnu partial sum
  int64_t nrev = 0;  // reverse steps taken (fold schedule)
  const int64_t nseg = ns > 0 ? (ns + k - 1) / k : 0;
  for (int64_t sgi = nseg - 1; sgi >= 0; --sgi) {
    const int64_t s0 = sgi * k;
    const int64_t s1 = (s0 + k < ns) ? s0 + k : ns;
    // recompute the states s0 .. s1 - 1 (u = uh + d for FP32)
    {
      const T* src = ck + sgi * CAP * CKW;
#pragma unroll
      for (int j = 0; j < C; ++j) {
        v[j] = src[j * NT + tid];
        d[j] = SPLIT ? src[CAP + j * NT + tid] : T(0);
      }
    }
    for (int64_t st = s0; st < s1; ++st) {
      T* dst = sg + (st - s0) * CAP;
#pragma unroll
      for (int j = 0; j < C; ++j) dst[j * NT + tid] = SPLIT ? v[j] + d[j] : v[j];
      if (st + 1 == s1) break;
      adj_fwd_step<T, NT, C, BCT>(v, d, st, p, r, h, s, sh);
    }
    // transposed steps backwards through the segment; the state of the next
    // (earlier) step is loaded while this one computes
    T vn[C];
    {
      const T* us = sg + (s1 - 1 - s0) * CAP;
#pragma unroll
      for (int j = 0; j < C; ++j) vn[j] = us[j * NT + tid];
    }
    for (int64_t st = s1 - 1; st >= s0; --st) {
#pragma unroll
      for (int j = 0; j < C; ++j) v[j] = vn[j];
      if (st > s0) {
        const T* us = sg + (st - 1 - s0) * CAP;
#pragma unroll
        for (int j = 0; j < C; ++j) vn[j] = us[j * NT + tid];
      }
      T w[C];  // lambda of this step
#pragma unroll
      for (int j = 0; j < C; ++j) w[j] = SPLIT ? lam[j] + lamd[j] : lam[j];
      T fl[2] = {v[0], w[0]}, la[2] = {v[C - 1], w[C - 1]}, L[2], R[2];
      adj_xch<T, NT, 2>(fl, la, p, sh, L, R);
      p ^= 1;
      T ul = L[0], ll = L[1], part = T(0);
#pragma unroll
      for (int j = 0; j < C; ++j) {
        const T u = v[j];
        const T ur = (j + 1 < C) ? v[j + 1] : R[0];
        const T lr = (j + 1 < C) ? w[j + 1] : R[1];
        bool upI = true, upR = true, upL = true;  // node, right, left neighbour updated
        if constexpr (BCT == BC_DIRICHLET) {
          const int gi = base + j;  // the row has CAP nodes; 0 and CAP - 1 are held
          upI = gi != 0 && gi != CAP - 1;
          upR = gi + 1 < CAP - 1;
          upL = gi - 1 > 0;
        }
        const T dl = u - ul, dr = ur - u;
        // 1 - diagonal of the step's Jacobian
        const T cI = upI ? tfma(r, (u > T(0) ? dl : dr) + tabs(u), T(2) * s) : T(0);
        T inc = -cI * w[j];
        if (upR) inc = tfma(tfma(r, tmax(ur, T(0)), s), lr, inc);
        if (upL) inc = tfma(tfma(-r, tmin(ul, T(0)), s), ll, inc);
        if (upI) part = tfma(w[j], dr - dl, part);
        if constexpr (SPLIT) lamd[j] += inc;
        else lam[j] = w[j] + inc;
        ul = u;
        ll = w[j];
      }
      if constexpr (SPLIT) nus.add(part);
      else gacc += double(part);
      if constexpr (SPLIT) {
        if (++nrev % SPLIT_FOLD == 0) {
#pragma unroll
          for (int j = 0; j < C; ++j) {
            const T t = lam[j] + lamd[j];
            lamd[j] = lamd[j] - (t - lam[j]);
            lam[j] = t;
          }
          nus.fold(gacc);
        }
      }
    }
  }
  if constexpr (SPLIT) nus.fold(gacc);
  // ---- outputs
#pragma unroll
  for (int j = 0; j < C; ++j) gu0[rd.offset + base + j] = SPLIT ? lam[j] + lamd[j] : lam[j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) gacc += __shfl_xor_sync(FULL_MASK, gacc, o);
  if ((tid & 31) == 0) sh.red[tid >> 5] = gacc;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < NT / 32; ++w) t += sh.red[w];
    gnu[ar.out_index] = t * rd.ds_dnu;
  }
  __syncthreads();
}

// FP32 rows of exactly NT*C nodes with C even: the same adjoint on packed
// f32x2 pairs (nodes k and k + C/2 of a thread's chunk, as in the forward
// kernel). The forward step is that of explicit_steps_split_x2 (bitwise the
// scalar step above: p = s - r min(u, 0) is the rounding of s + (r/2)(|u| - u),
// -q = -(s + r max(u, 0))), folded on the same global step index, so the
// checkpoints and recomputes are those of the scalar form; the stored states
// are pairs, [k][thread]. The reverse step applies the transposed stencil to
// both nodes of a pair at once; the nu gradient sums each lane's nodes
// separately (two partial sums per thread).
template <int NT, int C, int BCT>
__device__ __forceinline__ void adj_fwd_step_x2(float2 (&V)[C / 2], float2 (&D)[C / 2], int64_t st,
                                                int& p, float r, float s,
                                                AdjFastShared<float, NT>& sh) {
  constexpr int H = C / 2;
  const int tid = threadIdx.x;
  const float2 NR = make_float2(-r, -r), S2 = make_float2(s, s), NS = make_float2(-s, -s);
  const float2 U0 = add2(V[0], D[0]);
  const float2 UL = add2(V[H - 1], D[H - 1]);
  float fl[1] = {U0.x}, la[1] = {UL.y}, L[1], R[1];
  adj_xch<float, NT, 1>(fl, la, p, sh, L, R);
  p ^= 1;
  float2 Uk = U0;
  float2 DL = sub2(U0, make_float2(L[0], UL.x));  // u - u_l of pair 0
#pragma unroll
  for (int k = 0; k < H; ++k) {
    const float2 UR = (k + 1 < H) ? add2(V[k + 1], D[k + 1]) : make_float2(U0.y, R[0]);
    const float2 E = sub2(UR, Uk);  // u_r - u
    const float2 m = make_float2(fminf(Uk.x, 0.f), fminf(Uk.y, 0.f));
    const float2 M = make_float2(fmaxf(Uk.x, 0.f), fmaxf(Uk.y, 0.f));
    const float2 P = fma2(NR, m, S2);   // p
    const float2 NQ = fma2(NR, M, NS);  // -q
    const float2 dn = fma2(P, E, fma2(NQ, DL, D[k]));
    bool keepx = false, keepy = false;
    if constexpr (BCT == BC_DIRICHLET) {
      keepx = k == 0 && tid == 0;
      keepy = k == H - 1 && tid == NT - 1;
    }
    if (!keepx) D[k].x = dn.x;
    if (!keepy) D[k].y = dn.y;
    DL = E;
    Uk = UR;
  }
  if ((st + 1) % SPLIT_FOLD == 0) {
#pragma unroll
    for (int k = 0; k < H; ++k) {
      const float2 t = add2(V[k], D[k]);
      D[k] = sub2(D[k], sub2(t, V[k]));
      V[k] = t;
    }
  }
}

template <int NT, int C, int BCT>
__device__ __forceinline__ void adj_explicit_exact_row_x2(const float* __restrict__ u0,
                                                          const float* gT, float* gu0,
                                                          double* __restrict__ gnu,
                                                          const RowDesc& rd, const AdjRow& ar,
                                                          float* __restrict__ ws,
                                                          AdjFastShared<float, NT>& sh) {
  constexpr int H = C / 2, CAP = NT * C, HP = NT * H;  // a state slot: HP pairs
  const int tid = threadIdx.x, base = tid * C;
  const float r = float(rd.r), s = float(rd.s);
  const int64_t ns = rd.nsteps, k = ar.stride;
  float2* ck = reinterpret_cast<float2*>(ws + ar.ckpt);  // (V, D) pairs per checkpoint
  float2* sg = reinterpret_cast<float2*>(ws + ar.seg);   // u pairs per segment state
  int p = 0;
  float2 V[H], D[H];
#pragma unroll
  for (int q = 0; q < H; ++q) {
    V[q] = make_float2(u0[rd.offset + base + q], u0[rd.offset + base + q + H]);
    D[q] = make_float2(0.f, 0.f);
  }
  // ---- forward pass with checkpoints every k steps
  for (int64_t st = 0; st < ns; ++st) {
    if (st % k == 0) {
      float2* dst = ck + (st / k) * 2 * HP;
#pragma unroll
      for (int q = 0; q < H; ++q) {
        dst[q * NT + tid] = V[q];
        dst[HP + q * NT + tid] = D[q];
      }
    }
    if (st + 1 == ns) break;
    adj_fwd_step_x2<NT, C, BCT>(V, D, st, p, r, s, sh);
  }
  // ---- reverse pass (split lambda state, folded every SPLIT_FOLD steps)
  float2 LH[H], LD[H];
#pragma unroll
  for (int q = 0; q < H; ++q) {
    LH[q] = make_float2(gT[rd.offset + base + q], gT[rd.offset + base + q + H]);
    LD[q] = make_float2(0.f, 0.f);
  }
  const float2 R2 = make_float2(r, r), NR2 = make_float2(-r, -r), S2 = make_float2(s, s);
  const float2 TS2 = make_float2(2.f * s, 2.f * s), Z2 = make_float2(0.f, 0.f);
  double gacc = 0.0;
  NuSum2 nus;  // this fold block's dJ/dnu partial sums
  int64_t nrev = 0;
  const int64_t nseg = ns > 0 ? (ns + k - 1) / k : 0;
  for (int64_t sgi = nseg - 1; sgi >= 0; --sgi) {
    const int64_t s0 = sgi * k;
    const int64_t s1 = (s0 + k < ns) ? s0 + k : ns;
    {
      const float2* src = ck + sgi * 2 * HP;
#pragma unroll
      for (int q = 0; q < H; ++q) {
        V[q] = src[q * NT + tid];
        D[q] = src[HP + q * NT + tid];
      }
    }
    for (int64_t st = s0; st < s1; ++st) {
      float2* dst = sg + (st - s0) * HP;
#pragma unroll
      for (int q = 0; q < H; ++q) dst[q * NT + tid] = add2(V[q], D[q]);
      if (st + 1 == s1) break;
      adj_fwd_step_x2<NT, C, BCT>(V, D, st, p, r, s, sh);
    }
    float2 UN[H];
    {
      const float2* us = sg + (s1 - 1 - s0) * HP;
#pragma unroll
      for (int q = 0; q < H; ++q) UN[q] = us[q * NT + tid];
    }
    for (int64_t st = s1 - 1; st >= s0; --st) {
      float2 U[H];
#pragma unroll
      for (int q = 0; q < H; ++q) U[q] = UN[q];
      if (st > s0) {
        const float2* us = sg + (st - 1 - s0) * HP;
#pragma unroll
        for (int q = 0; q < H; ++q) UN[q] = us[q * NT + tid];
      }
      float2 W[H];  // lambda of this step
#pragma unroll
      for (int q = 0; q < H; ++q) W[q] = add2(LH[q], LD[q]);
      float fl[2] = {U[0].x, W[0].x}, la[2] = {U[H - 1].y, W[H - 1].y}, L[2], R[2];
      adj_xch<float, NT, 2>(fl, la, p, sh, L, R);
      p ^= 1;
      float2 ul = make_float2(L[0], U[H - 1].x), ll = make_float2(L[1], W[H - 1].x);
      float2 part = Z2;
#pragma unroll
      for (int q = 0; q < H; ++q) {
        const float2 u = U[q];
        const float2 ur = (q + 1 < H) ? U[q + 1] : make_float2(U[0].y, R[0]);
        const float2 lr = (q + 1 < H) ? W[q + 1] : make_float2(W[0].y, R[1]);
        const float2 dl = sub2(u, ul), dr = sub2(ur, u);
        // 1 - diagonal of the step's Jacobian: r ((u > 0 ? dl : dr) + |u|) + 2s
        const float2 sel = make_float2(u.x > 0.f ? dl.x : dr.x, u.y > 0.f ? dl.y : dr.y);
        const float2 cI = fma2(R2, add2(sel, make_float2(fabsf(u.x), fabsf(u.y))), TS2);
        float2 inc = mul2(make_float2(-cI.x, -cI.y), W[q]);
        const float2 incR = fma2(fma2(R2, make_float2(fmaxf(ur.x, 0.f), fmaxf(ur.y, 0.f)), S2), lr, inc);
        const float2 incRL = fma2(fma2(NR2, make_float2(fminf(ul.x, 0.f), fminf(ul.y, 0.f)), S2), ll, incR);
        const float2 pn = fma2(W[q], sub2(dr, dl), part);
        if constexpr (BCT == BC_DIRICHLET) {
          // rows 0 and CAP - 1 are held: no update of their own, none sent
          // to or taken from them by their neighbours
          const int gx = base + q, gy = base + q + H;
          const bool upIx = gx != 0 && gx != CAP - 1, upIy = gy != 0 && gy != CAP - 1;
          const bool upRx = gx + 1 < CAP - 1, upRy = gy + 1 < CAP - 1;
          const bool upLx = gx - 1 > 0, upLy = gy - 1 > 0;
          float2 ix = make_float2(upIx ? inc.x : 0.f, upIy ? inc.y : 0.f);
          // replay the scalar order: -cI w, then the right term, then the left
          if (upRx) ix.x = fmaf(fmaf(r, fmaxf(ur.x, 0.f), s), lr.x, ix.x);
          if (upRy) ix.y = fmaf(fmaf(r, fmaxf(ur.y, 0.f), s), lr.y, ix.y);
          if (upLx) ix.x = fmaf(fmaf(-r, fminf(ul.x, 0.f), s), ll.x, ix.x);
          if (upLy) ix.y = fmaf(fmaf(-r, fminf(ul.y, 0.f), s), ll.y, ix.y);
          part = make_float2(upIx ? pn.x : part.x, upIy ? pn.y : part.y);
          LD[q] = add2(LD[q], ix);
        } else {
          part = pn;
          LD[q] = add2(LD[q], incRL);
        }
        ul = u;
        ll = W[q];
      }
      nus.add(part);
      if (++nrev % SPLIT_FOLD == 0) {
#pragma unroll
        for (int q = 0; q < H; ++q) {
          const float2 t = add2(LH[q], LD[q]);
          LD[q] = sub2(LD[q], sub2(t, LH[q]));
          LH[q] = t;
        }
        nus.fold(gacc);
      }
    }
  }
  nus.fold(gacc);
  // ---- outputs
#pragma unroll
  for (int q = 0; q < H; ++q) {
    const float2 g = add2(LH[q], LD[q]);
    gu0[rd.offset + base + q] = g.x;
    gu0[rd.offset + base + q + H] = g.y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) gacc += __shfl_xor_sync(FULL_MASK, gacc, o);
  if ((tid & 31) == 0) sh.red[tid >> 5] = gacc;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < NT / 32; ++w) t += sh.red[w];
    gnu[ar.out_index] = t * rd.ds_dnu;
  }
  __syncthreads();
}

// Persistent CTAs take rows from an atomic counter.
template <typename T, int NT, int C>
__device__ __forceinline__ void adj_explicit_exact_rows(
    const T* __restrict__ u0, const T* gT, T* gu0, double* __restrict__ gnu,
    const RowDesc* __restrict__ rows, const AdjRow* __restrict__ arows, int count,
    int* __restrict__ counter, T* __restrict__ ws) {
  __shared__ AdjFastShared<T, NT> sh;
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= count) return;
    const RowDesc rd = rows[item];
    const AdjRow ar = arows[item];
    // packed pairs for 16 nodes a thread (at 8 the packed form needed 106
    // registers against the scalar form's 80)
    if constexpr (sizeof(T) == 4 && C == 16) {
      if (rd.bc == BC_PERIODIC)
        adj_explicit_exact_row_x2<NT, C, BC_PERIODIC>(u0, gT, gu0, gnu, rd, ar, ws, sh);
      else
        adj_explicit_exact_row_x2<NT, C, BC_DIRICHLET>(u0, gT, gu0, gnu, rd, ar, ws, sh);
    } else if (rd.bc == BC_PERIODIC) {
      adj_explicit_exact_row<T, NT, C, BC_PERIODIC>(u0, gT, gu0, gnu, rd, ar, ws, sh);
    } else {
      adj_explicit_exact_row<T, NT, C, BC_DIRICHLET>(u0, gT, gu0, gnu, rd, ar, ws, sh);
    }
  }
}

template <typename T, int NT, int C>
__global__ void __launch_bounds__(NT) k_adjoint_explicit_exact(
    const T* __restrict__ u0, const T* gT, T* gu0, double* __restrict__ gnu,
    const RowDesc* __restrict__ rows, const AdjRow* __restrict__ arows, int count,
    int* __restrict__ counter, T* __restrict__ ws) {
  adj_explicit_exact_rows<T, NT, C>(u0, gT, gu0, gnu, rows, arows, count, counter, ws);
}

// FP32 on packed pairs, 16 nodes a thread, capped at 512 threads a SM (128
// registers; uncapped the packed form takes 160 and runs three CTAs of 128).
// Its own kernel: a minimum-blocks bound on the other shapes, even 1, moves
// ptxas to more registers for them.
template <int NT>
__global__ void __launch_bounds__(NT, 512 / NT) k_adjoint_explicit_exact_x2(
    const float* __restrict__ u0, const float* gT, float* gu0, double* __restrict__ gnu,
    const RowDesc* __restrict__ rows, const AdjRow* __restrict__ arows, int count,
    int* __restrict__ counter, float* __restrict__ ws) {
  static_assert(NT <= 512, "at least one CTA a SM");
  adj_explicit_exact_rows<float, NT, 16>(u0, gT, gu0, gnu, rows, arows, count, counter, ws);
}

template <typename T, int NT, int C>
const void* adj_exact_kernel() {
  if constexpr (sizeof(T) == 4 && C == 16)
    return reinterpret_cast<const void*>(&k_adjoint_explicit_exact_x2<NT>);
  else
    return reinterpret_cast<const void*>(&k_adjoint_explicit_exact<T, NT, C>);
}

#define REG_ADJ(T, DT, NT, C)                                                                      \
  reg.push_back({K_ADJ_EXPLICIT, DT, NT, C, 0, reinterpret_cast<const void*>(&k_adjoint<T, NT, C, 0>), \
                 0});                                                                              \
  reg.push_back({K_ADJ_EXPLICIT, DT, NT, C, 1, adj_exact_kernel<T, NT, C>(), 0});                  \
  reg.push_back({K_ADJ_BTCS, DT, NT, C, 0, reinterpret_cast<const void*>(&k_adjoint<T, NT, C, 1>), 0});

void register_adjoint(std::vector<KernelEntry>& reg) {
  REG_ADJ(float, 0, 32, 1) REG_ADJ(float, 0, 32, 4) REG_ADJ(float, 0, 64, 8)
  REG_ADJ(float, 0, 128, 8) REG_ADJ(float, 0, 128, 16) REG_ADJ(float, 0, 256, 16)
  REG_ADJ(double, 1, 32, 1) REG_ADJ(double, 1, 32, 4) REG_ADJ(double, 1, 64, 8)
  REG_ADJ(double, 1, 128, 8) REG_ADJ(double, 1, 256, 8)
}


// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {
struct AShape {
  int nt, c;
};
const AShape kAdj32[] = {{32, 1}, {32, 4}, {64, 8}, {128, 8}, {128, 16}, {256, 16}};
const AShape kAdj64[] = {{32, 1}, {32, 4}, {64, 8}, {128, 8}, {256, 8}};
}  // namespace

int64_t adjoint_max_n(int dtype) { return dtype == 0 ? 256 * 16 : 256 * 8; }

burgers_status adjoint_run(burgers_ctx* ctx, int scheme, const burgers_batch* batch,
                           const void* u0, const void* gT, void* gu0, double* gnu,
                           int64_t stride, cudaStream_t st) {
  const int dtype = batch->dtype;
  const AShape* shapes = dtype == 0 ? kAdj32 : kAdj64;
  const int nshapes = dtype == 0 ? 6 : 5;
  const int kind = scheme == BURGERS_EXPLICIT ? K_ADJ_EXPLICIT : K_ADJ_BTCS;
  const size_t esz = dtype == 0 ? 4 : 8;
  // groups by (shape, exact): explicit rows of exactly nt * c nodes take the
  // k_adjoint_explicit_exact kernel of that shape
  std::vector<std::vector<std::pair<double, int64_t>>> groups(static_cast<size_t>(2 * nshapes));
  std::vector<int64_t> longs;  // explicit rows longer than one CTA holds (adjoint_long.cu)
  for (int64_t b = 0; b < batch->count; ++b) {
    const burgers_instance& in = batch->inst[b];
    if (in.n > adjoint_max_n(dtype)) {
      longs.push_back(b);
      continue;
    }
    int pick = -1;
    for (int i = 0; i < nshapes && pick < 0; ++i)
      if (int64_t(shapes[i].nt) * shapes[i].c >= in.n && shapes[i].c < in.n) pick = i;
    if (pick < 0) return set_error(BURGERS_EINVAL, "adjoint: no kernel shape fits the row");
    const bool ex = scheme == BURGERS_EXPLICIT && in.n == int64_t(shapes[pick].nt) * shapes[pick].c;
    groups[size_t(2 * pick + (ex ? 1 : 0))].emplace_back(double(in.n) * double(in.nsteps + 1), b);
  }
  std::vector<RowDesc> rows;
  std::vector<AdjRow> arows;
  std::vector<std::pair<int, int>> ranges;  // (shape, count)
  int64_t ws = 0;
  for (int gx = 0; gx < 2 * nshapes; ++gx) {
    const int g = gx / 2;
    auto& G = groups[size_t(gx)];
    if (G.empty()) continue;
    std::stable_sort(G.begin(), G.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    for (auto& pr : G) {
      const burgers_instance& in = batch->inst[pr.second];
      RowDesc d;
      d.offset = in.offset;
      d.nsteps = in.nsteps;
      d.r = in.dt / in.dx;
      d.s = in.nu * in.dt / (in.dx * in.dx);
      d.ds_dnu = in.dt / (in.dx * in.dx);
      d.n = in.n;
      d.bc = in.bc;
      set_fp32_coefs(d);
      AdjRow a;
      int64_t k = stride > 0 ? stride : int64_t(ceil(sqrt(double(std::max<int64_t>(in.nsteps, 1)))));
      if (k < 1) k = 1;
      a.stride = k;
      a.nckpt = in.nsteps > 0 ? (in.nsteps + k - 1) / k : 0;
      // state slots of the kernel shape's capacity (its [j][thread] layout)
      const int64_t cap = int64_t(shapes[g].nt) * shapes[g].c;
      a.ckpt = ws;
      ws += ((a.nckpt * cap * (dtype == 0 ? 2 : 1) + 63) / 64) * 64;
      a.seg = ws;
      ws += (((k + 1) * cap + 63) / 64) * 64;
      a.out_index = int32_t(pr.second);
      a.pad = 0;
      rows.push_back(d);
      arows.push_back(a);
    }
    ranges.emplace_back(gx, int(G.size()));
  }
  cudaError_t e = ctx->adjws.ensure(size_t(std::max<int64_t>(ws, 1)) * esz);
  if (e != cudaSuccess) return set_error(BURGERS_ENOMEM, "adjoint workspace: out of device memory");
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t o_rows = 0, o_arows = al(rows.size() * sizeof(RowDesc));
  const size_t o_ctr = al(o_arows + arows.size() * sizeof(AdjRow));
  const size_t total = al(o_ctr + ranges.size() * sizeof(int));
  e = ctx->adjdesc.ensure(total);
  if (e == cudaSuccess) e = ctx->adjhost.ensure_host(total);
  if (e != cudaSuccess) return set_error(BURGERS_ENOMEM, "adjoint descriptors");
  if (ctx->adj_event) {  // the previous upload must have left the staging buffer
    e = cudaEventSynchronize(ctx->adj_event);
    if (e != cudaSuccess) return cuda_error(e, "adjoint staging");
  } else {
    e = cudaEventCreateWithFlags(&ctx->adj_event, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_error(e, "cudaEventCreate");
  }
  char* h = static_cast<char*>(ctx->adjhost.hptr);
  memcpy(h + o_rows, rows.data(), rows.size() * sizeof(RowDesc));
  memcpy(h + o_arows, arows.data(), arows.size() * sizeof(AdjRow));
  memset(h + o_ctr, 0, ranges.size() * sizeof(int));
  char* dbase = static_cast<char*>(ctx->adjdesc.ptr);
  e = cudaMemcpyAsync(dbase, h, total, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->adj_event, st);
  if (e != cudaSuccess) return cuda_error(e, "adjoint upload");
  int begin = 0;
  for (size_t q = 0; q < ranges.size(); ++q) {
    const AShape sh = shapes[ranges[q].first / 2];
    const KernelEntry* k = find_kernel(kind, dtype, sh.nt, sh.c, ranges[q].first % 2);
    if (!k) return set_error(BURGERS_EINVAL, "adjoint kernel shape missing");
    int cnt = ranges[q].second;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k->fn, k->nt, 0) != cudaSuccess || occ < 1)
      occ = 1;
    int grid = std::min(cnt, ctx->sm_count * occ);
    const RowDesc* rp = reinterpret_cast<const RowDesc*>(dbase + o_rows) + begin;
    const AdjRow* ap = reinterpret_cast<const AdjRow*>(dbase + o_arows) + begin;
    int* ctr = reinterpret_cast<int*>(dbase + o_ctr) + q;
    void* wsp = ctx->adjws.ptr;
    void* args[] = {(void*)&u0, (void*)&gT, &gu0, &gnu, &rp, &ap, &cnt, &ctr, &wsp};
    e = cudaLaunchKernel(k->fn, dim3(grid), dim3(k->nt), args, 0, st);
    if (e != cudaSuccess) return cuda_error(e, "adjoint launch");
    ctx->launches += 1;
    begin += cnt;
  }
  if (!longs.empty())
    return adjoint_long_run(ctx, scheme, batch, longs, u0, gT, gu0, gnu, stride, st);
  return BURGERS_OK;
}

}  // namespace burgers
