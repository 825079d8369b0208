// btcs.cu -- implicit BTCS step with lagged upwind coefficients (Sec. 2.4,
// Eq. 23): A(u^n) u^{n+1} = u^n with, for node i and a = u^n_i,
//   l_i = -r a+ - s,   d_i = 1 + r|a| + 2s,   c_i = r a- - s,
// periodic rows cyclic (Eq. 18), Dirichlet end nodes held (Eq. 16-17, written
// here as identity rows). The coefficients are formed from u^n in registers and
// never stored.
//
// Partitioned elimination. Thread t owns a chunk of C consecutive rows with
// end row e. A forward sweep normalises each row to
//     x_i + ch_i x_{i+1} + ah_i L = dh_i          (L = x of the previous chunk's end)
// and a backward sweep turns the rows before e into
//     x_i = delta_i - alpha_i L - gamma_i X_t      (X_t = x_e).
// Substituting the next chunk's first-row relation into row e gives one
// tridiagonal row per chunk in the unknowns X_{t-1}, X_t, X_{t+1}: a reduced
// system of NT rows (cyclic for periodic rows). Warp 0 solves it: the
// cyclic corners are split off by Sherman-Morrison (gamma = -B_0, correction
// factor (v.y)/(1 + v.z) evaluated in FP64), each lane eliminates Q = NT/32
// reduced rows the same way, and the remaining 32-row system is solved by
// parallel cyclic reduction over warp shuffles. Back-substitution then
// recovers every node from delta, alpha, gamma and the chunk-end values.
//
// All pivots are >= 1 because every matrix involved is diagonally dominant by
// a margin of one (an M-matrix and its Schur complements), so no pivoting is
// needed.
#include "btcs_common.cuh"
#include "common.cuh"
#include "kernels.h"

namespace burgers {

// Advances the row held by this CTA `nsteps` BTCS steps; thread t owns nodes
// [tC, tC + C).
//
// Increment form: with a = u^n, A(u^n) u^n = u^n - Delta(u^n) where Delta is the
// explicit forward-Euler increment of the same r, s (Eq. 21), so the step is
//     A(u^n) delta = Delta(u^n),   u^{n+1} = u^n + delta,
// the same solution as A u^{n+1} = u^n in exact arithmetic. Solving for the
// small increment instead of the full state keeps the FP32 solve error
// proportional to |delta| rather than |u|. Dirichlet end rows and padding rows
// are identity rows with a zero increment.
//
// The row state lives in shared memory, laid out [j][thread] so a warp's
// accesses are conflict-free, and the elimination holds only its three
// coefficient arrays in registers. FP32 adds u + delta with Kahan compensation
// (the term lo per node, also in shared memory): BTCS steps are long, so an
// increment can be a sizeable part of u and must be compensated every step.
//
// Two barriers per step. Each thread publishes the reduced-system data of its
// chunk; warp 0 forms the reduced rows, solves them, and also computes the
// next step's value of every chunk's first and last node (the owner computes
// the same numbers from the same operands), so the neighbour values of the
// next step need no exchange of their own.
template <typename T, int NT, int C, bool EXACT, int BCT>
__device__ __forceinline__ void btcs_steps(int64_t nsteps, T r, T s, int n, BtcsShared<T, NT>& sm,
                                           T* hfirst, T* hlast, T* us, T* lo) {
  constexpr bool PER = BCT == BC_PERIODIC;
  constexpr int Q = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tl = EXACT ? NT - 1 : (n - 1) / C;  // chunk holding node n-1
  const int jstar = n - 1 - tid * C;              // local index of node n-1
  const int je = EXACT ? C - 1 : (jstar < C ? jstar : C - 1);  // chunk end row
  const T ds1 = T(1) + T(2) * s;
  auto uval = [&](int j, int t) -> T { return us[j * NT + t]; };
  // u^{n+1} of node j of chunk t from its increment (the owner's arithmetic)
  auto next_u = [&](int j, int t, T delta) -> T {
    T l0 = T(0);
    if constexpr (Kahan<T>::on) l0 = lo[j * NT + t];
    return comp_add(us[j * NT + t], delta, l0);
  };
  T ch[C], ah[C], dd[C];
  for (int64_t step = 0; step < nsteps; ++step) {
    T left = T(0), right = T(0);
    if (tid > 0) left = hlast[tid - 1];
    else if constexpr (PER) left = hlast[tl];
    if (tid < tl) right = hfirst[tid + 1];
    else if constexpr (PER) right = hfirst[0];
    // ---- assembly of rows and right-hand sides fused with the forward sweep
    T chp = T(0), ahp = T(-1), dhp = T(0);
    T ul = left, a = uval(0, tid);
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const T an = (j + 1 < C) ? uval(j + 1, tid) : right;
      T ur = an;
      if constexpr (!EXACT) {
        if (j == jstar) ur = right;
      }
      const T ra = r * a;
      T l = -s - tmax(ra, T(0));
      T c = tmin(ra, T(0)) - s;
      T d = ds1 + tabs(ra);
      // explicit increment (Eq. 21) from the same coefficients: -c (ur - a) + l (a - ul)
      T rhs = tfma(l, a - ul, -c * (ur - a));
      bool ident = false;
      if constexpr (BCT == BC_DIRICHLET) {
        if constexpr (EXACT)
          ident = (j == 0 && tid == 0) || (j == C - 1 && tid == NT - 1);
        else
          ident = (j == 0 && tid == 0) || j == jstar;
      }
      if constexpr (!EXACT) {
        if (j > jstar) ident = true;
      }
      if (ident) { l = T(0); c = T(0); d = T(1); rhs = T(0); }
      const T inv = recip(tfma(-l, chp, d));
      const T li = l * inv;
      chp = c * inv;
      ahp = -li * ahp;
      dhp = tfma(-li, dhp, rhs * inv);
      ch[j] = chp;
      ah[j] = ahp;
      dd[j] = dhp;
      ul = a;
      a = an;
    }
    T e_ch = T(0), e_ah = T(0), e_dh = T(0);
    if constexpr (EXACT) {
      e_ch = ch[C - 1]; e_ah = ah[C - 1]; e_dh = dd[C - 1];
    } else {
#pragma unroll
      for (int j = 0; j < C; ++j)
        if (j == je) { e_ch = ch[j]; e_ah = ah[j]; e_dh = dd[j]; }
    }
    // ---- backward sweep: (delta, alpha, gamma) into (dd, ah, ch)
    T cd = T(0), ca = T(0), cg = T(-1);
    if constexpr (EXACT) {
      dd[C - 1] = T(0); ah[C - 1] = T(0); ch[C - 1] = T(-1);
#pragma unroll
      for (int j = C - 2; j >= 0; --j) {
        const T cj = ch[j];
        cd = tfma(-cj, cd, dd[j]);
        ca = tfma(-cj, ca, ah[j]);
        cg = -cj * cg;
        dd[j] = cd; ah[j] = ca; ch[j] = cg;
      }
    } else {
#pragma unroll
      for (int j = C - 1; j >= 0; --j) {
        const T cj = ch[j];
        T nd = tfma(-cj, cd, dd[j]);
        T na = tfma(-cj, ca, ah[j]);
        T ng = -cj * cg;
        const bool past = j > je, at = j == je;
        if (past || at) { nd = T(0); na = T(0); ng = at ? T(-1) : T(0); }
        dd[j] = nd; ah[j] = na; ch[j] = ng;
        if (past || at) { cd = T(0); ca = T(0); cg = T(-1); }
        else { cd = nd; ca = na; cg = ng; }
      }
    }
    // ---- this chunk's first-row and end-row relations
    sm.rd[sk(tid)] = dd[0];
    sm.ra[sk(tid)] = ah[0];
    sm.rg[sk(tid)] = ch[0];
    {
      const int si = sk(tid);
      sm.A[si] = e_ah;
      sm.Cc[si] = e_ch;
      sm.D[si] = e_dh;
    }
    __syncthreads();
    if (warp == 0) {
      // reduced row of each of this lane's chunks: end row of chunk t with the
      // first-row relation of chunk t + 1 substituted (chunk 0 after the last)
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int t = lane * Q + q, i = sk(t);
        T A = T(0), B = T(1), Cc = T(0), D = T(0);
        if (t <= tl) {
          const int nx = (t == tl) ? 0 : t + 1;
          const T ech = sm.Cc[i];
          A = sm.A[i];
          B = T(1) - ech * sm.ra[sk(nx)];
          Cc = -ech * sm.rg[sk(nx)];
          D = tfma(-ech, sm.rd[sk(nx)], sm.D[i]);
        }
        sm.A[i] = A; sm.B[i] = B; sm.Cc[i] = Cc; sm.D[i] = D; sm.U[i] = T(0);
      }
      __syncwarp();
      reduced_solve<T, NT, PER>(sm, tl, lane);
      __syncwarp();
      // next step's first and last node of each chunk
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int t = lane * Q + q;
        if (t <= tl) {
          const T Xt = sm.X[sk(t)];
          T L = T(0);
          if (t > 0) L = sm.X[sk(t - 1)];
          else if constexpr (PER) L = sm.X[sk(tl)];
          const int jt = (t == tl) ? (n - 1) - t * C : C - 1;  // end row of chunk t
          const T d0 = jt == 0 ? Xt : tfma(-sm.rg[sk(t)], Xt, tfma(-sm.ra[sk(t)], L, sm.rd[sk(t)]));
          hfirst[t] = next_u(0, t, d0);
          hlast[t] = next_u(jt, t, Xt);
        }
      }
    }
    __syncthreads();
    // ---- back-substitution of the increment and the update of the state
    if (tid <= tl) {
      T L = T(0);
      if (tid > 0) L = sm.X[sk(tid - 1)];
      else if constexpr (PER) L = sm.X[sk(tl)];
      const T Xt = sm.X[sk(tid)];
#pragma unroll
      for (int j = 0; j < C; ++j) {
        if (EXACT || j <= je) {
          const T delta = (j == je) ? Xt : tfma(-ch[j], Xt, tfma(-ah[j], L, dd[j]));
          const int o = j * NT + tid;
          T l0 = T(0);
          if constexpr (Kahan<T>::on) l0 = lo[o];
          us[o] = comp_add(us[o], delta, l0);
          if constexpr (Kahan<T>::on) lo[o] = l0;
        }
      }
    }
  }
}

// FP32: at most 128 registers per thread, so 512 threads' worth of CTAs fit
// on an SM (four CTAs of the 128 x 32 shape hide each other's serial phase).
template <typename T, int NT, int C, bool EXACT>
__global__ void __launch_bounds__(NT, (sizeof(T) == 4 && NT <= 512) ? 512 / NT : 1)
    k_btcs_resident(T* __restrict__ u,
                                                      const RowDesc* __restrict__ rows, int count,
                                                      int* __restrict__ counter) {
  __shared__ BtcsShared<T, NT> sm;
  __shared__ T hfirst[NT], hlast[NT];
  __shared__ int s_item;
  extern __shared__ __align__(16) unsigned char dsm[];
  T* us = reinterpret_cast<T*>(dsm);  // C * NT values
  T* lo = us + C * NT;                // C * NT values (FP32)
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= count) return;
    const RowDesc rd = rows[item];
    T* row = u + rd.offset;
    const int base = tid * C;
    const int n = rd.n;
    const int tl = EXACT ? NT - 1 : (n - 1) / C;
    const int jt = (tid == tl) ? (n - 1) - base : C - 1;
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const T x = (EXACT || base + j < n) ? row[base + j] : T(0);
      us[j * NT + tid] = x;
      if constexpr (Kahan<T>::on) lo[j * NT + tid] = T(0);
      if (j == 0) hfirst[tid] = x;
      if (j == jt) hlast[tid] = x;
    }
    __syncthreads();
    const T r = T(rd.r), s = T(rd.s);
    if (rd.bc == BC_PERIODIC)
      btcs_steps<T, NT, C, EXACT, BC_PERIODIC>(rd.nsteps, r, s, n, sm, hfirst, hlast, us, lo);
    else
      btcs_steps<T, NT, C, EXACT, BC_DIRICHLET>(rd.nsteps, r, s, n, sm, hfirst, hlast, us, lo);
#pragma unroll
    for (int j = 0; j < C; ++j)
      if (EXACT || base + j < n) row[base + j] = us[j * NT + tid];
    __syncthreads();
  }
}

#define BTCS_DSM(T, NT, C) (sizeof(T) * size_t(NT) * size_t(C) * (Kahan<T>::on ? 2 : 1))
#define REG_BTCS(T, DT, NT, C)                                                                  \
  reg.push_back({K_BTCS_RESIDENT, DT, NT, C, 1,                                                 \
                 reinterpret_cast<const void*>(&k_btcs_resident<T, NT, C, true>),              \
                 BTCS_DSM(T, NT, C)});                                                          \
  reg.push_back({K_BTCS_RESIDENT, DT, NT, C, 0,                                                 \
                 reinterpret_cast<const void*>(&k_btcs_resident<T, NT, C, false>),             \
                 BTCS_DSM(T, NT, C)});

void register_btcs(std::vector<KernelEntry>& reg) {
  REG_BTCS(float, 0, 32, 1) REG_BTCS(float, 0, 32, 2) REG_BTCS(float, 0, 32, 4)
  REG_BTCS(float, 0, 32, 8) REG_BTCS(float, 0, 64, 8) REG_BTCS(float, 0, 128, 8)
  REG_BTCS(float, 0, 256, 8) REG_BTCS(float, 0, 128, 16) REG_BTCS(float, 0, 256, 16)
  REG_BTCS(float, 0, 512, 8) REG_BTCS(float, 0, 512, 16) REG_BTCS(float, 0, 1024, 8)
  REG_BTCS(float, 0, 64, 32) REG_BTCS(float, 0, 128, 32) REG_BTCS(float, 0, 256, 32)
  REG_BTCS(double, 1, 32, 1) REG_BTCS(double, 1, 32, 2) REG_BTCS(double, 1, 32, 4)
  REG_BTCS(double, 1, 32, 8) REG_BTCS(double, 1, 64, 8) REG_BTCS(double, 1, 128, 8)
  REG_BTCS(double, 1, 256, 8) REG_BTCS(double, 1, 512, 8) REG_BTCS(double, 1, 256, 16)
  REG_BTCS(double, 1, 128, 16)
}

}  // namespace burgers
