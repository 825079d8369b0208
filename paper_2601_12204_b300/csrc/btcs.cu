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

// Advances the C nodes held by this thread `nsteps` BTCS steps.
//
// Increment form: with a = u^n, A(u^n) u^n = u^n - Delta(u^n) where Delta is the
// explicit forward-Euler increment of the same r, s (Eq. 21), so the step is
//     A(u^n) delta = Delta(u^n),   u^{n+1} = u^n + delta,
// the same solution as A u^{n+1} = u^n in exact arithmetic. Solving for the
// small increment instead of the full state keeps the FP32 solve error
// proportional to |delta| rather than |u|, and the FP32 addition is Kahan-
// compensated like the explicit kernel. Dirichlet end rows and padding rows
// are identity rows with a zero increment.
// u^n and (FP32) the Kahan terms wait in shared memory, laid out [j][thread]
// so a warp's accesses are conflict-free, while the elimination holds only its
// three coefficient arrays in registers.
template <typename T, int NT, int C, bool EXACT, int BCT>
__device__ __forceinline__ void btcs_steps(T (&v)[C], int64_t nsteps, T r, T s, int n,
                                           BtcsShared<T, NT>& sm, T* sh_last, T* sh_first,
                                           T* sh_wrap, T* un, T* lo) {
  constexpr int NW = NT / 32;
  constexpr bool WRAPX = (!EXACT && BCT == BC_PERIODIC);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int base = tid * C;
  const int tl = EXACT ? NT - 1 : (n - 1) / C;  // chunk holding node n-1
  const int jstar = n - 1 - base;                // local index of node n-1
  const int je = EXACT ? C - 1 : (jstar < C ? jstar : C - 1);  // chunk end row (<0: none)
  const T ds1 = T(1) + T(2) * s;
  T ch[C], ah[C], dd[C];
  if constexpr (Kahan<T>::on) {
#pragma unroll
    for (int j = 0; j < C; ++j) lo[j * NT + tid] = T(0);
  }
  for (int64_t step = 0; step < nsteps; ++step) {
    // ---- neighbour values of u^n across threads (as in the explicit kernel)
    const int p = int(step & 1);
    const T first = v[0], last = v[C - 1];
    T left = shfl(last, (lane + 31) & 31);
    T right = shfl(first, (lane + 1) & 31);
    if constexpr (NW > 1) {
      if (lane == 31) sh_last[p * NW + warp] = last;
      if (lane == 0) sh_first[p * NW + warp] = first;
    }
    if constexpr (WRAPX) {
      if (jstar >= 0 && jstar < C) {
        T sel = v[0];
#pragma unroll
        for (int j = 1; j < C; ++j)
          if (j == jstar) sel = v[j];
        sh_wrap[p * 2 + 0] = sel;
      }
      if (tid == 0) sh_wrap[p * 2 + 1] = first;
    }
    if constexpr (NW > 1 || WRAPX) __syncthreads();
    if constexpr (NW > 1) {
      if (lane == 0) left = sh_last[p * NW + (warp + NW - 1) % NW];
      if (lane == 31) right = sh_first[p * NW + (warp + 1) % NW];
    }
    T wrapL = T(0), wrapR = T(0);
    if constexpr (WRAPX) {
      wrapL = sh_wrap[p * 2 + 0];
      wrapR = sh_wrap[p * 2 + 1];
    }
    // ---- assembly of rows and right-hand sides fused with the forward sweep
    T chp = T(0), ahp = T(-1), dhp = T(0);
    T prev = left;
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const T a = v[j];
      un[j * NT + tid] = a;
      T ul = prev;
      T ur = (j + 1 < C) ? v[j + 1] : right;
      if constexpr (WRAPX) {
        if (j == 0 && tid == 0) ul = wrapL;
        if (j == jstar) ur = wrapR;
      }
      prev = a;
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
    // ---- reduced row of this chunk
    sm.rd[tid] = dd[0];
    sm.ra[tid] = ah[0];
    sm.rg[tid] = ch[0];
    __syncthreads();
    T A = T(0), B = T(1), Cc = T(0), D = T(0);
    if (tid <= tl) {
      const int nx = (tid == tl) ? 0 : tid + 1;
      const T dn = sm.rd[nx], an = sm.ra[nx], gn = sm.rg[nx];
      A = e_ah;
      B = T(1) - e_ch * an;
      Cc = -e_ch * gn;
      D = tfma(-e_ch, dn, e_dh);
    }
    const int si = sk(tid);
    sm.A[si] = A; sm.B[si] = B; sm.Cc[si] = Cc; sm.D[si] = D; sm.U[si] = T(0);
    __syncthreads();
    if (warp == 0) reduced_solve<T, NT, BCT == BC_PERIODIC>(sm, tl, lane);
    __syncthreads();
    // ---- back-substitution of the increment and the compensated update
    if (tid <= tl) {
      T L = T(0);
      if (tid > 0) L = sm.X[tid - 1];
      else if constexpr (BCT == BC_PERIODIC) L = sm.X[tl];
      const T Xt = sm.X[tid];
#pragma unroll
      for (int j = 0; j < C; ++j) {
        const T delta = tfma(-ch[j], Xt, tfma(-ah[j], L, dd[j]));
        T l0 = T(0);
        if constexpr (Kahan<T>::on) l0 = lo[j * NT + tid];
        v[j] = comp_add(un[j * NT + tid], delta, l0);
        if constexpr (Kahan<T>::on) lo[j * NT + tid] = l0;
      }
    } else {
#pragma unroll
      for (int j = 0; j < C; ++j) v[j] = un[j * NT + tid];
    }
  }
}

template <typename T, int NT, int C, bool EXACT>
__global__ void __launch_bounds__(NT) k_btcs_resident(T* __restrict__ u,
                                                      const RowDesc* __restrict__ rows, int count,
                                                      int* __restrict__ counter) {
  constexpr int NW = NT / 32;
  __shared__ BtcsShared<T, NT> sm;
  __shared__ T sh_last[2 * NW], sh_first[2 * NW], sh_wrap[4];
  __shared__ int s_item;
  extern __shared__ __align__(16) unsigned char dsm[];
  T* un = reinterpret_cast<T*>(dsm);  // C * NT values
  T* lo = un + C * NT;                // C * NT values (FP32)
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= count) return;
    const RowDesc rd = rows[item];
    T* row = u + rd.offset;
    const int base = threadIdx.x * C;
    T v[C];
#pragma unroll
    for (int j = 0; j < C; ++j) v[j] = (EXACT || base + j < rd.n) ? row[base + j] : T(0);
    const T r = T(rd.r), s = T(rd.s);
    if (rd.bc == BC_PERIODIC)
      btcs_steps<T, NT, C, EXACT, BC_PERIODIC>(v, rd.nsteps, r, s, rd.n, sm, sh_last, sh_first,
                                               sh_wrap, un, lo);
    else
      btcs_steps<T, NT, C, EXACT, BC_DIRICHLET>(v, rd.nsteps, r, s, rd.n, sm, sh_last,
                                                sh_first, sh_wrap, un, lo);
#pragma unroll
    for (int j = 0; j < C; ++j)
      if (EXACT || base + j < rd.n) row[base + j] = v[j];
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
