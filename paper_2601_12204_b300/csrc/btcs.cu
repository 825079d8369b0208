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
#include "common.cuh"
#include "kernels.h"

namespace burgers {

__device__ __forceinline__ int sk(int i) { return i + (i >> 5); }  // bank skew

template <typename T, int NT>
struct BtcsShared {
  static constexpr int SK = NT + NT / 32;
  T rd[NT], ra[NT], rg[NT];              // first-row relation per chunk; reused for z
  T A[SK], B[SK], Cc[SK], D[SK], U[SK];  // reduced rows (skewed)
  T X[NT];                               // chunk-end solution
};

// Solves the reduced system held in sm (rows 0..NT-1, rows beyond tl are
// decoupled identities) with warp 0; leaves the solution in sm.X.
template <typename T, int NT, bool CYC>
__device__ __forceinline__ void reduced_solve(BtcsShared<T, NT>& sm, int tl, int lane) {
  constexpr int Q = NT / 32;
  double fad = 0.0;  // A_0 / gamma of the Sherman-Morrison split, FP64
  if constexpr (CYC) {
    const T A0 = sm.A[sk(0)], B0 = sm.B[sk(0)], Ct = sm.Cc[sk(tl)], Bt = sm.B[sk(tl)];
    const T gam = -B0;
    fad = double(A0) / double(gam);
    __syncwarp();
    if (lane == 0) {
      sm.B[sk(0)] = B0 - gam;
      sm.A[sk(0)] = T(0);
      sm.U[sk(0)] = gam;
      sm.B[sk(tl)] = Bt - Ct * T(fad);
      sm.Cc[sk(tl)] = T(0);
      sm.U[sk(tl)] = Ct;
    }
    __syncwarp();
  }
  const int r0 = lane * Q;
  // forward sweep over this lane's Q reduced rows
  T chp = T(0), ahp = T(-1), dhp = T(0), uhp = T(0);
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int i = sk(r0 + q);
    const T a = sm.A[i], b = sm.B[i], c = sm.Cc[i], d = sm.D[i];
    const T inv = recip(tfma(-a, chp, b));
    const T ai = a * inv;
    chp = c * inv;
    ahp = -ai * ahp;
    dhp = tfma(-ai, dhp, d * inv);
    sm.Cc[i] = chp;
    sm.A[i] = ahp;
    sm.D[i] = dhp;
    if constexpr (CYC) {
      uhp = tfma(-ai, uhp, sm.U[i] * inv);
      sm.U[i] = uhp;
    }
  }
  const T e_ch = chp, e_ah = ahp, e_dh = dhp, e_uh = uhp;
  // backward sweep: rows before the lane's end row, relation to (L, X_end)
  T cd = T(0), ca = T(0), cg = T(-1), cu = T(0);
#pragma unroll
  for (int q = Q - 2; q >= 0; --q) {
    const int i = sk(r0 + q);
    const T ch = sm.Cc[i];
    cd = tfma(-ch, cd, sm.D[i]);
    ca = tfma(-ch, ca, sm.A[i]);
    cg = -ch * cg;
    sm.D[i] = cd;
    sm.A[i] = ca;
    sm.Cc[i] = cg;
    if constexpr (CYC) {
      cu = tfma(-ch, cu, sm.U[i]);
      sm.U[i] = cu;
    }
  }
  // next lane's first-row relation
  T nd = shfl_down(cd, 1), na = shfl_down(ca, 1), ng = shfl_down(cg, 1), nu = shfl_down(cu, 1);
  if (lane == 31) { nd = T(0); na = T(0); ng = T(0); nu = T(0); }
  T a32 = e_ah, b32 = T(1) - e_ch * na, c32 = -e_ch * ng;
  T d32 = tfma(-e_ch, nd, e_dh), u32 = tfma(-e_ch, nu, e_uh);
  {
    const T inv = recip(b32);
    a32 *= inv; c32 *= inv; d32 *= inv; u32 *= inv;
  }
  // parallel cyclic reduction over the 32 lanes (non-cyclic after the split)
#pragma unroll
  for (int k = 1; k < 32; k <<= 1) {
    T am = shfl_up(a32, k), cm = shfl_up(c32, k), dm = shfl_up(d32, k);
    T ap = shfl_down(a32, k), cp = shfl_down(c32, k), dp = shfl_down(d32, k);
    T um = T(0), up = T(0);
    if constexpr (CYC) { um = shfl_up(u32, k); up = shfl_down(u32, k); }
    if (lane < k) { am = T(0); cm = T(0); dm = T(0); um = T(0); }
    if (lane + k > 31) { ap = T(0); cp = T(0); dp = T(0); up = T(0); }
    const T inv = recip(T(1) - a32 * cm - c32 * ap);
    const T na2 = -a32 * am * inv, nc2 = -c32 * cp * inv;
    const T nd2 = (d32 - a32 * dm - c32 * dp) * inv;
    if constexpr (CYC) u32 = (u32 - a32 * um - c32 * up) * inv;
    a32 = na2; c32 = nc2; d32 = nd2;
  }
  const T Ye = d32, Ze = u32;
  T YL = shfl_up(Ye, 1), ZL = shfl_up(Ze, 1);
  if (lane == 0) { YL = T(0); ZL = T(0); }
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int i = sk(r0 + q);
    T y = Ye, z = Ze;
    if (q < Q - 1) {
      y = tfma(-sm.Cc[i], Ye, tfma(-sm.A[i], YL, sm.D[i]));
      if constexpr (CYC) z = tfma(-sm.Cc[i], Ze, tfma(-sm.A[i], ZL, sm.U[i]));
    }
    sm.X[r0 + q] = y;
    if constexpr (CYC) sm.rd[r0 + q] = z;
  }
  if constexpr (CYC) {
    __syncwarp();
    // x = y - (v.y)/(1 + v.z) z,  v = e_0 + (A_0/gamma) e_tl
    const double y0 = double(sm.X[0]), yt = double(sm.X[tl]);
    const double z0 = double(sm.rd[0]), zt = double(sm.rd[tl]);
    const double fac = (y0 + fad * yt) / (1.0 + z0 + fad * zt);
    __syncwarp();
#pragma unroll
    for (int q = 0; q < Q; ++q)
      sm.X[r0 + q] = T(double(sm.X[r0 + q]) - fac * double(sm.rd[r0 + q]));
  }
}

// Advances the C nodes held by this thread `nsteps` BTCS steps.
template <typename T, int NT, int C, bool EXACT, int BCT>
__device__ __forceinline__ void btcs_steps(T (&v)[C], int64_t nsteps, T r, T s, int n,
                                           BtcsShared<T, NT>& sm) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int base = tid * C;
  const int tl = EXACT ? NT - 1 : (n - 1) / C;  // chunk holding node n-1
  const int jstar = n - 1 - base;                // local index of node n-1
  const int je = EXACT ? C - 1 : (jstar < C ? jstar : C - 1);  // chunk end row (<0: none)
  const T ds1 = T(1) + T(2) * s;
  T ch[C], ah[C];
  for (int64_t step = 0; step < nsteps; ++step) {
    // ---- assembly fused with the forward sweep
    T chp = T(0), ahp = T(-1), dhp = T(0);
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const T a = v[j];
      const T ra = r * a;
      T l = -s - tmax(ra, T(0));
      T c = tmin(ra, T(0)) - s;
      T d = ds1 + tabs(ra);
      T rhs = a;
      bool ident = false;
      if constexpr (BCT == BC_DIRICHLET) {
        if constexpr (EXACT)
          ident = (j == 0 && tid == 0) || (j == C - 1 && tid == NT - 1);
        else
          ident = (j == 0 && tid == 0) || j == jstar;
      }
      if constexpr (!EXACT) {
        if (j > jstar) { ident = true; rhs = T(0); }
      }
      if (ident) { l = T(0); c = T(0); d = T(1); }
      const T inv = recip(tfma(-l, chp, d));
      const T li = l * inv;
      chp = c * inv;
      ahp = -li * ahp;
      dhp = tfma(-li, dhp, rhs * inv);
      ch[j] = chp;
      ah[j] = ahp;
      v[j] = dhp;
    }
    T e_ch = T(0), e_ah = T(0), e_dh = T(0);
    if constexpr (EXACT) {
      e_ch = ch[C - 1]; e_ah = ah[C - 1]; e_dh = v[C - 1];
    } else {
#pragma unroll
      for (int j = 0; j < C; ++j)
        if (j == je) { e_ch = ch[j]; e_ah = ah[j]; e_dh = v[j]; }
    }
    // ---- backward sweep: (delta, alpha, gamma) into (v, ah, ch)
    T cd = T(0), ca = T(0), cg = T(-1);
    if constexpr (EXACT) {
      v[C - 1] = T(0); ah[C - 1] = T(0); ch[C - 1] = T(-1);
#pragma unroll
      for (int j = C - 2; j >= 0; --j) {
        const T cj = ch[j];
        cd = tfma(-cj, cd, v[j]);
        ca = tfma(-cj, ca, ah[j]);
        cg = -cj * cg;
        v[j] = cd; ah[j] = ca; ch[j] = cg;
      }
    } else {
#pragma unroll
      for (int j = C - 1; j >= 0; --j) {
        const T cj = ch[j];
        T nd = tfma(-cj, cd, v[j]);
        T na = tfma(-cj, ca, ah[j]);
        T ng = -cj * cg;
        const bool past = j > je, at = j == je;
        if (past || at) { nd = T(0); na = T(0); ng = at ? T(-1) : T(0); }
        v[j] = nd; ah[j] = na; ch[j] = ng;
        if (past || at) { cd = T(0); ca = T(0); cg = T(-1); }
        else { cd = nd; ca = na; cg = ng; }
      }
    }
    // ---- reduced row of this chunk
    sm.rd[tid] = v[0];
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
    // ---- back-substitution
    if (tid <= tl) {
      T L = T(0);
      if (tid > 0) L = sm.X[tid - 1];
      else if constexpr (BCT == BC_PERIODIC) L = sm.X[tl];
      const T Xt = sm.X[tid];
#pragma unroll
      for (int j = 0; j < C; ++j) v[j] = tfma(-ch[j], Xt, tfma(-ah[j], L, v[j]));
    }
  }
}

template <typename T, int NT, int C, bool EXACT>
__global__ void __launch_bounds__(NT) k_btcs_resident(T* __restrict__ u,
                                                      const RowDesc* __restrict__ rows, int count,
                                                      int* __restrict__ counter) {
  __shared__ BtcsShared<T, NT> sm;
  __shared__ int s_item;
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
      btcs_steps<T, NT, C, EXACT, BC_PERIODIC>(v, rd.nsteps, r, s, rd.n, sm);
    else
      btcs_steps<T, NT, C, EXACT, BC_DIRICHLET>(v, rd.nsteps, r, s, rd.n, sm);
#pragma unroll
    for (int j = 0; j < C; ++j)
      if (EXACT || base + j < rd.n) row[base + j] = v[j];
    __syncthreads();
  }
}

#define REG_BTCS(T, DT, NT, C)                                                           \
  reg.push_back({K_BTCS_RESIDENT, DT, NT, C, 1,                                          \
                 reinterpret_cast<const void*>(&k_btcs_resident<T, NT, C, true>), 0});  \
  reg.push_back({K_BTCS_RESIDENT, DT, NT, C, 0,                                          \
                 reinterpret_cast<const void*>(&k_btcs_resident<T, NT, C, false>), 0});

void register_btcs(std::vector<KernelEntry>& reg) {
  REG_BTCS(float, 0, 32, 1) REG_BTCS(float, 0, 32, 2) REG_BTCS(float, 0, 32, 4)
  REG_BTCS(float, 0, 32, 8) REG_BTCS(float, 0, 64, 8) REG_BTCS(float, 0, 128, 8)
  REG_BTCS(float, 0, 256, 8) REG_BTCS(float, 0, 128, 16) REG_BTCS(float, 0, 256, 16)
  REG_BTCS(float, 0, 512, 8) REG_BTCS(float, 0, 512, 16) REG_BTCS(float, 0, 1024, 8)
  REG_BTCS(double, 1, 32, 1) REG_BTCS(double, 1, 32, 2) REG_BTCS(double, 1, 32, 4)
  REG_BTCS(double, 1, 32, 8) REG_BTCS(double, 1, 64, 8) REG_BTCS(double, 1, 128, 8)
  REG_BTCS(double, 1, 256, 8) REG_BTCS(double, 1, 512, 8) REG_BTCS(double, 1, 256, 16)
}

}  // namespace burgers
