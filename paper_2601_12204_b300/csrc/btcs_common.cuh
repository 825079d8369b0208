// btcs_common.cuh -- pieces of the partitioned tridiagonal elimination shared
// by the resident BTCS kernel and the multi-level solver: the shared-memory
// layout of a CTA's reduced system and its one-warp solver (Sherman-Morrison
// split of the cyclic corners with an extended-precision correction
// denominator, per-lane elimination, parallel cyclic reduction over warp
// shuffles).
#pragma once

#include "common.cuh"

namespace burgers {

__device__ __forceinline__ int sk(int i) { return i + (i >> 5); }  // bank skew

template <typename T, int NT>
struct BtcsShared {
  static constexpr int SK = NT + NT / 32;
  // indexed through sk(): lane l of warp 0 handles rows lQ..lQ+Q-1, and the
  // skew keeps those strided accesses free of bank conflicts
  T rd[SK], ra[SK], rg[SK];              // first-row relation per chunk
  T A[SK], B[SK], Cc[SK], D[SK], U[SK];  // reduced rows
  T X[SK];                               // chunk-end solution
  T Z[SK];                               // cyclic case: solution for the correction vector
};

// Error-free sum (Knuth's TwoSum): a + b = s + e exactly. The intrinsics
// keep the compiler from fusing or reassociating the operations.
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}

// Sherman-Morrison factor (v.y)/(1 + v.z) for v = e_0 + fa e_tl. The
// denominator can sit near cancellation (it falls toward zero as the
// diffusion number s = nu dt / dx^2 grows: about 1e-3 at s = 1e4 and 1e-5 at
// s = 1e6 on a 64-node row), so it is formed in extended precision: FP64 for an FP64 solve; for FP32 an
// unevaluated pair hi + lo of floats from error-free transformations (the
// product by FMA, fa ztl = p + pe exactly, then two TwoSums and the sum of
// the three error terms), which keeps about 48 bits where an FP64 evaluation
// keeps 53 -- on B300 the FP64 pipe runs at a small fraction of the FP32 rate
// with a long latency, and this factor sits on the serial path of every
// solve. The FP32 numerator is one FMA (a single rounding of the exact dot
// product), and the quotient by hi + lo is a reciprocal estimate with one
// residual correction (within about one ulp).
template <typename T>
__device__ __forceinline__ T sm_factor(T fa, T y0, T ytl, T z0, T ztl) {
  if constexpr (sizeof(T) == 4) {
    const float num = __fmaf_rn(fa, ytl, y0);
    const float p = __fmul_rn(fa, ztl);
    const float pe = __fmaf_rn(fa, ztl, -p);
    float e1, e2;
    const float s1 = two_sum(z0, p, e1);
    const float hi = two_sum(1.0f, s1, e2);
    const float lo = __fadd_rn(__fadd_rn(pe, e1), e2);
    const float r = recip(hi);
    const float q0 = __fmul_rn(num, r);
    const float res = __fmaf_rn(-q0, lo, __fmaf_rn(-q0, hi, num));
    return __fmaf_rn(res, r, q0);
  } else {
    const double vy = fma(fa, ytl, y0);
    const double den = 1.0 + fma(fa, ztl, z0);
    return vy / den;
  }
}

// Solves the reduced system held in sm (rows 0..NT-1, rows beyond tl are
// decoupled identities) with warp 0; leaves the solution in sm.X.
// PRESPLIT: the caller has already applied the split below to rows 0 and tl
// (and set U) and passes the ratio in fa_pre.
template <typename T, int NT, bool CYC, bool PRESPLIT = false>
__device__ __forceinline__ void reduced_solve(BtcsShared<T, NT>& sm, int tl, int lane,
                                              T fa_pre = T(0)) {
  constexpr int Q = NT / 32;
  // Sherman-Morrison split: gamma = -B_0, v = e_0 + (A_0/gamma) e_tl. The ratio
  // is rounded once to T and used both in the modified diagonal and in v, so
  // T~ + u v^T reproduces the cyclic matrix up to the rounding of that ratio.
  T fa = T(0);
  if constexpr (CYC && PRESPLIT) {
    fa = fa_pre;
  } else if constexpr (CYC) {
    const T A0 = sm.A[sk(0)], B0 = sm.B[sk(0)], Ct = sm.Cc[sk(tl)], Bt = sm.B[sk(tl)];
    const T gam = -B0;
    fa = A0 * recip(gam);
    __syncwarp();
    if (lane == 0) {
      sm.B[sk(0)] = B0 - gam;
      sm.A[sk(0)] = T(0);
      sm.U[sk(0)] = gam;
      sm.B[sk(tl)] = Bt - Ct * fa;
      sm.Cc[sk(tl)] = T(0);
      sm.U[sk(tl)] = Ct;
    }
    __syncwarp();
  }
  const int r0 = lane * Q;
  // FP32 with up to 4 rows a lane keeps the sweeps' results in registers (rc,
  // ra, rd, ru); otherwise they go back to shared memory (in FP64 the extra
  // registers would cost resident CTAs)
  constexpr bool REGQ = Q <= 4 && sizeof(T) == 4;
  constexpr int QR = REGQ ? Q : 1;
  T rc[QR], ra[QR], rd[QR], ru[QR];
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
    if constexpr (CYC) uhp = tfma(-ai, uhp, sm.U[i] * inv);
    if constexpr (REGQ) {
      rc[q] = chp; ra[q] = ahp; rd[q] = dhp; ru[q] = uhp;
    } else {
      sm.Cc[i] = chp;
      sm.A[i] = ahp;
      sm.D[i] = dhp;
      if constexpr (CYC) sm.U[i] = uhp;
    }
  }
  const T e_ch = chp, e_ah = ahp, e_dh = dhp, e_uh = uhp;
  // backward sweep: rows before the lane's end row, relation to (L, X_end)
  T cd = T(0), ca = T(0), cg = T(-1), cu = T(0);
#pragma unroll
  for (int q = Q - 2; q >= 0; --q) {
    const int i = sk(r0 + q);
    if constexpr (REGQ) {
      const T ch = rc[q];
      cd = tfma(-ch, cd, rd[q]);
      ca = tfma(-ch, ca, ra[q]);
      cg = -ch * cg;
      if constexpr (CYC) cu = tfma(-ch, cu, ru[q]);
      rd[q] = cd; ra[q] = ca; rc[q] = cg; ru[q] = cu;
    } else {
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
  // up to 8 rows a lane keep y and z in registers through the correction;
  // more go through shared memory
  constexpr bool YREG = Q <= 8;
  T y[YREG ? Q : 1], z[YREG ? Q : 1];
  T ysel = T(0), zsel = T(0);  // row tl's values, on the lane that holds it
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int i = sk(r0 + q);
    T yq = Ye, zq = Ze;
    if (q < Q - 1) {
      if constexpr (REGQ) {
        yq = tfma(-rc[q], Ye, tfma(-ra[q], YL, rd[q]));
        if constexpr (CYC) zq = tfma(-rc[q], Ze, tfma(-ra[q], ZL, ru[q]));
      } else {
        yq = tfma(-sm.Cc[i], Ye, tfma(-sm.A[i], YL, sm.D[i]));
        if constexpr (CYC) zq = tfma(-sm.Cc[i], Ze, tfma(-sm.A[i], ZL, sm.U[i]));
      }
    }
    if constexpr (CYC) {
      if (r0 + q == tl) { ysel = yq; zsel = zq; }
    }
    if constexpr (YREG) {
      y[q] = yq;
      z[q] = zq;
    } else {
      sm.X[i] = yq;
      if constexpr (CYC) sm.Z[i] = zq;
    }
  }
  if constexpr (CYC) {
    // x = y - (v.y)/(1 + v.z) z with v.y = y_0 + fa y_tl, v.z likewise: the
    // corner values come from lane 0 (row 0) and the lane holding row tl.
    // Every lane evaluates the factor from the same four values (one shuffle
    // round, no broadcast of the result on the serial path).
    const T ytl = shfl(ysel, tl / Q), ztl = shfl(zsel, tl / Q);
    const T y0 = shfl(YREG ? y[0] : sm.X[sk(0)], 0), z0 = shfl(YREG ? z[0] : sm.Z[sk(0)], 0);
    const T fac = sm_factor(fa, y0, ytl, z0, ztl);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int i = sk(r0 + q);
      if constexpr (YREG) sm.X[i] = tfma(-fac, z[q], y[q]);
      else sm.X[i] = tfma(-fac, sm.Z[i], sm.X[i]);
    }
  } else if constexpr (YREG) {
#pragma unroll
    for (int q = 0; q < Q; ++q) sm.X[sk(r0 + q)] = y[q];
  }
}

// Forward sweep over the C rows of one chunk; rows j > je are inert padding.
// row(j, l, d, c, rhs) supplies row j. Leaves ch, ah, v = dh per row and the
// forward outputs of the end row je in e_ch, e_ah, e_dh (zero if je < 0).
template <typename T, int C, typename RowFn>
__device__ __forceinline__ void chunk_forward(T (&v)[C], T (&ah)[C], T (&ch)[C], int je, RowFn&& row,
                                              T& e_ch, T& e_ah, T& e_dh) {
  T chp = T(0), ahp = T(-1), dhp = T(0);
  e_ch = T(0); e_ah = T(0); e_dh = T(0);
#pragma unroll
  for (int j = 0; j < C; ++j) {
    T l, d, c, rhs;
    row(j, l, d, c, rhs);
    if (j > je) { l = T(0); c = T(0); d = T(1); rhs = T(0); }
    const T inv = recip(tfma(-l, chp, d));
    const T li = l * inv;
    chp = c * inv;
    ahp = -li * ahp;
    dhp = tfma(-li, dhp, rhs * inv);
    ch[j] = chp;
    ah[j] = ahp;
    v[j] = dhp;
    if (j == je) { e_ch = chp; e_ah = ahp; e_dh = dhp; }
  }
}

// Backward sweep: rows before the end row je become x_j = v_j - ah_j L - ch_j X
// (delta, alpha, gamma); the end row is x = X; padding rows become 0.
template <typename T, int C>
__device__ __forceinline__ void chunk_backward(T (&v)[C], T (&ah)[C], T (&ch)[C], int je) {
  T cd = T(0), ca = T(0), cg = T(-1);
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

}  // namespace burgers
