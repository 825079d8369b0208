// btcs_x2.cuh -- the FP32 resident implicit-step kernel on packed f32x2
// arithmetic (lagged BTCS, Crank-Nicolson, Picard and Newton; the algebra of
// each variant is that of btcs_kernel.cuh), for rows of exactly NT*C nodes and for
// ragged rows of its capacity class (chunks of C or C - 1 nodes, below).
//
// Each thread's chunk of C nodes is two half-chunks, A = nodes [0, C/2) and
// B = [C/2, C), eliminated side by side: pair k holds node k of A and node k
// of B, so every step of both eliminations is one packed instruction for the
// two lanes (the reciprocals stay scalar). Splitting the chunk also halves the
// length of each elimination's dependent chain.
//
// The chunk then has two unknown end values, X_A (node C/2 - 1) and X_B (node
// C - 1). Substituting B's first-row relation into A's end row gives the row
//     bA X_A + aA X_B(t-1) + cA X_B(t) = dA,
// which the thread divides by bA and publishes (pa, pc, pd) with A's first-row
// relation; substituting the next thread's first-row relation into B's end
// row and eliminating X_A(t) and X_A(t+1) through their rows leaves one
// tridiagonal row per thread in X_B(t-1), X_B(t), X_B(t+1): the same NT-row
// reduced system (cyclic for periodic rows) as the scalar kernel, solved by
// warp 0 with the same reduced_solve. Back-substitution recovers X_A from its
// row and every node from its half's relation.
//
// Signs: the packed forms have no negated operands, so the sweeps carry
// -rhs, -dh and -delta (and -ch beside ch), chosen so that every rounding is
// that of the corresponding scalar operation (negation commutes with
// round-to-nearest).
#pragma once

#include "btcs_kernel.cuh"

namespace burgers {

template <int NT>
struct X2Shared {
  static constexpr int SK = NT + NT / 32;
  float pa[SK], pc[SK], pd[SK];  // thread's A row divided by bA
  float c0[4];                   // thread 0: eBa, eBc, pa, pc (periodic corner split)
};

template <int NT, int C, int VAR>
constexpr size_t btcs_x2_dsm() {
  return sizeof(float2) * size_t(NT) * size_t(C / 2) *
         (2 + ((VAR == VAR_PICARD || VAR == VAR_NEWTON) ? 1 : 0));
}

// Thread 0's reduced row coefficients A_0, B_0 from its published values and
// thread 1's (the same arithmetic wherever it is evaluated).
__device__ __forceinline__ void x2_row0(const float* c0, float ran1, float rgn1, float pa1,
                                        float& A0, float& B0) {
  const float bB = 1.f - c0[1] * ran1;
  const float cB = -c0[1] * rgn1;
  A0 = -c0[0] * c0[2];
  B0 = bB - c0[0] * c0[3] - cB * pa1;
}

template <int NT, int C, int BCT, int VAR, bool EXACT>
__device__ __forceinline__ void btcs_steps_x2(int64_t nsteps, int iters, float r, float s,
                                              BtcsShared<float, NT>& sm, X2Shared<NT>& xs,
                                              float* hfirst, float* hlast, float2* us, float2* lo,
                                              float2* es, int solver, int tl_, bool shrt,
                                              bool padwarp) {
  static_assert(C % 2 == 0 && C >= 2, "two half-chunks");
  constexpr int H = C / 2;
  constexpr bool ITER = VAR == VAR_PICARD || VAR == VAR_NEWTON;
  // Newton's Jacobian diagonal holds w_{i+1} - w_{i-1}, so its sweeps take
  // the neighbours' values directly (published by their owners in the
  // previous back-substitution, one more CTA barrier per iteration) instead
  // of deferring them to the reduced rows: no deferred terms (kappa = 0)
  constexpr bool DEFER = VAR != VAR_NEWTON;
  constexpr bool PER = BCT == BC_PERIODIC;
  const float kap = VAR == VAR_CN ? 2.f : (DEFER ? 1.f : 0.f);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // last chunk holding nodes (ragged rows: chunks past it hold none, and the
  // short chunks end one pair early in their second half)
  const int tl = EXACT ? NT - 1 : tl_;
  const bool dlast = !EXACT && BCT == BC_DIRICHLET && tid == tl;
  const float rm = VAR == VAR_CN ? 0.5f * r : r, smat = VAR == VAR_CN ? 0.5f * s : s;
  const float2 RM2 = make_float2(rm, rm), SM2 = make_float2(smat, smat);
  const float ds1 = 1.f + 2.f * smat;
  const float2 DS1 = make_float2(ds1, ds1);
  const float hr = 0.5f * rm;  // Newton: r/2
  const float2 HR2 = make_float2(hr, hr), NS2 = make_float2(-smat, -smat);
  const int nit = ITER ? iters : 1;
  auto W = [&](int k) -> float2 {
    if constexpr (ITER) return add2(us[k * NT + tid], es[k * NT + tid]);
    else return us[k * NT + tid];
  };
  float2 CH[H], AH[H], ND[H];  // forward: -ch, ah, -dh; backward: gamma, alpha, -delta
  for (int64_t step = 0; step < nsteps; ++step) {
  if constexpr (ITER) {
#pragma unroll
    for (int k = 0; k < H; ++k) es[k * NT + tid] = make_float2(0.f, 0.f);
  }
  for (int it = 0; it < nit; ++it) {
    const bool last = it + 1 == nit;
    // ---- forward sweep of both halves. A's first row stands in for its own
    // left neighbour (deferred, as in the scalar kernel); B's first row reads
    // node C/2 - 1; A's end row reads node C/2; B's end row stands in for its
    // own right neighbour (deferred). Warps without nodes (ragged rows) skip
    // it where that costs no registers (up to 16 nodes a thread; with 32 the
    // branch around the sweep spilled): nothing reads what they publish.
    float eBc = 0.f, eBa = 0.f, eBd = 0.f, pa = 0.f, pc = 0.f, pd0 = 0.f;
    if (EXACT || C > 16 || !padwarp) {
    // Newton: the current iterate's values left of the chunk and right of it
    float nleft = 0.f, nright = 0.f;
    if constexpr (!DEFER) {
      nleft = tid > 0 ? hlast[tid - 1] : (PER ? hlast[tl] : 0.f);
      nright = tid < tl ? hfirst[tid + 1] : (PER ? hfirst[0] : 0.f);
    }
    float2 a = W(0);
    float2 ul = make_float2(DEFER ? a.x : nleft, W(H - 1).x);
    float2 DL = sub2(a, ul);  // a - u_l
    float2 chp = make_float2(0.f, 0.f), ahp = make_float2(-1.f, -1.f), ndhp = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < H; ++k) {
      float2 an = (k + 1 < H) ? W(k + 1) : make_float2(W(0).y, DEFER ? a.y : nright);
      // a short chunk's second half ends at pair H - 2 and stands in for its
      // own right neighbour there (its pair H - 1 is padding)
      if constexpr (!EXACT) {
        if (k == H - 2 && shrt) an.y = DEFER ? a.y : nright;
      }
      const float2 ER = sub2(an, a);  // u_r - a
      float2 nl, c, nc, d, nrhs;      // -l, c, -c, d, -rhs
      if constexpr (VAR == VAR_NEWTON) {
        // J rows l = -(r/2) w - s, d = 1 + (r/2)(w_r - w_l) + 2s, c = (r/2) w - s;
        // -rhs = F = e + (r/2) w (w_r - w_l) - s (w_r - 2 w + w_l)
        const float2 ha = mul2(HR2, a);
        const float2 cdf = sub2(an, ul);
        nl = add2(ha, SM2);
        c = sub2(ha, SM2);
        nc = sub2(SM2, ha);
        d = fma2(HR2, cdf, DS1);
        nrhs = fma2(NS2, sub2(ER, DL), fma2(ha, cdf, es[k * NT + tid]));
      } else {
        const float2 ra = mul2(RM2, a);
        const float2 M = make_float2(fmaxf(ra.x, 0.f), fmaxf(ra.y, 0.f));
        const float2 m = make_float2(fminf(ra.x, 0.f), fminf(ra.y, 0.f));
        nl = add2(SM2, M);
        c = sub2(m, SM2);
        nc = sub2(SM2, m);
        d = add2(DS1, sub2(M, m));
        // -rhs = -(l (a - u_l) - c (u_r - a)) of the increment form
        nrhs = fma2(nl, DL, mul2(c, ER));
        if constexpr (VAR == VAR_CN) nrhs = mul2(make_float2(2.f, 2.f), nrhs);
        if constexpr (ITER) nrhs = add2(nrhs, es[k * NT + tid]);
      }
      if constexpr (BCT == BC_DIRICHLET) {  // the row's end nodes are identity rows
        if (k == 0 && tid == 0) { nl.x = 0.f; c.x = 0.f; nc.x = 0.f; d.x = 1.f; nrhs.x = 0.f; }
        // (ragged rows: the last node only zeroes its chunk's end relation, below)
        if (EXACT && k == H - 1 && tid == NT - 1) {
          nl.y = 0.f; c.y = 0.f; nc.y = 0.f; d.y = 1.f; nrhs.y = 0.f;
        }
      }
      const float2 den = fma2(nl, chp, d);
      const float2 inv = make_float2(recip(den.x), recip(den.y));
      const float2 nli = mul2(nl, inv);
      chp = mul2(c, inv);
      CH[k] = mul2(nc, inv);
      ahp = mul2(nli, ahp);
      ndhp = fma2(nli, ndhp, mul2(nrhs, inv));
      AH[k] = ahp;
      ND[k] = ndhp;
      DL = ER;
      ul = a;
      a = an;
    }
    // end rows of both halves: x_e = dh - ah L - ch x_next
    const float eAc = chp.x, eAa = ahp.x, eAd = -ndhp.x;
    eBc = chp.y; eBa = ahp.y; eBd = -ndhp.y;
    if constexpr (!EXACT) {
      if (shrt) { eBc = -CH[H - 2].y; eBa = AH[H - 2].y; eBd = -ND[H - 2].y; }
      if (dlast) { eBc = 0.f; eBa = 0.f; eBd = 0.f; }  // Dirichlet: an identity end row
    }
    // ---- backward sweep: x_j = delta_j - alpha_j L - gamma_j X_e
    {
      float2 ncd = make_float2(0.f, 0.f), ca = make_float2(0.f, 0.f), cg = make_float2(-1.f, -1.f);
      ND[H - 1] = ncd;
      AH[H - 1] = ca;
      CH[H - 1] = cg;
#pragma unroll
      for (int k = H - 2; k >= 0; --k) {
        const float2 ncj = CH[k];
        ncd = fma2(ncj, ncd, ND[k]);
        ca = fma2(ncj, ca, AH[k]);
        cg = mul2(ncj, cg);
        if constexpr (!EXACT) {
          if (k == H - 2 && shrt) { ncd.y = 0.f; ca.y = 0.f; cg.y = -1.f; }  // its end row
        }
        ND[k] = ncd;
        AH[k] = ca;
        CH[k] = cg;
      }
    }
    // ---- A's row, divided by bA, without the deferred term of its left
    // neighbour (pd0: every reader adds -kap pa (u_left - u_0) after the
    // first barrier, from the edge values the owners published); A's
    // first-row relation
    const float bA = 1.f - eAc * AH[0].y;
    const float cA = -eAc * CH[0].y;
    const float dA0 = tfma(-eAc, -ND[0].y, eAd);
    const float ib = 1.f / bA;
    pa = eAa * ib; pc = cA * ib; pd0 = dA0 * ib;
    sm.rd[sk(tid)] = -ND[0].x;
    sm.ra[sk(tid)] = AH[0].x;
    sm.rg[sk(tid)] = CH[0].x;
    xs.pa[sk(tid)] = pa;
    xs.pc[sk(tid)] = pc;
    xs.pd[sk(tid)] = pd0;
    if constexpr (PER) {
      if (tid == 0) { xs.c0[0] = eBa; xs.c0[1] = eBc; xs.c0[2] = pa; xs.c0[3] = pc; }
    }
    }  // sweep
    __syncthreads();
    // u_left - u_0 of this chunk and A's row with it
    const float lt = tid > 0 ? hlast[tid - 1] - hfirst[tid] : (PER ? hlast[tl] - hfirst[0] : 0.f);
    const float pd = tfma(-kap * pa, lt, pd0);
    // ---- the reduced row in X_B: B's end row with the next thread's
    // first-row relation substituted, X_A(t) and X_A(t+1) eliminated
    float fa = 0.f;
    {
      const int t = tid, i = sk(t);
      const int nx = (t == tl) ? 0 : t + 1;
      // (ragged rows: threads past tl hold no chunk and give identity rows)
      const bool has_next = (PER || t < tl) && (EXACT || t <= tl);
      float A = -eBa * pa, B = 1.f, Cc = 0.f, D = 0.f, U = 0.f;
      const float Dt0 = eBd;
      if (has_next) {
        const float e = hlast[t], fn = hfirst[nx];
        const float rt = fn - e;
        const float ran = sm.ra[sk(nx)], rgn = sm.rg[sk(nx)];
        const float rdn = tfma(-kap * ran, e - fn, sm.rd[sk(nx)]);
        const float Dt = tfma(-kap * eBc, rt, Dt0);
        const float bB = 1.f - eBc * ran;
        const float cB = -eBc * rgn;
        const float dB = tfma(-eBc, rdn, Dt);
        const float pan = xs.pa[sk(nx)], pcn = xs.pc[sk(nx)];
        const float pdn = tfma(-kap * pan, e - fn, xs.pd[sk(nx)]);  // its u_left - u_0 is e - fn
        B = bB - eBa * pc - cB * pan;
        Cc = -cB * pcn;
        D = dB - eBa * pd - cB * pdn;
      } else {  // Dirichlet: the row's last node is an identity row
        B = 1.f - eBa * pc;
        D = Dt0 - eBa * pd;
      }
      if constexpr (PER) {
        float A0, B0;
        x2_row0(xs.c0, sm.ra[sk(1)], sm.rg[sk(1)], xs.pa[sk(1)], A0, B0);
        const float gam = -B0;
        fa = A0 * recip(gam);
        if (t == 0) { B = B0 - gam; A = 0.f; U = gam; }
        if (t == tl) { B = B - Cc * fa; U = Cc; Cc = 0.f; }
      }
      if constexpr (!EXACT) {
        if (t > tl) { A = 0.f; B = 1.f; Cc = 0.f; D = 0.f; U = 0.f; }
      }
      sm.A[i] = A; sm.B[i] = B; sm.Cc[i] = Cc; sm.D[i] = D; sm.U[i] = U;
    }
    __syncthreads();
    if (warp == solver) reduced_solve<float, NT, PER, true>(sm, tl, lane, fa);
    __syncthreads();
    // ---- X_A from its row; every node from its half's relation; the update
    if (EXACT || tid <= tl) {
      float XBm = 0.f;
      if (tid > 0) XBm = sm.X[sk(tid - 1)];
      else if constexpr (PER) XBm = sm.X[sk(tl)];
      const float XB = sm.X[sk(tid)];
      const float XA = pd - pa * XBm - pc * XB;
      const float2 Lp = make_float2(tfma(kap, lt, XBm), XA);
      const float2 Xp = make_float2(XA, XB);
#pragma unroll
      for (int k = 0; k < H; ++k) {
        float2 ndelta = fma2(CH[k], Xp, fma2(AH[k], Lp, ND[k]));
        if constexpr (!EXACT) {
          if (k == H - 1 && shrt) ndelta.y = 0.f;  // the padding pair keeps its value
        }
        const int o = k * NT + tid;
        float2 nv;
        if constexpr (ITER) {
          const float2 inc = sub2(es[o], ndelta);
          if (!last) {
            es[o] = inc;
            nv = add2(us[o], inc);  // the next iterate's value (edges below)
          } else {
            const float2 u = us[o], l0 = lo[o];
            const float2 y = sub2(inc, l0);
            nv = add2(u, y);
            lo[o] = sub2(sub2(nv, u), y);
            us[o] = nv;
          }
        } else {
          const float2 u = us[o], l0 = lo[o];
          const float2 ny = add2(ndelta, l0);
          nv = sub2(u, ny);
          lo[o] = add2(sub2(nv, u), ny);
          us[o] = nv;
        }
        if (k == 0) hfirst[tid] = nv.x;
        if (k == H - 1 && (EXACT || !shrt)) hlast[tid] = nv.y;
        if constexpr (!EXACT) {
          if (k == H - 2 && shrt) hlast[tid] = nv.y;
        }
      }
    }
    // Newton: the next sweep reads its neighbours' new edge values
    if constexpr (!DEFER) __syncthreads();
  }  // iterations
  }  // steps
}

// FP32 rows of NT*C nodes (EXACT), or ragged rows of n < NT*C nodes whose
// capacity class has this shape (n > NT*C/2). Persistent CTAs take rows from
// an atomic counter; the row state lives in shared memory as node pairs
// (k, k + C/2) laid out [k][thread].
//
// Ragged rows: tk = ceil(n / C) threads hold chunks, the last bk = tk C - n of
// them C - 1 nodes (second half one node short); since n > NT C / 2, tk >
// NT / 2 >= C > bk, so every such length has this split. A short chunk's end
// sits at a position known at compile time (pair C/2 - 2 of its second half),
// so all warps run the same sweep with a few selects there; warps wholly past
// tk skip the sweep and threads past it give identity reduced rows.
template <int NT, int C, int VAR, bool EXACT = true>
__global__ void __launch_bounds__(NT, NT <= 512 ? 512 / NT : 1)
    k_btcs_resident_x2(float* __restrict__ u, const RowDesc* __restrict__ rows, int count,
                       int* __restrict__ counter) {
  constexpr int H = C / 2;
  static_assert(EXACT || C >= 4, "a short chunk keeps a node in its second half");
  __shared__ BtcsShared<float, NT> sm;
  __shared__ X2Shared<NT> xs;
  __shared__ float hfirst[NT], hlast[NT];
  __shared__ int s_item, s_solver;
  extern __shared__ __align__(16) unsigned char dsm[];
  float2* us = reinterpret_cast<float2*>(dsm);  // H * NT pairs
  float2* lo = us + H * NT;                      // H * NT pairs
  float2* es = us + 2 * H * NT;                  // H * NT pairs (Picard)
  const int tid = threadIdx.x;
  // The last warp solves the reduced systems: warp 0 also carries the row's
  // first node (its Dirichlet identity row, the periodic corner terms), and
  // on a B300 the last warp as solver ran 4-7% faster over the exact shapes
  // of 2048 to 8192 nodes. (Co-resident CTAs already have their warps 0 on different
  // schedulers: the hardware rotates each CTA's warps across them.)
  constexpr int NW = NT / 32;
  if (tid == 0) s_solver = NW - 1;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= count) return;
    const int solver = s_solver;
    const RowDesc rd = rows[item];
    const int n = EXACT ? NT * C : rd.n;
    const int tk = EXACT ? NT : (n + C - 1) / C;  // chunks holding nodes
    const int bk = tk * C - n;                     // short chunks (the last ones)
    const bool active = tid < tk;
    const bool shrt = !EXACT && active && tid >= tk - bk;
    const int cstart = tid * C - (shrt ? tid - (tk - bk) : 0);
    const int clen = active ? (shrt ? C - 1 : C) : 0;
    const bool padwarp = !EXACT && __all_sync(FULL_MASK, !active);
    float* row = u + rd.offset + cstart;
#pragma unroll
    for (int k = 0; k < H; ++k) {
      float2 x;
      if constexpr (EXACT) {
        x = make_float2(row[k], row[k + H]);
      } else {
        x = make_float2(k < clen ? row[k] : 0.f, k + H < clen ? row[k + H] : 0.f);
      }
      us[k * NT + tid] = x;
      lo[k * NT + tid] = make_float2(0.f, 0.f);
      if (k == 0) hfirst[tid] = x.x;
      if (k == H - 1 && !shrt) hlast[tid] = x.y;
      if (!EXACT && k == H - 2 && shrt) hlast[tid] = x.y;
    }
    __syncthreads();
    const float r = rd.rf, s = rd.sf;
    if (rd.bc == BC_PERIODIC)
      btcs_steps_x2<NT, C, BC_PERIODIC, VAR, EXACT>(rd.nsteps, rd.iters, r, s, sm, xs, hfirst,
                                                    hlast, us, lo, es, solver, tk - 1, shrt,
                                                    padwarp);
    else
      btcs_steps_x2<NT, C, BC_DIRICHLET, VAR, EXACT>(rd.nsteps, rd.iters, r, s, sm, xs, hfirst,
                                                     hlast, us, lo, es, solver, tk - 1, shrt,
                                                     padwarp);
#pragma unroll
    for (int k = 0; k < H; ++k) {
      const float2 x = us[k * NT + tid];
      if (EXACT || k < clen) row[k] = x.x;
      if (EXACT || k + H < clen) row[k + H] = x.y;
    }
    __syncthreads();
  }
}

// Registry entry of the ragged FP32 rows of a shape: the packed kernel when
// its chunks have at least two node pairs, else the scalar one.
template <int NT, int C, int VAR>
inline KernelEntry ragged_fp32_entry(int kind) {
  if constexpr (C >= 4)
    return KernelEntry{kind, 0, NT, C, 0,
                       reinterpret_cast<const void*>(&k_btcs_resident_x2<NT, C, VAR, false>),
                       btcs_x2_dsm<NT, C, VAR>()};
  else
    return KernelEntry{kind, 0, NT, C, 0,
                       reinterpret_cast<const void*>(&k_btcs_resident<float, NT, C, false, VAR>),
                       btcs_dsm<float, NT, C, VAR>()};
}

}  // namespace burgers
