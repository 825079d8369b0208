// btcs_kernel.cuh -- the resident implicit-step kernel (lagged BTCS and the
// variants that solve the same tridiagonal shape), instantiated by btcs.cu,
// btcs_cn.cu, btcs_picard.cu and btcs_newton.cu.
#pragma once

#include <type_traits>

#include "btcs_common.cuh"
#include "common.cuh"
#include "kernels.h"

namespace burgers {

enum : int { VAR_BTCS = 0, VAR_CN = 1, VAR_PICARD = 2, VAR_NEWTON = 3 };

// Dynamic shared memory of k_btcs_resident: the state (and FP32 Kahan term)
// per node, plus e = w - u^n for the iterating variants.
template <typename T, int NT, int C, int VAR>
constexpr size_t btcs_dsm() {
  return sizeof(T) * size_t(NT) * size_t(C) *
         ((Kahan<T>::on ? 2 : 1) + ((VAR == VAR_PICARD || VAR == VAR_NEWTON) ? 1 : 0));
}


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
// Three CTA barriers per solve: after each thread publishes its chunk's
// first-row relation, after each thread forms its chunk's reduced row, and
// after the last warp has solved the reduced system.
//
// Neighbour values. A chunk's rows need the value left of its first node and
// right of its end node. In BTCS, CN and Picard the row coefficients depend
// on the node's own value only, so those two values enter the right-hand side
// alone, linearly, through the differences u_left - u_0 and u_right - u_end.
// The sweeps run with each edge node standing in for its own neighbour (both
// differences zero); row 0 then reads
//     l (x_{-1} + kap (u_left - u_0)) + d x_0 + c x_1 = rhs'
// (kap = 2 for CN, whose matrix has half the step's coefficients; 1
// otherwise), and likewise at the end row, so the chunk relations hold with L
// replaced by L + kap (u_left - u_0) and warp 0 adds the neighbour terms when
// it forms the reduced rows. The difference is the operand the right-hand side
// itself holds, so the increment keeps its precision. The edge values of a
// solve are those the owners publish (hfirst, hlast) during the previous
// back-substitution, bitwise the values their sweeps read, and the first
// barrier orders them before every read. Newton's Jacobian diagonal holds
// w_{i+1} - w_{i-1}, so there the sweeps take the neighbours directly and warp
// 0 computes every chunk's next edge values (the owner computes the same
// numbers from the same operands) after the reduced solve.
//
// VAR selects the implicit scheme; every variant solves tridiagonal systems
// of this shape in increment form:
//   VAR_BTCS    one lagged solve (above).
//   VAR_CN      Crank-Nicolson, convecting velocity lagged at u^n:
//               (I - dt/2 L) delta = dt L u^n, i.e. the BTCS rows with r/2,
//               s/2 and the full forward-Euler increment as right-hand side.
//   VAR_PICARD  `iters` Picard iterations A(w) w' = u^n: with w = u^n + e,
//               A(w) delta = Delta(w) - e, e += delta (coefficients from w).
//   VAR_NEWTON  `iters` Newton-Raphson iterations on the residual F of Eq. 11
//               (central convection, Eq. 10-14): J(w) delta = -F(w) with
//               J rows l = -r/2 w_i - s, d = 1 + r/2 (w_{i+1} - w_{i-1}) + 2s,
//               c = r/2 w_i - s, and -F_i = -e_i - r/2 w_i (w_{i+1} - w_{i-1})
//               + s (w_{i+1} - 2 w_i + w_{i-1}).
// The iterating variants keep e = w - u^n per node in shared memory (es) and
// add it to u^n, compensated, after the last iteration. The Newton Jacobian is
// not an M-matrix in general (central convection): |l| + |c| = max(2s, r|w_i|)
// and d >= 1 + 2s - r max|w|, so it is strictly diagonally dominant while
// r max|w| < 1/2.
template <typename T, int NT, int C, bool EXACT, int BCT, int VAR>
__device__ __forceinline__ void btcs_steps(int64_t nsteps, int iters, T r, T s, int n,
                                           BtcsShared<T, NT>& sm, T* hfirst, T* hlast, T* c0,
                                           T* us, T* lo, T* es) {
  constexpr bool ITER = VAR == VAR_PICARD || VAR == VAR_NEWTON;
  constexpr bool PER = BCT == BC_PERIODIC;
  constexpr bool DEFER = VAR != VAR_NEWTON;  // neighbour values folded into the reduced rows
  const T kap = VAR == VAR_CN ? T(2) : T(1);
  constexpr int Q = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tl = EXACT ? NT - 1 : (n - 1) / C;  // chunk holding node n-1
  const int jstar = n - 1 - tid * C;              // local index of node n-1
  const int je = EXACT ? C - 1 : (jstar < C ? jstar : C - 1);  // chunk end row
  // Ragged rows: only the warp holding node n-1 runs the general sweep (its
  // backward sweep restarts at the chunk's end row); warps inside the row run the exact-row
  // sweep and warps wholly past the end skip it. Warp-uniform: no warp runs
  // two paths. Both sweeps in one kernel need registers for both: FP32
  // shapes of up to 16 nodes a thread and 512 threads have them; the others
  // keep the general sweep in every warp (two copies of a 32-node sweep
  // spill).
  constexpr bool WSPLIT = !EXACT && sizeof(T) == 4 && C <= 16 && NT <= 512;
  // (a chunk that ends exactly at node n-1 is an interior one, unless it
  // holds a Dirichlet end row; lanes past the end compute values nobody reads)
  const bool rw_edge =
      WSPLIT ? __any_sync(FULL_MASK, (jstar >= 0 && jstar < C - 1) ||
                                         (BCT == BC_DIRICHLET && tid == tl)) != 0
             : !EXACT;
  const bool rw_pad = WSPLIT && __all_sync(FULL_MASK, jstar < 0) != 0;
  const bool endslot = !EXACT && jstar >= 0 && jstar < C - 1;  // padding after node n-1
  // matrix coefficients (Crank-Nicolson: half of the step's r and s)
  const T rm = VAR == VAR_CN ? T(0.5) * r : r, smat = VAR == VAR_CN ? T(0.5) * s : s;
  const T ds1 = T(1) + T(2) * smat;
  const T hr = T(0.5) * r;
  const int nit = ITER ? iters : 1;
  // the current iterate (u^n itself for the single-solve variants)
  auto uval = [&](int j, int t) -> T {
    if constexpr (ITER) return us[j * NT + t] + es[j * NT + t];
    else return us[j * NT + t];
  };
  // value of node j of chunk t for the next solve, from this solve's
  // increment (the owner's arithmetic)
  auto next_u = [&](int j, int t, T delta, bool last) -> T {
    T inc = delta;
    if constexpr (ITER) {
      inc = es[j * NT + t] + delta;
      if (!last) return us[j * NT + t] + inc;
    }
    T l0 = T(0);
    if constexpr (Kahan<T>::on) l0 = lo[j * NT + t];
    return comp_add(us[j * NT + t], inc, l0);
  };
  T ch[C], ah[C], dd[C];
  for (int64_t step = 0; step < nsteps; ++step) {
  if constexpr (ITER) {
#pragma unroll
    for (int j = 0; j < C; ++j) es[j * NT + tid] = T(0);
  }
  for (int it = 0; it < nit; ++it) {
    const bool last = it + 1 == nit;
    T left = T(0), right = T(0);
    if constexpr (!DEFER) {
      if (tid > 0) left = hlast[tid - 1];
      else if constexpr (PER) left = hlast[tl];
      if (tid < tl) right = hfirst[tid + 1];
      else if constexpr (PER) right = hfirst[0];
    }
    // ---- assembly of rows and right-hand sides fused with the forward sweep,
    // then the backward sweep: (delta, alpha, gamma) into (dd, ah, ch). G: the
    // general chunk (the row's end or padding inside it) of a ragged row.
    T e_ch = T(0), e_ah = T(0), e_dh = T(0);
    auto sweep = [&](auto gen_tag) {
    constexpr bool G = decltype(gen_tag)::value;
    if constexpr (G) {
      // the end row reads its right neighbour from the first padding slot
      // (deferred rows: the node itself); padding slots have es = 0
      if (endslot) us[(jstar + 1) * NT + tid] = DEFER ? uval(jstar, tid) : right;
    }
    T chp = T(0), ahp = T(-1), dhp = T(0);
    T ul = left, a = uval(0, tid);
    if constexpr (DEFER) ul = a;
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const T an = (j + 1 < C) ? uval(j + 1, tid) : right;
      T ur = an;
      if constexpr (DEFER) {
        if (j == C - 1) ur = a;  // end row of the chunk
      }
      T l, c, d, rhs;
      if constexpr (VAR == VAR_NEWTON) {
        const T e = es[j * NT + tid];
        const T ha = hr * a;
        l = -ha - s;
        c = ha - s;
        d = tfma(hr, ur - ul, ds1);
        rhs = tfma(s, (ur - a) - (a - ul), tfma(-ha, ur - ul, -e));
      } else {
        const T ra = rm * a;
        l = -smat - tmax(ra, T(0));
        c = tmin(ra, T(0)) - smat;
        d = ds1 + tabs(ra);
        // explicit increment (Eq. 21) from the same coefficients: -c (ur - a) + l (a - ul)
        rhs = tfma(l, a - ul, -c * (ur - a));
        if constexpr (VAR == VAR_CN) rhs = T(2) * rhs;  // the full step's increment
        if constexpr (VAR == VAR_PICARD) rhs = rhs - es[j * NT + tid];
      }
      bool ident = false;
      if constexpr (BCT == BC_DIRICHLET) {
        if constexpr (EXACT)
          ident = (j == 0 && tid == 0) || (j == C - 1 && tid == NT - 1);
        else  // ragged: the row's first node (its last one: end relation below)
          ident = j == 0 && tid == 0;
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
    T cd = T(0), ca = T(0), cg = T(-1);
    if constexpr (!G) {
      e_ch = ch[C - 1]; e_ah = ah[C - 1]; e_dh = dd[C - 1];
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
      // restarted at the end row je; rows past it (padding, finite values of
      // a diagonally dominant system) are never used
      e_ch = ch[C - 1]; e_ah = ah[C - 1]; e_dh = dd[C - 1];
      dd[C - 1] = T(0); ah[C - 1] = T(0); ch[C - 1] = T(-1);
#pragma unroll
      for (int j = C - 2; j >= 0; --j) {
        const T cj = ch[j];
        const bool at = j == je;
        if (at) { e_ch = cj; e_ah = ah[j]; e_dh = dd[j]; }
        cd = at ? T(0) : tfma(-cj, cd, dd[j]);
        ca = at ? T(0) : tfma(-cj, ca, ah[j]);
        cg = at ? T(-1) : -cj * cg;
        dd[j] = cd; ah[j] = ca; ch[j] = cg;
      }
      // Dirichlet: the row's last node is an identity row, which leaves the
      // chunk's end relation zero
      if (BCT == BC_DIRICHLET && tid == tl) { e_ch = T(0); e_ah = T(0); e_dh = T(0); }
    }
    };
    if constexpr (!WSPLIT) {
      if constexpr (EXACT) sweep(std::false_type{});
      else sweep(std::true_type{});
    } else if (!rw_edge && !rw_pad) {
      sweep(std::false_type{});
    } else if (rw_edge) {
      sweep(std::true_type{});
    } else {  // padding chunks: identity rows, what the general sweep leaves
      dd[0] = T(0); ah[0] = T(0); ch[0] = T(0);
    }
    // ---- this chunk's first-row relation (the previous chunk's row reads it);
    // chunk 0 also publishes its end relation (every row's corner split does)
    sm.rd[sk(tid)] = dd[0];
    sm.ra[sk(tid)] = ah[0];
    sm.rg[sk(tid)] = ch[0];
    if constexpr (PER) {
      if (tid == 0) { c0[0] = e_ah; c0[1] = e_ch; }
    }
    __syncthreads();
    // u_left - u_0 of this chunk, from the values published before the barrier
    T lft = T(0);
    if constexpr (DEFER) {
      if (tid > 0) lft = hlast[tid - 1] - hfirst[tid];
      else if constexpr (PER) lft = hlast[tl] - hfirst[0];
    }
    // ---- the reduced row of this thread's chunk t: its end row with the
    // first-row relation of chunk t + 1 substituted (chunk 0 after the last).
    // Periodic rows split their corners off here (Sherman-Morrison, gamma =
    // -B_0, as reduced_solve does): threads 0 and tl modify their rows, and
    // every thread knows the ratio A_0 / gamma.
    T fa = T(0);
    {
      const int t = tid, i = sk(t);
      T A = T(0), B = T(1), Cc = T(0), D = T(0), U = T(0);
      if (t <= tl) {
        const int nx = (t == tl) ? 0 : t + 1;
        const T ech = e_ch, ran = sm.ra[sk(nx)];
        A = e_ah;
        T Dt = e_dh, rdn = sm.rd[sk(nx)];
        if constexpr (DEFER) {
          // neighbour differences of chunk t's edges; the end node of chunk t
          // is the left neighbour of chunk nx's first node
          const T f = hfirst[t], e = hlast[t], fn = hfirst[nx];
          T lt = T(0), rt = T(0);
          if (t > 0) lt = hlast[t - 1] - f;
          else if constexpr (PER) lt = hlast[tl] - f;
          if (t < tl) rt = fn - e;
          else if constexpr (PER) rt = fn - e;
          Dt = tfma(-kap * A, lt, tfma(-kap * ech, rt, Dt));
          rdn = tfma(-kap * ran, e - fn, rdn);
        }
        B = T(1) - ech * ran;
        Cc = -ech * sm.rg[sk(nx)];
        D = tfma(-ech, rdn, Dt);
      }
      if constexpr (PER) {
        // chunk 0's row (tl >= 1: its next chunk is chunk 1), as thread 0 forms it
        const T A0 = c0[0], B0 = T(1) - c0[1] * sm.ra[sk(1)];
        const T gam = -B0;
        fa = A0 * recip(gam);
        if (t == 0) { B = B0 - gam; A = T(0); U = gam; }
        if (t == tl) { B = B - Cc * fa; U = Cc; Cc = T(0); }
      }
      sm.A[i] = A; sm.B[i] = B; sm.Cc[i] = Cc; sm.D[i] = D; sm.U[i] = U;
    }
    __syncthreads();
    if (warp == Q - 1) {  // the last warp (warp 0 also carries the row's first node)
      reduced_solve<T, NT, PER, true>(sm, tl, lane, fa);
      // next step's first and last node of each chunk (Newton)
      if constexpr (!DEFER) {
      __syncwarp();
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
          hfirst[t] = next_u(0, t, d0, last);
          hlast[t] = next_u(jt, t, Xt, last);
        }
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
      if constexpr (DEFER) L = tfma(kap, lft, L);
      auto update = [&](auto gen_tag) {
      constexpr bool G = decltype(gen_tag)::value;
#pragma unroll
      for (int j = 0; j < C; ++j) {
        const bool jend = G ? j == je : j == C - 1;
        if (!G || j <= je) {
          const T delta = jend ? Xt : tfma(-ch[j], Xt, tfma(-ah[j], L, dd[j]));
          const int o = j * NT + tid;
          T inc = delta;
          if constexpr (ITER) {
            inc = es[o] + delta;
            if (!last) {
              es[o] = inc;
              if constexpr (DEFER) {
                // the next iterate's edge values
                if (j == 0) hfirst[tid] = us[o] + inc;
                if (jend) hlast[tid] = us[o] + inc;
              }
              continue;
            }
          }
          T l0 = T(0);
          if constexpr (Kahan<T>::on) l0 = lo[o];
          const T nv = comp_add(us[o], inc, l0);
          us[o] = nv;
          if constexpr (Kahan<T>::on) lo[o] = l0;
          if constexpr (DEFER) {
            if (j == 0) hfirst[tid] = nv;
            if (jend) hlast[tid] = nv;
          }
        }
      }
      };
      if constexpr (!WSPLIT) {
        if constexpr (EXACT) update(std::false_type{});
        else update(std::true_type{});
      } else if (rw_edge) {
        update(std::true_type{});
      } else {
        update(std::false_type{});
      }
    }
  }  // iterations
  }  // steps
}

// FP32: at most 128 registers per thread, so 512 threads' worth of CTAs fit
// on an SM (four CTAs of the 128 x 32 shape hide each other's serial phase).
template <typename T, int NT, int C, bool EXACT, int VAR>
__global__ void __launch_bounds__(NT, (sizeof(T) == 4 && NT <= 512) ? 512 / NT : 1)
    k_btcs_resident(T* __restrict__ u,
                                                      const RowDesc* __restrict__ rows, int count,
                                                      int* __restrict__ counter) {
  __shared__ BtcsShared<T, NT> sm;
  __shared__ T hfirst[NT], hlast[NT], c0[2];
  __shared__ int s_item;
  extern __shared__ __align__(16) unsigned char dsm[];
  T* us = reinterpret_cast<T*>(dsm);                   // C * NT values
  T* lo = us + C * NT;                                 // C * NT values (FP32)
  T* es = us + (Kahan<T>::on ? 2 : 1) * C * NT;        // C * NT values (iterating variants)
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
      btcs_steps<T, NT, C, EXACT, BC_PERIODIC, VAR>(rd.nsteps, rd.iters, r, s, n, sm, hfirst,
                                                    hlast, c0, us, lo, es);
    else
      btcs_steps<T, NT, C, EXACT, BC_DIRICHLET, VAR>(rd.nsteps, rd.iters, r, s, n, sm, hfirst,
                                                     hlast, c0, us, lo, es);
#pragma unroll
    for (int j = 0; j < C; ++j)
      if (EXACT || base + j < n) row[base + j] = us[j * NT + tid];
    __syncthreads();
  }
}

}  // namespace burgers
