// explicit.cu -- explicit forward-Euler upwind/central kernels (Eq. 21,
// upwind side by the sign of u_i as in Sec. 2.2).
//
// Layout: thread t of a CTA holds C consecutive nodes of a row in registers.
// Neighbour values cross lanes by warp shuffles and cross warps through a
// double-buffered shared-memory slot per warp, so one step costs one
// __syncthreads (none for single-warp rows) and, per node, five FMA-pipe
// operations (FP64: six); FP32 adds one to evaluate its split state (value at
// the last fold plus the increments since) and three every 32 steps to fold
// it, and runs them on packed f32x2 pairs (half the instructions to issue)
// with the upwind min/max on the ALU pipe.
//
//  * k_explicit_resident: the whole row lives in registers for all of its
//    steps (the paper's time loop runs inside the kernel). CTAs are
//    persistent and take rows from an atomic counter over a host list sorted
//    by cost, so one launch drains thousands of uneven rows.
//  * k_explicit_stream: rows too long to stay resident. A CTA loads a window
//    of W = NT*C nodes, advances it K steps (the valid region shrinks by one
//    node per side per step: trapezoidal temporal blocking) and writes the
//    central W - 2K nodes, so a pass costs about 2*sizeof(T) bytes of HBM per
//    node for K steps.
#include <type_traits>

#include "common.cuh"
#include "kernels.h"
#include "step1.cuh"

namespace burgers {

enum : int { MODE_EXACT = 0, MODE_RAGGED = 1, MODE_WINDOW = 2, MODE_WINDOW_DIR = 3 };
enum : int { INTEG_EULER = 0, INTEG_RK4 = 1 };

// Exchanges this thread's edge values for its neighbours' (left = value of
// the node before its first, right = after its last). Periodic rows wrap
// through the slots of the first and last warp; WRAPX rows (ragged periodic)
// also publish node n-1 and node 0 (wrap_sel, first of thread 0).
// Branch-free: within a warp the values move by shuffles; across warps lane
// 31 publishes its last value and lane 0 its first with one predicated
// store, and after the barrier every lane reads the neighbour warps' slots
// (broadcast loads) and the edge lanes select them.
template <typename T, int NT, bool WRAPX>
__device__ __forceinline__ void halo_exchange(T first, T last, T wrap_sel, bool has_wrap, int p,
                                              T* sh_last, T* sh_first, T* sh_wrap, T& left,
                                              T& right, T& wrapL, T& wrapR) {
  constexpr int NW = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  left = shfl(last, (lane + 31) & 31);
  right = shfl(first, (lane + 1) & 31);
  if constexpr (NW > 1) {
    const bool lo_lane = lane == 0;
    st_shared_if((lo_lane ? sh_first : sh_last) + p * NW + warp, lo_lane ? first : last,
                 lo_lane || lane == 31);
  }
  if constexpr (WRAPX) {
    st_shared_if(sh_wrap + p * 2 + 0, wrap_sel, has_wrap);
    st_shared_if(sh_wrap + p * 2 + 1, first, tid == 0);
  }
  if constexpr (NW > 1 || WRAPX) __syncthreads();
  if constexpr (NW > 1) {
    const T lv = sh_last[p * NW + (warp + NW - 1) % NW];
    const T rv = sh_first[p * NW + (warp + 1) % NW];
    left = lane == 0 ? lv : left;
    right = lane == 31 ? rv : right;
  }
  if constexpr (WRAPX) {
    wrapL = sh_wrap[p * 2 + 0];
    wrapR = sh_wrap[p * 2 + 1];
  }
}

// Whether node j of this thread keeps its value (end rows, padding).
template <int NT, int C, int MODE, int BCT>
__device__ __forceinline__ bool keep_node(int j, int jstar, int64_t gbase, int n) {
  const int tid = threadIdx.x;
  if constexpr (MODE == MODE_EXACT && BCT == BC_DIRICHLET) {
    return (j == 0 && tid == 0) || (j == C - 1 && tid == NT - 1);
  } else if constexpr (MODE == MODE_RAGGED) {
    bool keep = j > jstar;  // padding
    if constexpr (BCT == BC_DIRICHLET) keep = keep || j == jstar || (j == 0 && tid == 0);
    return keep;
  } else if constexpr (MODE == MODE_WINDOW_DIR) {
    const int64_t gi = gbase + j;
    return gi == 0 || gi == n - 1;
  } else {
    return false;
  }
}

// Ragged rows (MODE_RAGGED): only the warp holding node n-1 needs the
// per-node end and padding tests; warps wholly inside the row run the loop
// of an exact row, and warps wholly past its end (padding) skip the update.
// The tests are warp-uniform, so no warp runs two paths.
struct RaggedWarp {
  bool ragged, edge, pad;
};
template <int C, int MODE>
__device__ __forceinline__ RaggedWarp ragged_warp(int jstar) {
  if constexpr (MODE == MODE_RAGGED) {
    return {true, __any_sync(FULL_MASK, jstar >= 0 && jstar < C) != 0,
            __all_sync(FULL_MASK, jstar < 0) != 0};
  } else {
    return {false, false, false};
  }
}

// keep_node for the two warp classes of a ragged row: EDGE = the general
// test; otherwise (interior warp, every jstar >= C) only a Dirichlet row's
// first node is held.
template <int NT, int C, int MODE, int BCT, bool EDGE>
__device__ __forceinline__ bool keep_node_w(int j, int jstar, int64_t gbase, int n) {
  if constexpr (MODE == MODE_RAGGED && !EDGE) {
    return BCT == BC_DIRICHLET && j == 0 && threadIdx.x == 0;
  } else {
    return keep_node<NT, C, MODE, BCT>(j, jstar, gbase, n);
  }
}

// FP32 steps with a split state: each node carries uh (its value at the last
// fold) and d (the increments summed since), and a step evaluates the stencil
// on u = uh + d and adds the increment to d. Every SPLIT_FOLD steps, and after the
// last one, d is folded into uh with its rounding error kept in d (the same
// two-sum as compensated summation), so increments are never rounded against
// the full magnitude of u between folds. On entry and exit the state is
// (v, lo) with the true value v - lo, as in Kahan summation.
//
// Even C runs on packed FP32 pairs: pair k holds nodes k and k + C/2 of the
// thread's chunk, so the right neighbour of pair k is pair k + 1 in both
// lanes and only the last pair's right and the first pair's left neighbours
// are assembled from the other half and the halo. With m = min(u, 0) and
// M = max(u, 0), the upwind coefficients are p = s - r m = s + (r/2)(|u| - u)
// and q = s + r M = p + r u (Eq. 21), each one FMA from the min/max (which
// run on the ALU pipe), and the increment p (u_r - u) - q (u - u_l) is two
// more FMAs.
template <int NT, int C, int MODE, int BCT>
__device__ __forceinline__ void explicit_steps_split_x2(float (&v)[C], float (&lo)[C],
                                                        int64_t nsteps, float r, float s, int n,
                                                        int64_t gbase, float* sh_last,
                                                        float* sh_first, float* sh_wrap) {
  static_assert(C % 2 == 0, "pairs of nodes");
  constexpr int H = C / 2;
  constexpr bool WRAPX = (MODE == MODE_RAGGED && BCT == BC_PERIODIC);
  const int tid = threadIdx.x;
  const int jstar = int(n - 1 - gbase);  // local index of node n-1 (resident modes)
  const RaggedWarp rw = ragged_warp<C, MODE>(jstar);
  float2 V[H], D[H];
#pragma unroll
  for (int k = 0; k < H; ++k) {
    V[k] = make_float2(v[k], v[k + H]);
    D[k] = make_float2(-lo[k], -lo[k + H]);
  }
  const float2 NR = make_float2(-r, -r), S2 = make_float2(s, s), NS = make_float2(-s, -s);
  for (int64_t k0 = 0; k0 < nsteps; k0 += SPLIT_FOLD) {
   const int kb = int(nsteps - k0 < SPLIT_FOLD ? nsteps - k0 : int64_t(SPLIT_FOLD));
   for (int kk = 0; kk < kb; ++kk) {
    const int p = kk & 1;
    const float2 U0 = add2(V[0], D[0]);
    const float2 UL = add2(V[H - 1], D[H - 1]);
    float wsel = 0.f;
    bool has_wrap = false;
    if constexpr (WRAPX) {
      has_wrap = jstar >= 0 && jstar < C;
      if (rw.edge) {  // only the warp holding node n-1 looks for it
        float sv = V[0].x, sd = D[0].x;
#pragma unroll
        for (int j = 1; j < C; ++j)
          if (j == jstar) {
            sv = j < H ? V[j].x : V[j - H].y;
            sd = j < H ? D[j].x : D[j - H].y;
          }
        wsel = sv + sd;
      }
    }
    float left, right, wrapL = 0.f, wrapR = 0.f;
    halo_exchange<float, NT, WRAPX>(U0.x, UL.y, wsel, has_wrap, p, sh_last, sh_first, sh_wrap,
                                    left, right, wrapL, wrapR);
    float wl0 = left;
    if constexpr (WRAPX) {
      if (tid == 0) wl0 = wrapL;
    }
    auto update = [&](auto edge_tag) {
      constexpr bool EDGE = decltype(edge_tag)::value;
      float2 Uk = U0;
      float2 DL = sub2(U0, make_float2(wl0, UL.x));  // u - u_l of pair 0
#pragma unroll
      for (int k = 0; k < H; ++k) {
        float2 UR = (k + 1 < H) ? add2(V[k + 1], D[k + 1]) : make_float2(U0.y, right);
        const float2 Un = UR;
        if constexpr (WRAPX && EDGE) {
          if (k == jstar) UR.x = wrapR;
          if (k + H == jstar) UR.y = wrapR;
        }
        const float2 E = sub2(UR, Uk);  // u_r - u
        const float2 m = make_float2(fminf(Uk.x, 0.f), fminf(Uk.y, 0.f));
        const float2 M = make_float2(fmaxf(Uk.x, 0.f), fmaxf(Uk.y, 0.f));
        const float2 P = fma2(NR, m, S2);   // p
        const float2 NQ = fma2(NR, M, NS);  // -q
        const float2 dn = fma2(P, E, fma2(NQ, DL, D[k]));
        if (!keep_node_w<NT, C, MODE, BCT, EDGE>(k, jstar, gbase, n)) D[k].x = dn.x;
        if (!keep_node_w<NT, C, MODE, BCT, EDGE>(k + H, jstar, gbase, n)) D[k].y = dn.y;
        DL = E;
        Uk = Un;
      }
    };
    if (!rw.ragged || rw.edge) update(std::true_type{});
    else if (!rw.pad) update(std::false_type{});
   }
#pragma unroll
    for (int k = 0; k < H; ++k) {
      const float2 t = add2(V[k], D[k]);
      D[k] = sub2(D[k], sub2(t, V[k]));
      V[k] = t;
    }
  }
#pragma unroll
  for (int k = 0; k < H; ++k) {
    v[k] = V[k].x;
    v[k + H] = V[k].y;
    lo[k] = -D[k].x;
    lo[k + H] = -D[k].y;
  }
}

// Ragged FP32 rows on packed pairs, chunks of C or C - 1 nodes (as the BTCS
// kernels cut them): tl = ceil(n / C) - 1 is the last thread holding nodes,
// and a short chunk's second half ends at pair C/2 - 2, its pair C/2 - 1
// padding. Every end and padding position is known at compile time, so all
// warps run one loop with a few selects there; the periodic wrap pairs the
// last node of thread tl with thread 0's first through the wrap slots.
// Threads past tl update values that no node reads (their neighbour chain
// starts at thread tl's last node, whose right neighbour is replaced) and
// are never written back.
template <int NT, int C, int BCT>
__device__ __forceinline__ void explicit_steps_split_x2_cc(float (&v)[C], float (&lo)[C],
                                                           int64_t nsteps, float r, float s,
                                                           int tl, bool shrt, float* sh_last,
                                                           float* sh_first, float* sh_wrap) {
  static_assert(C % 2 == 0 && C >= 4, "pairs of nodes, a short half of at least one");
  // warps wholly past thread tl skip the update (their values stay zero)
  const bool padwarp = __all_sync(FULL_MASK, int(threadIdx.x) > tl) != 0;
  constexpr int H = C / 2;
  constexpr bool PER = BCT == BC_PERIODIC;
  const int tid = threadIdx.x;
  const bool dfirst = !PER && tid == 0;
  const bool dlast = !PER && tid == tl;
  float2 V[H], D[H];
#pragma unroll
  for (int k = 0; k < H; ++k) {
    V[k] = make_float2(v[k], v[k + H]);
    D[k] = make_float2(-lo[k], -lo[k + H]);
  }
  const float2 NR = make_float2(-r, -r), S2 = make_float2(s, s), NS = make_float2(-s, -s);
  for (int64_t k0 = 0; k0 < nsteps; k0 += SPLIT_FOLD) {
   const int kb = int(nsteps - k0 < SPLIT_FOLD ? nsteps - k0 : int64_t(SPLIT_FOLD));
   for (int kk = 0; kk < kb; ++kk) {
    const int p = kk & 1;
    const float2 U0 = add2(V[0], D[0]);
    const float2 UL = add2(V[H - 1], D[H - 1]);
    const float2 UE = add2(V[H - 2], D[H - 2]);
    const float last = shrt ? UE.y : UL.y;  // the chunk's last node
    float left, right, wrapL = 0.f, wrapR = 0.f;
    halo_exchange<float, NT, PER>(U0.x, last, last, tid == tl, p, sh_last, sh_first, sh_wrap,
                                  left, right, wrapL, wrapR);
    if constexpr (PER) {
      if (tid == 0) left = wrapL;
      if (tid == tl) right = wrapR;
    }
    if (padwarp) continue;
    float2 Uk = U0;
    float2 DL = sub2(U0, make_float2(left, UL.x));  // u - u_l of pair 0
#pragma unroll
    for (int k = 0; k < H; ++k) {
      float2 UR = (k + 1 < H) ? add2(V[k + 1], D[k + 1]) : make_float2(U0.y, right);
      const float2 Un = UR;
      if (k == H - 2 && shrt) UR.y = right;  // a short chunk's end node
      const float2 E = sub2(UR, Uk);         // u_r - u
      const float2 m = make_float2(fminf(Uk.x, 0.f), fminf(Uk.y, 0.f));
      const float2 M = make_float2(fmaxf(Uk.x, 0.f), fmaxf(Uk.y, 0.f));
      const float2 P = fma2(NR, m, S2);   // p
      const float2 NQ = fma2(NR, M, NS);  // -q
      const float2 dn = fma2(P, E, fma2(NQ, DL, D[k]));
      // held: a Dirichlet row's first and last nodes, a short chunk's padding
      bool keepx = false, keepy = false;
      if (k == 0) keepx = dfirst;
      if (k == H - 2) keepy = shrt && dlast;
      if (k == H - 1) keepy = shrt || dlast;
      if (!keepx) D[k].x = dn.x;
      if (!keepy) D[k].y = dn.y;
      DL = E;
      Uk = Un;
    }
   }
#pragma unroll
    for (int k = 0; k < H; ++k) {
      const float2 t = add2(V[k], D[k]);
      D[k] = sub2(D[k], sub2(t, V[k]));
      V[k] = t;
    }
  }
#pragma unroll
  for (int k = 0; k < H; ++k) {
    v[k] = V[k].x;
    v[k + H] = V[k].y;
    lo[k] = -D[k].x;
    lo[k + H] = -D[k].y;
  }
}

template <int NT, int C, int MODE, int BCT>
__device__ __forceinline__ void explicit_steps_split(float (&v)[C], float (&lo)[C], int64_t nsteps,
                                                     float r, float h, float s, int n,
                                                     int64_t gbase, float* sh_last,
                                                     float* sh_first, float* sh_wrap) {
  if constexpr (C % 2 == 0) {
    (void)h;
    explicit_steps_split_x2<NT, C, MODE, BCT>(v, lo, nsteps, r, s, n, gbase, sh_last, sh_first,
                                              sh_wrap);
    return;
  }
  constexpr bool WRAPX = (MODE == MODE_RAGGED && BCT == BC_PERIODIC);
  const int tid = threadIdx.x;
  const int jstar = int(n - 1 - gbase);  // local index of node n-1 (resident modes)
  const RaggedWarp rw = ragged_warp<C, MODE>(jstar);
  // lo becomes d = -lo
#pragma unroll
  for (int j = 0; j < C; ++j) lo[j] = -lo[j];
  // blocks of SPLIT_FOLD steps (the last one shorter) with a fold after each;
  // SPLIT_FOLD is even, so kk & 1 is the parity of the global step index
  for (int64_t k0 = 0; k0 < nsteps; k0 += SPLIT_FOLD) {
   const int kb = int(nsteps - k0 < SPLIT_FOLD ? nsteps - k0 : int64_t(SPLIT_FOLD));
   for (int kk = 0; kk < kb; ++kk) {
    const int p = kk & 1;
    const float first = v[0] + lo[0];
    const float last = v[C - 1] + lo[C - 1];
    float wsel = 0.f;
    bool has_wrap = false;
    if constexpr (WRAPX) {
      has_wrap = jstar >= 0 && jstar < C;
      if (rw.edge) {  // only the warp holding node n-1 looks for it
        float sv = v[0], sd = lo[0];
#pragma unroll
        for (int j = 1; j < C; ++j)
          if (j == jstar) { sv = v[j]; sd = lo[j]; }
        wsel = sv + sd;
      }
    }
    float left, right, wrapL = 0.f, wrapR = 0.f;
    halo_exchange<float, NT, WRAPX>(first, last, wsel, has_wrap, p, sh_last, sh_first, sh_wrap,
                                    left, right, wrapL, wrapR);
    float wl0 = left;
    if constexpr (WRAPX) {
      if (tid == 0) wl0 = wrapL;
    }
    auto update = [&](auto edge_tag) {
      constexpr bool EDGE = decltype(edge_tag)::value;
      float wl = wl0, wc = first;
#pragma unroll
      for (int j = 0; j < C; ++j) {
        float wr = (j + 1 < C) ? v[j + 1] + lo[j + 1] : right;
        if constexpr (WRAPX && EDGE) {
          if (j == jstar) wr = wrapR;
        }
        const float dn = explicit_increment(wc, wl, wr, r, h, s, lo[j]);
        if (!keep_node_w<NT, C, MODE, BCT, EDGE>(j, jstar, gbase, n)) lo[j] = dn;
        wl = wc;
        wc = wr;
      }
    };
    if (!rw.ragged || rw.edge) update(std::true_type{});
    else if (!rw.pad) update(std::false_type{});
   }
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const float t = v[j] + lo[j];
      lo[j] = lo[j] - (t - v[j]);
      v[j] = t;
    }
  }
#pragma unroll
  for (int j = 0; j < C; ++j) lo[j] = -lo[j];
}

// Classical fourth-order Runge-Kutta in time (Eq. 22) on the same spatial
// operator. With Delta(w) the forward-Euler increment of the state w for the
// whole dt (p (w_r - w) - q (w - w_l), as above), a step is
//   K1 = Delta(u), K2 = Delta(u + K1/2), K3 = Delta(u + K2/2), K4 = Delta(u + K3),
//   u' = u + (K1 + 2 K2 + 2 K3 + K4)/6,
// i.e. Eq. 22 with k_j = K_j/dt. Every stage needs its own neighbour exchange.
// Held nodes (Dirichlet ends, padding) have zero increments in every stage.
// FP32 keeps the split state of explicit_steps_split (the stage states are
// evaluated from it; the step's combined increment goes into d); FP64 adds the
// combined increment to u directly.
// FP32 RK4 with even C on packed pairs (nodes k and k + C/2, as in
// explicit_steps_split_x2); bitwise the arithmetic of rk4_steps below.
template <int NT, int C, int MODE, int BCT>
__device__ __forceinline__ void rk4_steps_x2(float (&v)[C], float (&lo)[C], int64_t nsteps,
                                             float r, float s, int n, int64_t gbase,
                                             float* sh_last, float* sh_first, float* sh_wrap) {
  static_assert(C % 2 == 0, "pairs of nodes");
  constexpr int H = C / 2;
  constexpr bool WRAPX = (MODE == MODE_RAGGED && BCT == BC_PERIODIC);
  const int tid = threadIdx.x;
  const int jstar = int(n - 1 - gbase);
  const RaggedWarp rw = ragged_warp<C, MODE>(jstar);
  float2 V[H], D[H], K[H], ACC[H];
#pragma unroll
  for (int k = 0; k < H; ++k) {
    V[k] = make_float2(v[k], v[k + H]);
    D[k] = make_float2(-lo[k], -lo[k + H]);
    K[k] = make_float2(0.f, 0.f);
  }
  const float2 NR = make_float2(-r, -r), S2 = make_float2(s, s), NS = make_float2(-s, -s);
  const float2 Z2 = make_float2(0.f, 0.f);
  for (int64_t k0 = 0; k0 < nsteps; k0 += SPLIT_FOLD) {
   const int kb = int(nsteps - k0 < SPLIT_FOLD ? nsteps - k0 : int64_t(SPLIT_FOLD));
   for (int kk = 0; kk < kb; ++kk) {
    float2 U[H];
#pragma unroll
    for (int k = 0; k < H; ++k) U[k] = add2(V[k], D[k]);
#pragma unroll
    for (int st = 0; st < 4; ++st) {
      const float cs = st == 0 ? 0.f : (st == 3 ? 1.f : 0.5f);
      const float2 CST = make_float2(cs, cs);
      float2 W[H];
#pragma unroll
      for (int k = 0; k < H; ++k) W[k] = st == 0 ? U[k] : fma2(CST, K[k], U[k]);
      float wsel = 0.f;
      bool has_wrap = false;
      if constexpr (WRAPX) {
        has_wrap = jstar >= 0 && jstar < C;
        if (rw.edge) {
          wsel = W[0].x;
#pragma unroll
          for (int j = 1; j < C; ++j)
            if (j == jstar) wsel = j < H ? W[j].x : W[j - H].y;
        }
      }
      float left, right, wrapL = 0.f, wrapR = 0.f;
      halo_exchange<float, NT, WRAPX>(W[0].x, W[H - 1].y, wsel, has_wrap, st & 1, sh_last,
                                      sh_first, sh_wrap, left, right, wrapL, wrapR);
      float wl0 = left;
      if constexpr (WRAPX) {
        if (tid == 0) wl0 = wrapL;
      }
      auto stage = [&](auto edge_tag) {
        constexpr bool EDGE = decltype(edge_tag)::value;
        float2 DL = sub2(W[0], make_float2(wl0, W[H - 1].x));
#pragma unroll
        for (int k = 0; k < H; ++k) {
          float2 WR = (k + 1 < H) ? W[k + 1] : make_float2(W[0].y, right);
          if constexpr (WRAPX && EDGE) {
            if (k == jstar) WR.x = wrapR;
            if (k + H == jstar) WR.y = wrapR;
          }
          const float2 E = sub2(WR, W[k]);
          const float2 m = make_float2(fminf(W[k].x, 0.f), fminf(W[k].y, 0.f));
          const float2 M = make_float2(fmaxf(W[k].x, 0.f), fmaxf(W[k].y, 0.f));
          const float2 P = fma2(NR, m, S2);
          const float2 NQ = fma2(NR, M, NS);
          float2 kn = fma2(P, E, fma2(NQ, DL, Z2));
          if (keep_node_w<NT, C, MODE, BCT, EDGE>(k, jstar, gbase, n)) kn.x = 0.f;
          if (keep_node_w<NT, C, MODE, BCT, EDGE>(k + H, jstar, gbase, n)) kn.y = 0.f;
          if (st == 0) ACC[k] = kn;
          else {
            const float w = st == 3 ? 1.f : 2.f;
            ACC[k] = fma2(make_float2(w, w), kn, ACC[k]);
          }
          K[k] = kn;
          DL = E;
        }
      };
      if (!rw.ragged || rw.edge) {
        stage(std::true_type{});
      } else if (!rw.pad) {
        stage(std::false_type{});
      } else {
#pragma unroll
        for (int k = 0; k < H; ++k) {
          if (st == 0) ACC[k] = Z2;
          K[k] = Z2;
        }
      }
    }
    const float sx = 1.f / 6.f;
    const float2 SIX = make_float2(sx, sx);
#pragma unroll
    for (int k = 0; k < H; ++k) D[k] = fma2(SIX, ACC[k], D[k]);
   }
#pragma unroll
    for (int k = 0; k < H; ++k) {
      const float2 t = add2(V[k], D[k]);
      D[k] = sub2(D[k], sub2(t, V[k]));
      V[k] = t;
    }
  }
#pragma unroll
  for (int k = 0; k < H; ++k) {
    v[k] = V[k].x;
    v[k + H] = V[k].y;
    lo[k] = -D[k].x;
    lo[k + H] = -D[k].y;
  }
}

// RK4 (as rk4_steps_x2) on ragged FP32 rows cut into chunks of C or C - 1
// nodes, as explicit_steps_split_x2_cc cuts them: every stage exchanges the
// stage state's chunk edges (the periodic wrap through the wrap slots), and
// held nodes (a Dirichlet row's ends, a short chunk's padding) have zero
// increments in every stage.
template <int NT, int C, int BCT>
__device__ __forceinline__ void rk4_steps_x2_cc(float (&v)[C], float (&lo)[C], int64_t nsteps,
                                                float r, float s, int tl, bool shrt,
                                                float* sh_last, float* sh_first, float* sh_wrap) {
  static_assert(C % 2 == 0 && C >= 4, "pairs of nodes, a short half of at least one");
  constexpr int H = C / 2;
  constexpr bool PER = BCT == BC_PERIODIC;
  const int tid = threadIdx.x;
  const bool dfirst = !PER && tid == 0;
  const bool dlast = !PER && tid == tl;
  const bool padwarp = __all_sync(FULL_MASK, tid > tl) != 0;
  float2 V[H], D[H], K[H], ACC[H];
#pragma unroll
  for (int k = 0; k < H; ++k) {
    V[k] = make_float2(v[k], v[k + H]);
    D[k] = make_float2(-lo[k], -lo[k + H]);
    K[k] = make_float2(0.f, 0.f);
  }
  const float2 NR = make_float2(-r, -r), S2 = make_float2(s, s), NS = make_float2(-s, -s);
  const float2 Z2 = make_float2(0.f, 0.f);
  for (int64_t k0 = 0; k0 < nsteps; k0 += SPLIT_FOLD) {
   const int kb = int(nsteps - k0 < SPLIT_FOLD ? nsteps - k0 : int64_t(SPLIT_FOLD));
   for (int kk = 0; kk < kb; ++kk) {
    float2 U[H];
#pragma unroll
    for (int k = 0; k < H; ++k) U[k] = add2(V[k], D[k]);
#pragma unroll
    for (int st = 0; st < 4; ++st) {
      const float cs = st == 0 ? 0.f : (st == 3 ? 1.f : 0.5f);
      const float2 CST = make_float2(cs, cs);
      float2 W[H];
#pragma unroll
      for (int k = 0; k < H; ++k) W[k] = st == 0 ? U[k] : fma2(CST, K[k], U[k]);
      const float last = shrt ? W[H - 2].y : W[H - 1].y;  // the chunk's last node
      float left, right, wrapL = 0.f, wrapR = 0.f;
      halo_exchange<float, NT, PER>(W[0].x, last, last, tid == tl, st & 1, sh_last, sh_first,
                                    sh_wrap, left, right, wrapL, wrapR);
      if constexpr (PER) {
        if (tid == 0) left = wrapL;
        if (tid == tl) right = wrapR;
      }
      if (padwarp) {
#pragma unroll
        for (int k = 0; k < H; ++k) {
          if (st == 0) ACC[k] = Z2;
          K[k] = Z2;
        }
        continue;
      }
      float2 DL = sub2(W[0], make_float2(left, W[H - 1].x));
#pragma unroll
      for (int k = 0; k < H; ++k) {
        float2 WR = (k + 1 < H) ? W[k + 1] : make_float2(W[0].y, right);
        if (k == H - 2 && shrt) WR.y = right;  // a short chunk's end node
        const float2 E = sub2(WR, W[k]);
        const float2 m = make_float2(fminf(W[k].x, 0.f), fminf(W[k].y, 0.f));
        const float2 M = make_float2(fmaxf(W[k].x, 0.f), fmaxf(W[k].y, 0.f));
        const float2 P = fma2(NR, m, S2);
        const float2 NQ = fma2(NR, M, NS);
        float2 kn = fma2(P, E, fma2(NQ, DL, Z2));
        bool keepx = false, keepy = false;
        if (k == 0) keepx = dfirst;
        if (k == H - 2) keepy = shrt && dlast;
        if (k == H - 1) keepy = shrt || dlast;
        if (keepx) kn.x = 0.f;
        if (keepy) kn.y = 0.f;
        if (st == 0) ACC[k] = kn;
        else {
          const float w = st == 3 ? 1.f : 2.f;
          ACC[k] = fma2(make_float2(w, w), kn, ACC[k]);
        }
        K[k] = kn;
        DL = E;
      }
    }
    const float sx = 1.f / 6.f;
    const float2 SIX = make_float2(sx, sx);
#pragma unroll
    for (int k = 0; k < H; ++k) D[k] = fma2(SIX, ACC[k], D[k]);
   }
#pragma unroll
    for (int k = 0; k < H; ++k) {
      const float2 t = add2(V[k], D[k]);
      D[k] = sub2(D[k], sub2(t, V[k]));
      V[k] = t;
    }
  }
#pragma unroll
  for (int k = 0; k < H; ++k) {
    v[k] = V[k].x;
    v[k + H] = V[k].y;
    lo[k] = -D[k].x;
    lo[k + H] = -D[k].y;
  }
}

template <typename T, int NT, int C, int MODE, int BCT>
__device__ __forceinline__ void rk4_steps(T (&v)[C], T (&lo)[C], int64_t nsteps, T r, T h, T s,
                                          int n, int64_t gbase, T* sh_last, T* sh_first,
                                          T* sh_wrap) {
  if constexpr (sizeof(T) == 4 && C % 2 == 0) {
    (void)h;
    rk4_steps_x2<NT, C, MODE, BCT>(v, lo, nsteps, r, s, n, gbase, sh_last, sh_first, sh_wrap);
    return;
  }
  constexpr bool SPLIT = Kahan<T>::on;
  constexpr bool WRAPX = (MODE == MODE_RAGGED && BCT == BC_PERIODIC);
  const int tid = threadIdx.x;
  const int jstar = int(n - 1 - gbase);
  const RaggedWarp rw = ragged_warp<C, MODE>(jstar);
  if constexpr (SPLIT) {
#pragma unroll
    for (int j = 0; j < C; ++j) lo[j] = -lo[j];  // lo becomes d
  }
  T K[C], acc[C];
#pragma unroll
  for (int j = 0; j < C; ++j) K[j] = T(0);
  // blocks of SPLIT_FOLD steps (the last one shorter); FP32 folds after each
  for (int64_t k0 = 0; k0 < nsteps; k0 += SPLIT_FOLD) {
   const int kb = int(nsteps - k0 < SPLIT_FOLD ? nsteps - k0 : int64_t(SPLIT_FOLD));
   for (int kk = 0; kk < kb; ++kk) {
#pragma unroll
    for (int st = 0; st < 4; ++st) {
      const T cst = st == 0 ? T(0) : (st == 3 ? T(1) : T(0.5));
      // state of this stage at node j: u + cst * K_prev
      auto wv = [&](int j) -> T {
        T u = v[j];
        if constexpr (SPLIT) u = v[j] + lo[j];
        return st == 0 ? u : tfma(cst, K[j], u);
      };
      const T first = wv(0), last = wv(C - 1);
      T wsel = T(0);
      bool has_wrap = false;
      if constexpr (WRAPX) {
        has_wrap = jstar >= 0 && jstar < C;
        if (rw.edge) {
          T sv = v[0], sd = lo[0], sk = K[0];
#pragma unroll
          for (int j = 1; j < C; ++j)
            if (j == jstar) { sv = v[j]; sd = lo[j]; sk = K[j]; }
          T su = sv;
          if constexpr (SPLIT) su = sv + sd;
          wsel = st == 0 ? su : tfma(cst, sk, su);
        }
      }
      T left, right, wrapL = T(0), wrapR = T(0);
      halo_exchange<T, NT, WRAPX>(first, last, wsel, has_wrap, st & 1, sh_last, sh_first,
                                  sh_wrap, left, right, wrapL, wrapR);
      T wl0 = left;
      if constexpr (WRAPX) {
        if (tid == 0) wl0 = wrapL;
      }
      auto stage = [&](auto edge_tag) {
        constexpr bool EDGE = decltype(edge_tag)::value;
        T wl = wl0, wc = first;
#pragma unroll
        for (int j = 0; j < C; ++j) {
          T wr = (j + 1 < C) ? wv(j + 1) : right;
          if constexpr (WRAPX && EDGE) {
            if (j == jstar) wr = wrapR;
          }
          T kn = explicit_increment(wc, wl, wr, r, h, s, T(0));
          if (keep_node_w<NT, C, MODE, BCT, EDGE>(j, jstar, gbase, n)) kn = T(0);
          if (st == 0) acc[j] = kn;
          else acc[j] = tfma((st == 3) ? T(1) : T(2), kn, acc[j]);
          K[j] = kn;
          wl = wc;
          wc = wr;
        }
      };
      if (!rw.ragged || rw.edge) {
        stage(std::true_type{});
      } else if (!rw.pad) {
        stage(std::false_type{});
      } else {  // padding: held nodes, zero increments
#pragma unroll
        for (int j = 0; j < C; ++j) {
          if (st == 0) acc[j] = T(0);
          K[j] = T(0);
        }
      }
    }
    const T sixth = T(1) / T(6);
    if constexpr (SPLIT) {
#pragma unroll
      for (int j = 0; j < C; ++j) lo[j] = tfma(sixth, acc[j], lo[j]);
    } else {
#pragma unroll
      for (int j = 0; j < C; ++j) v[j] = tfma(sixth, acc[j], v[j]);
    }
   }
    if constexpr (SPLIT) {
#pragma unroll
      for (int j = 0; j < C; ++j) {
        const T t = v[j] + lo[j];
        lo[j] = lo[j] - (t - v[j]);
        v[j] = t;
      }
    }
  }
  if constexpr (SPLIT) {
#pragma unroll
    for (int j = 0; j < C; ++j) lo[j] = -lo[j];
  }
}

// Advances the C nodes held by this thread `nsteps` steps.
//   MODE_EXACT      row length n == NT*C; periodic wrap through the halo slots.
//   MODE_RAGGED     n < NT*C; nodes >= n are inert padding, the periodic wrap
//                   pairs node 0 with node n-1 explicitly.
//   MODE_WINDOW     streaming window; its two edges go stale one node per step.
//   MODE_WINDOW_DIR streaming window that contains a Dirichlet end node.
// gbase is the row index of this thread's first node. FP32 runs the split
// state above; FP64 updates the values in place. INTEG selects forward Euler
// (Eq. 21) or RK4 (Eq. 22).
template <typename T, int NT, int C, int MODE, int BCT, int INTEG = INTEG_EULER>
__device__ __forceinline__ void explicit_steps(T (&v)[C], T (&lo)[C], int64_t nsteps, T r, T h, T s,
                                               int n, int64_t gbase, T* sh_last, T* sh_first,
                                               T* sh_wrap) {
  if constexpr (INTEG == INTEG_RK4) {
    rk4_steps<T, NT, C, MODE, BCT>(v, lo, nsteps, r, h, s, n, gbase, sh_last, sh_first, sh_wrap);
  } else if constexpr (Kahan<T>::on) {
    explicit_steps_split<NT, C, MODE, BCT>(v, lo, nsteps, r, h, s, n, gbase, sh_last, sh_first,
                                           sh_wrap);
  } else {
    constexpr bool WRAPX = (MODE == MODE_RAGGED && BCT == BC_PERIODIC);
    const int tid = threadIdx.x;
    const int jstar = int(n - 1 - gbase);
    const RaggedWarp rw = ragged_warp<C, MODE>(jstar);
    for (int64_t k = 0; k < nsteps; ++k) {
      const int p = int(k & 1);
      const T first = v[0], last = v[C - 1];
      T wsel = T(0);
      bool has_wrap = false;
      if constexpr (WRAPX) {
        has_wrap = jstar >= 0 && jstar < C;
        if (rw.edge) {
          wsel = v[0];
#pragma unroll
          for (int j = 1; j < C; ++j)
            if (j == jstar) wsel = v[j];
        }
      }
      T left, right, wrapL = T(0), wrapR = T(0);
      halo_exchange<T, NT, WRAPX>(first, last, wsel, has_wrap, p, sh_last, sh_first, sh_wrap, left,
                                  right, wrapL, wrapR);
      T prev0 = left;
      if constexpr (WRAPX) {
        if (tid == 0) prev0 = wrapL;
      }
      auto update = [&](auto edge_tag) {
        constexpr bool EDGE = decltype(edge_tag)::value;
        T prev = prev0;
#pragma unroll
        for (int j = 0; j < C; ++j) {
          const T cur = v[j];
          T ur = (j + 1 < C) ? v[j + 1] : right;
          if constexpr (WRAPX && EDGE) {
            if (j == jstar) ur = wrapR;
          }
          const T nv = explicit_update(cur, prev, ur, r, h, s, lo[j]);
          if (!keep_node_w<NT, C, MODE, BCT, EDGE>(j, jstar, gbase, n)) v[j] = nv;
          prev = cur;
        }
      };
      if (!rw.ragged || rw.edge) update(std::true_type{});
      else if (!rw.pad) update(std::false_type{});
    }
  }
}

template <typename T, int NT, int C, bool EXACT, int INTEG = INTEG_EULER>
__global__ void __launch_bounds__(NT) k_explicit_resident(T* __restrict__ u,
                                                          const RowDesc* __restrict__ rows,
                                                          int count, int* __restrict__ counter) {
  constexpr int NW = NT / 32;
  __shared__ T sh_last[2 * NW], sh_first[2 * NW], sh_wrap[4];
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= count) return;
    const RowDesc rd = rows[item];
    T* row = u + rd.offset;
    const int base = threadIdx.x * C;
    // ragged FP32 rows on packed pairs: chunks of C or C - 1 nodes (forward
    // Euler, explicit_steps_split_x2_cc; RK4 from 16 nodes a thread,
    // rk4_steps_x2_cc: at 512 x 8 that form took 70 registers, one CTA a SM,
    // and measured no faster than the per-node end test); other ragged rows:
    // chunks of C with the end found per node in the warp holding it
    constexpr bool CC = !EXACT && sizeof(T) == 4 && C % 2 == 0 &&
                        (INTEG == INTEG_EULER ? C >= 4 : C >= 16);
    int cstart = base, clen = C, tl = NT - 1;
    bool shrt = false;
    if constexpr (CC) {
      const int tk = (rd.n + C - 1) / C, bk = tk * C - rd.n, ts = tk - bk;
      const bool active = int(threadIdx.x) < tk;
      shrt = active && int(threadIdx.x) >= ts;
      cstart = base - (shrt ? int(threadIdx.x) - ts : 0);
      clen = active ? (shrt ? C - 1 : C) : 0;
      tl = tk - 1;
    }
    T v[C], lo[C];
#pragma unroll
    for (int j = 0; j < C; ++j) {
      if constexpr (CC) v[j] = j < clen ? row[cstart + j] : T(0);
      else v[j] = (EXACT || base + j < rd.n) ? row[base + j] : T(0);
      lo[j] = T(0);
    }
    const T r = T(rd.r), h = T(0.5 * rd.r), s = T(rd.s);
    constexpr int M = EXACT ? MODE_EXACT : MODE_RAGGED;
    if constexpr (CC && INTEG == INTEG_RK4) {
      (void)h;
      if (rd.bc == BC_PERIODIC)
        rk4_steps_x2_cc<NT, C, BC_PERIODIC>(v, lo, rd.nsteps, r, s, tl, shrt, sh_last, sh_first,
                                            sh_wrap);
      else
        rk4_steps_x2_cc<NT, C, BC_DIRICHLET>(v, lo, rd.nsteps, r, s, tl, shrt, sh_last, sh_first,
                                             sh_wrap);
    } else if constexpr (CC) {
      (void)h;
      if (rd.bc == BC_PERIODIC)
        explicit_steps_split_x2_cc<NT, C, BC_PERIODIC>(v, lo, rd.nsteps, r, s, tl, shrt, sh_last,
                                                       sh_first, sh_wrap);
      else
        explicit_steps_split_x2_cc<NT, C, BC_DIRICHLET>(v, lo, rd.nsteps, r, s, tl, shrt, sh_last,
                                                        sh_first, sh_wrap);
    } else if (rd.bc == BC_PERIODIC) {
      explicit_steps<T, NT, C, M, BC_PERIODIC, INTEG>(v, lo, rd.nsteps, r, h, s, rd.n, base,
                                                      sh_last, sh_first, sh_wrap);
    } else {
      explicit_steps<T, NT, C, M, BC_DIRICHLET, INTEG>(v, lo, rd.nsteps, r, h, s, rd.n, base,
                                                       sh_last, sh_first, sh_wrap);
    }
#pragma unroll
    for (int j = 0; j < C; ++j) {
      if constexpr (CC) {
        if (j < clen) row[cstart + j] = v[j];
      } else if (EXACT || base + j < rd.n) {
        row[base + j] = v[j];
      }
    }
    __syncthreads();
  }
}

template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
  using type = float4;
  static constexpr int width = 4;
};
template <>
struct Vec2<double> {
  using type = double2;
  static constexpr int width = 2;
};

template <typename T, int C>
__device__ __forceinline__ void load_vec(T (&v)[C], const T* p) {
  using V = typename Vec2<T>::type;
  constexpr int Wd = Vec2<T>::width;
  static_assert(C % Wd == 0, "C must be a multiple of the vector width");
#pragma unroll
  for (int q = 0; q < C / Wd; ++q) {
    V x = __ldg(reinterpret_cast<const V*>(p) + q);
    if constexpr (Wd == 4) {
      v[4 * q + 0] = x.x; v[4 * q + 1] = x.y; v[4 * q + 2] = x.z; v[4 * q + 3] = x.w;
    } else {
      v[2 * q + 0] = x.x; v[2 * q + 1] = x.y;
    }
  }
}

__device__ __forceinline__ int skew32(int i) { return i + (i >> 5); }

// 16-byte asynchronous copy global -> shared (cp.async); each thread waits
// for its own copies with cp.async.wait_group, which needs no spin loop.
__device__ __forceinline__ void stream_cp16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(
                   static_cast<unsigned>(__cvta_generic_to_shared(smem))),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void stream_cp_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void stream_cp_wait() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// FP32 RK4 windows of 16 or more nodes a thread prefetch the CTA's next
// window (below): the RK4 window kernel holds one 256-thread CTA per SM (its
// registers), so a window's load latency is not covered by another CTA's
// steps (6% faster with the prefetch on 2^22-node rows); the forward-Euler
// kernel runs two CTAs per SM and was 1-2% slower with it. Dynamic shared
// memory of the streaming kernel: the output stage (values and, FP32,
// compensation bytes), then the two prefetch buffers of W values and W bytes.
template <typename T, int NT, int C, int INTEG>
constexpr bool stream_prefetch() {
  return sizeof(T) == 4 && C % 16 == 0 && INTEG == INTEG_RK4;
}
template <typename T, int NT, int C, int INTEG>
constexpr size_t stream_dsm() {
  constexpr size_t WS = size_t(NT) * C + size_t(NT) * C / 32;
  constexpr size_t stage = (sizeof(T) + (Kahan<T>::on ? 1 : 0)) * WS;
  return stream_prefetch<T, NT, C, INTEG>() ? ((stage + 15) & ~size_t(15)) + 10 * size_t(NT) * C
                                            : stage;
}

// Streaming window kernel. Pass `step_base` advances every row by
// min(K, nsteps - step_base) steps from src into dst (rows already done are
// copied through, so src/dst stay consistent for the ping-pong). FP32 passes
// carry the Kahan compensation term through lo_src / lo_dst, one byte per node
// in the rows' layout (lo8_encode); FP64 passes get null pointers. Results
// leave through a skewed shared-memory stage so the stores of the W - 2K
// output nodes are coalesced. FP32 RK4 windows of 16 or more nodes a thread: while
// a window runs its K steps, each thread copies its own chunk of the CTA's
// next window (state and compensation bytes) into one of two shared-memory
// buffers with cp.async, so the window's HBM latency is off the CTA's path
// (windows inside their row whose state and bytes start 16-byte aligned --
// the same test for every thread, each chunk starting at a multiple of 16
// nodes; other windows load directly). The buffer a copy fills was last read
// one window earlier, by the same thread.
template <typename T, int NT, int C, int INTEG = INTEG_EULER>
__global__ void __launch_bounds__(NT) k_explicit_stream(const T* __restrict__ src,
                                                        T* __restrict__ dst,
                                                        const signed char* __restrict__ lo_src,
                                                        signed char* __restrict__ lo_dst,
                                                        const RowDesc* __restrict__ rows,
                                                        const TileItem* __restrict__ items,
                                                        int nitems, int K, int64_t step_base) {
  constexpr int NW = NT / 32;
  constexpr int W = NT * C;
  constexpr int WS = W + W / 32;
  extern __shared__ __align__(16) unsigned char dsm[];
  T* stage = reinterpret_cast<T*>(dsm);                                  // WS values
  signed char* stage_lo = reinterpret_cast<signed char*>(stage + WS);   // WS bytes (FP32 only)
  constexpr bool PREF = stream_prefetch<T, NT, C, INTEG>();
  constexpr size_t PREF_OFF = ((sizeof(T) + (Kahan<T>::on ? 1 : 0)) * size_t(WS) + 15) & ~size_t(15);
  float* pv = reinterpret_cast<float*>(dsm + PREF_OFF);                 // [2][W] values
  signed char* plo = reinterpret_cast<signed char*>(pv + 2 * W);        // [2][W] bytes
  __shared__ T sh_last[2 * NW], sh_first[2 * NW], sh_wrap[4];
  // each step (each RK4 stage) makes one more node per side stale
  const int H = K * (INTEG == INTEG_RK4 ? 4 : 1);
  const int O = W - 2 * H;
  const int base = threadIdx.x * C;
  // copies this thread's chunk of item `it`'s window into buffer `buf`;
  // false (nothing copied) for windows this kernel loads directly
  auto prefetch = [&](int it, int buf) -> bool {
    if constexpr (!PREF) {
      (void)it;
      (void)buf;
      return false;
    } else {
      if (it >= nitems) return false;
      const TileItem ti = items[it];
      const RowDesc rd = rows[ti.row];
      const int64_t ws = int64_t(ti.tile) * O - H;
      if (rd.nsteps - step_base <= 0 || ws < 0 || ws + W > rd.n) return false;
      const T* sp = src + rd.offset + ws;
      const signed char* lp = lo_src + rd.offset + ws;
      if (((reinterpret_cast<uintptr_t>(sp) | reinterpret_cast<uintptr_t>(lp)) & 15) != 0)
        return false;
      float* dv = pv + buf * W + base;
      signed char* dl = plo + buf * W + base;
#pragma unroll
      for (int q = 0; q < C / 4; ++q) stream_cp16(dv + 4 * q, sp + base + 4 * q);
#pragma unroll
      for (int q = 0; q < C / 16; ++q) stream_cp16(dl + 16 * q, lp + base + 16 * q);
      stream_cp_commit();
      return true;
    }
  };
  int buf = 0;
  bool pre = prefetch(int(blockIdx.x), 0);
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const bool have = pre;  // this window is in buffer `cur`
    const int cur = buf;
    const TileItem ti = items[it];
    const RowDesc rd = rows[ti.row];
    const int64_t n = rd.n;
    const int64_t out_lo = int64_t(ti.tile) * O;
    const int64_t out_hi = min(out_lo + O, n);
    const int64_t ws = out_lo - H;
    const int64_t rem = rd.nsteps - step_base;
    const int kk = rem <= 0 ? 0 : (rem < K ? int(rem) : K);
    const T* srow = src + rd.offset;
    T* drow = dst + rd.offset;
    if (kk == 0) {
      for (int64_t g = out_lo + threadIdx.x; g < out_hi; g += NT) {
        drow[g] = srow[g];
        if constexpr (Kahan<T>::on) lo_dst[rd.offset + g] = lo_src[rd.offset + g];
      }
      buf ^= 1;
      pre = prefetch(it + int(gridDim.x), buf);
      continue;
    }
    T v[C], lo[C];
    const int64_t g0 = ws + base;
    const bool interior = ws >= 0 && ws + W <= n;
    const bool aligned = (reinterpret_cast<uintptr_t>(srow + ws) & 15) == 0;
    bool loaded = false;
    if constexpr (PREF) {
      if (have) {  // the same decode as the aligned global path below
        stream_cp_wait();
        const float4* sv = reinterpret_cast<const float4*>(pv + cur * W + base);
        const uint4* sb = reinterpret_cast<const uint4*>(plo + cur * W + base);
#pragma unroll
        for (int q = 0; q < C / 4; ++q) {
          const float4 x = sv[q];
          v[4 * q + 0] = x.x; v[4 * q + 1] = x.y; v[4 * q + 2] = x.z; v[4 * q + 3] = x.w;
        }
#pragma unroll
        for (int k = 0; k < C / 16; ++k) {
          const uint4 w = sb[k];
          const unsigned ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
          for (int e = 0; e < 16; ++e)
            lo[16 * k + e] = lo8_decode(v[16 * k + e],
                                        static_cast<signed char>(ww[e >> 2] >> (8 * (e & 3))));
        }
        loaded = true;
      }
    }
    if (!loaded) {
    if (interior && aligned && (C % Vec2<T>::width == 0)) {
      load_vec<T, C>(v, srow + g0);
    } else {
#pragma unroll
      for (int j = 0; j < C; ++j) {
        int64_t gi = g0 + j;
        if (rd.bc == BC_PERIODIC) {
          gi %= n;
          if (gi < 0) gi += n;
        } else {
          gi = gi < 0 ? 0 : (gi >= n ? n - 1 : gi);
        }
        v[j] = srow[gi];
      }
    }
#pragma unroll
    for (int j = 0; j < C; ++j) lo[j] = T(0);
    if constexpr (Kahan<T>::on) {
      // one byte per node: 16-byte words inside the row where aligned, else per
      // node (the window's halo wraps or clamps)
      const signed char* lp = lo_src + rd.offset + g0;
      if (C % 16 == 0 && interior && (reinterpret_cast<uintptr_t>(lp) & 15) == 0) {
#pragma unroll
        for (int k = 0; k < C / 16; ++k) {
          const uint4 w = __ldg(reinterpret_cast<const uint4*>(lp) + k);
          const unsigned ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
          for (int e = 0; e < 16; ++e)
            lo[16 * k + e] = lo8_decode(v[16 * k + e],
                                        static_cast<signed char>(ww[e >> 2] >> (8 * (e & 3))));
        }
      } else {
#pragma unroll
        for (int j = 0; j < C; ++j) {
          int64_t gi = g0 + j;
          if (!interior) {
            if (rd.bc == BC_PERIODIC) {
              gi %= n;
              if (gi < 0) gi += n;
            } else {
              gi = gi < 0 ? 0 : (gi >= n ? n - 1 : gi);
            }
          }
          lo[j] = lo8_decode(v[j], __ldg(lo_src + rd.offset + gi));
        }
      }
    }
    }  // direct loads
    // the next window's copies go to the other buffer
    buf ^= 1;
    pre = prefetch(it + int(gridDim.x), buf);
    const RowCoefs<T> cf = row_coefs(rd, T(0));
    const bool has_end = rd.bc == BC_DIRICHLET && ((ws <= 0 && ws + W > 0) ||
                                                   (ws <= n - 1 && ws + W > n - 1));
    if (has_end)
      explicit_steps<T, NT, C, MODE_WINDOW_DIR, BC_DIRICHLET, INTEG>(v, lo, kk, cf.r, cf.h, cf.s,
                                                                     int(n), g0, sh_last, sh_first,
                                                                     sh_wrap);
    else
      explicit_steps<T, NT, C, MODE_WINDOW, BC_PERIODIC, INTEG>(v, lo, kk, cf.r, cf.h, cf.s,
                                                                int(n), g0, sh_last, sh_first,
                                                                sh_wrap);
#pragma unroll
    for (int j = 0; j < C; ++j) stage[skew32(base + j)] = v[j];
    if constexpr (Kahan<T>::on) {
      // bytes unskewed: each thread stores its C bytes as whole words (the
      // stage starts 16-byte aligned and base is a multiple of C)
      if constexpr (C % 4 == 0) {
#pragma unroll
        for (int k = 0; k < C / 4; ++k)
          reinterpret_cast<unsigned*>(stage_lo + base)[k] =
              pack4(lo8_encode(v[4 * k], lo[4 * k]), lo8_encode(v[4 * k + 1], lo[4 * k + 1]),
                    lo8_encode(v[4 * k + 2], lo[4 * k + 2]), lo8_encode(v[4 * k + 3], lo[4 * k + 3]));
      } else {
#pragma unroll
        for (int j = 0; j < C; ++j) stage_lo[base + j] = lo8_encode(v[j], lo[j]);
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < O; i += NT) {
      const int64_t gi = out_lo + i;
      if (gi < out_hi) {
        drow[gi] = stage[skew32(H + i)];
        if constexpr (Kahan<T>::on) lo_dst[rd.offset + gi] = stage_lo[H + i];
      }
    }
    __syncthreads();
  }
}

// One step per HBM pass (streaming with K = 1): the bandwidth-bound form of
// the explicit step, one tile of NT*C nodes per item (step1_tile, step1.cuh).
// Same arguments as k_explicit_stream (K is 1 here). Handles any tile; the
// bulk-copy kernel k_explicit_step1_bulk takes the full tiles of aligned rows.
template <typename T, int NT, int C>
__global__ void __launch_bounds__(NT) k_explicit_step1(const T* __restrict__ src,
                                                       T* __restrict__ dst,
                                                       const signed char* __restrict__ lo_src,
                                                       signed char* __restrict__ lo_dst,
                                                       const RowDesc* __restrict__ rows,
                                                       const TileItem* __restrict__ items,
                                                       int nitems, int K, int64_t step_base) {
  (void)K;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x)
    step1_tile<T, NT, C>(src, dst, lo_src, lo_dst, rows, items[it], step_base);
}

#define REG_RES(T, DT, NT, C)                                                               \
  reg.push_back({K_EXPLICIT_RESIDENT, DT, NT, C, 1,                                         \
                 reinterpret_cast<const void*>(&k_explicit_resident<T, NT, C, true>), 0});  \
  reg.push_back({K_EXPLICIT_RESIDENT, DT, NT, C, 0,                                         \
                 reinterpret_cast<const void*>(&k_explicit_resident<T, NT, C, false>), 0});
#define REG_RK4(T, DT, NT, C)                                                               \
  reg.push_back({K_RK4_RESIDENT, DT, NT, C, 1,                                              \
                 reinterpret_cast<const void*>(                                             \
                     &k_explicit_resident<T, NT, C, true, INTEG_RK4>),                      \
                 0});                                                                       \
  reg.push_back({K_RK4_RESIDENT, DT, NT, C, 0,                                              \
                 reinterpret_cast<const void*>(                                             \
                     &k_explicit_resident<T, NT, C, false, INTEG_RK4>),                     \
                 0});
#define REG_RK4_STREAM(T, DT, NT, C)                                                        \
  reg.push_back({K_RK4_STREAM, DT, NT, C, 0,                                               \
                 reinterpret_cast<const void*>(&k_explicit_stream<T, NT, C, INTEG_RK4>),  \
                 stream_dsm<T, NT, C, INTEG_RK4>()});
#define REG_STREAM(T, DT, NT, C)                                                            \
  reg.push_back({K_EXPLICIT_STREAM, DT, NT, C, 0,                                          \
                 reinterpret_cast<const void*>(&k_explicit_stream<T, NT, C>),             \
                 stream_dsm<T, NT, C, INTEG_EULER>()});

void register_explicit(std::vector<KernelEntry>& reg) {
  // FP32 resident shapes (capacity NT*C nodes)
  REG_RES(float, 0, 32, 1) REG_RES(float, 0, 32, 2) REG_RES(float, 0, 32, 4)
  REG_RES(float, 0, 32, 8) REG_RES(float, 0, 64, 8) REG_RES(float, 0, 128, 8)
  REG_RES(float, 0, 64, 16) REG_RES(float, 0, 128, 16) REG_RES(float, 0, 256, 8)
  REG_RES(float, 0, 256, 16) REG_RES(float, 0, 128, 32) REG_RES(float, 0, 512, 8)
  REG_RES(float, 0, 512, 16) REG_RES(float, 0, 256, 32) REG_RES(float, 0, 1024, 16)
  REG_RES(float, 0, 1024, 32)
  // FP64 resident shapes
  REG_RES(double, 1, 32, 1) REG_RES(double, 1, 32, 2) REG_RES(double, 1, 32, 4)
  REG_RES(double, 1, 32, 8) REG_RES(double, 1, 64, 8) REG_RES(double, 1, 128, 8)
  REG_RES(double, 1, 256, 8) REG_RES(double, 1, 128, 16) REG_RES(double, 1, 512, 8)
  REG_RES(double, 1, 256, 16) REG_RES(double, 1, 1024, 8) REG_RES(double, 1, 512, 16)
  // streaming window shapes
  REG_STREAM(float, 0, 32, 4) REG_STREAM(float, 0, 128, 16) REG_STREAM(float, 0, 256, 16)
  REG_STREAM(float, 0, 512, 16) REG_STREAM(float, 0, 256, 32)
  REG_STREAM(double, 1, 32, 4) REG_STREAM(double, 1, 128, 8) REG_STREAM(double, 1, 256, 8)
  REG_STREAM(double, 1, 256, 16)
  // RK4 (Eq. 22): resident and streaming shapes
  REG_RK4(float, 0, 32, 1) REG_RK4(float, 0, 32, 2) REG_RK4(float, 0, 32, 4)
  REG_RK4(float, 0, 32, 8) REG_RK4(float, 0, 64, 8) REG_RK4(float, 0, 128, 8)
  REG_RK4(float, 0, 64, 16) REG_RK4(float, 0, 128, 16) REG_RK4(float, 0, 256, 8)
  REG_RK4(float, 0, 256, 16) REG_RK4(float, 0, 512, 8) REG_RK4(float, 0, 512, 16)
  REG_RK4(double, 1, 32, 1) REG_RK4(double, 1, 32, 2) REG_RK4(double, 1, 32, 4)
  REG_RK4(double, 1, 32, 8) REG_RK4(double, 1, 64, 8) REG_RK4(double, 1, 128, 8)
  REG_RK4(double, 1, 256, 8) REG_RK4(double, 1, 512, 8) REG_RK4(double, 1, 128, 4)
  REG_RK4(double, 1, 256, 4) REG_RK4(double, 1, 512, 4) REG_RK4(double, 1, 1024, 4)
  REG_RK4_STREAM(float, 0, 32, 4) REG_RK4_STREAM(float, 0, 128, 16)
  REG_RK4_STREAM(float, 0, 256, 16)
  REG_RK4_STREAM(double, 1, 32, 4) REG_RK4_STREAM(double, 1, 128, 8)
  REG_RK4_STREAM(double, 1, 256, 8)
  // one step per pass
  reg.push_back({K_EXPLICIT_STEP1, 0, 256, 8, 0,
                 reinterpret_cast<const void*>(&k_explicit_step1<float, 256, 8>), 0});
  reg.push_back({K_EXPLICIT_STEP1, 0, 256, 16, 0,
                 reinterpret_cast<const void*>(&k_explicit_step1<float, 256, 16>), 0});
  reg.push_back({K_EXPLICIT_STEP1, 0, 128, 16, 0,
                 reinterpret_cast<const void*>(&k_explicit_step1<float, 128, 16>), 0});
  reg.push_back({K_EXPLICIT_STEP1, 0, 512, 8, 0,
                 reinterpret_cast<const void*>(&k_explicit_step1<float, 512, 8>), 0});
  reg.push_back({K_EXPLICIT_STEP1, 1, 256, 8, 0,
                 reinterpret_cast<const void*>(&k_explicit_step1<double, 256, 8>), 0});
  reg.push_back({K_EXPLICIT_STEP1, 1, 256, 4, 0,
                 reinterpret_cast<const void*>(&k_explicit_step1<double, 256, 4>), 0});
}

}  // namespace burgers
