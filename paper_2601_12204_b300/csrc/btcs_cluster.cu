// btcs_cluster.cu -- lagged upwind BTCS (Sec. 2.4, Eq. 23), and the
// Crank-Nicolson, Picard and Newton variants of tridiagonal rows, for rows
// too long for one CTA but short enough for a thread-block cluster: the row
// stays in the shared memory of CS CTAs for all of its steps, as in the
// resident kernel.
//
// Three levels of the same partitioned elimination:
//   chunk   each thread eliminates its C (or C - 1) rows (as two half-chunks
//           on packed f32x2 pairs, as btcs_x2.cuh does) and leaves one
//           reduced row per chunk in its unknown X_t (the chunk-end value);
//   block   one warp of each CTA expresses the reduced unknowns of its chunks
//           0..ti-1 through the value P before the block (the previous CTA's
//           interface) and its own interface Y = X_ti (ti = its last chunk):
//               X_t = y_t - alpha_t P - gamma_t Y,
//           by solving its block with three right-hand sides at once;
//   cluster substituting those relations into the interface rows leaves one
//           row per CTA in Y_{k-1}, Y_k, Y_{k+1} (cyclic when periodic), which
//           one warp of every CTA solves, one row per lane (Sherman-Morrison
//           correction with its denominator in extended precision).
// Every CTA pushes its contribution to the cluster system into the shared
// memory of every CTA of the cluster (slots double-buffered by step parity,
// written through distributed shared memory before the barrier, so no remote
// read sits on the critical path); after one cluster barrier the last warp of
// each CTA solves the same small system from its own copies with the same
// arithmetic, keeping its own Y and P and the new values
// of the nodes next to its ends (computed with the owners' arithmetic from
// their operands), so the neighbour values of the next step need no further
// exchange. A step costs one cluster barrier and four CTA barriers.
// Increment form and Kahan-compensated FP32 state as in btcs.cu.
#include <cooperative_groups.h>

#include "btcs_common.cuh"
#include "btcs_kernel.cuh"
#include "common.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace burgers {

// What each CTA contributes to the cluster system (read by every CTA of the
// cluster). Aligned and padded to 16 bytes, so that a remote read is a few
// vector loads.
template <typename T>
struct alignas(16) ClusterSlot {
  T eah, ech, edh;      // end relation of the interface chunk
  T rd0, ra0, rg0;      // first-row relation of chunk 0
  T yl, al, gl;         // block relation of chunk ti - 1 (when ti > 0)
  T y0, a0, g0;         // block relation of chunk 0 (when ti > 0)
  T uf, lf;             // state (and Kahan term) of the CTA's first node
  T ul, ll;             // ... of its last node (end of chunk ti)
  T ef, el;             // Picard, Newton: the iterate's offset e of those two nodes
  int ti;               // interface chunk
  int jf;               // end row of chunk 0 (0: chunk 0 is a single node)
};

// Copies a slot from (distributed) shared memory in 16-byte pieces.
template <typename T>
__device__ __forceinline__ ClusterSlot<T> load_slot(const ClusterSlot<T>* p) {
  static_assert(sizeof(ClusterSlot<T>) % 16 == 0, "slot size must be a multiple of 16 bytes");
  union {
    ClusterSlot<T> s;
    float4 v[sizeof(ClusterSlot<T>) / 16];
  } u;
  const float4* src = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int i = 0; i < int(sizeof(ClusterSlot<T>) / 16); ++i) u.v[i] = src[i];
  return u.s;
}

// Stores a slot into (distributed) shared memory in 16-byte pieces.
template <typename T>
__device__ __forceinline__ void store_slot(ClusterSlot<T>* p, const ClusterSlot<T>& s) {
  union {
    ClusterSlot<T> s;
    float4 v[sizeof(ClusterSlot<T>) / 16];
  } u;
  u.s = s;
  float4* dst = reinterpret_cast<float4*>(p);
#pragma unroll
  for (int i = 0; i < int(sizeof(ClusterSlot<T>) / 16); ++i) dst[i] = u.v[i];
}

// What the cluster solve leaves for its CTA.
template <typename T>
struct ClusterReply {
  T Y, P;               // own interface value and the one before the block
  T halo_l, halo_r;     // new values of the nodes before the first / after the last
};

template <typename T, int NT>
struct ClusterShared {
  BtcsShared<T, NT> sm;
  T V[NT + NT / 32];    // block right-hand side of the interface coupling
  T Wg[NT + NT / 32];   // ... and its solution (gamma)
  T hfirst[NT], hlast[NT];
  T iface[3];                   // end relation of the interface chunk tl
  ClusterSlot<T> slots[2][16];  // [step parity][contributing CTA] (clusters up to 16)
  ClusterReply<T> reply;
};

// Block solve of one warp: rows 0..NT-1 of sm (identity beyond the block) with
// right-hand sides D, U and V; leaves the solutions in X, Z and Wg. Same
// elimination as reduced_solve (per-lane rows, then cyclic reduction over
// the 32 lanes), non-cyclic, three right-hand sides.
template <typename T, int NT>
__device__ __forceinline__ void block_solve3(ClusterShared<T, NT>& cs, int lane) {
  constexpr int Q = NT / 32;
  BtcsShared<T, NT>& sm = cs.sm;
  const int r0 = lane * Q;
  // up to 4 rows a lane keep the sweeps' results in registers
  constexpr bool REGQ = Q <= 4;
  constexpr int QR = REGQ ? Q : 1;
  T rc[QR], ra[QR], rd[QR], ru[QR], rv[QR];
  T chp = T(0), ahp = T(-1), dhp = T(0), uhp = T(0), vhp = T(0);
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int i = sk(r0 + q);
    const T a = sm.A[i], b = sm.B[i], c = sm.Cc[i];
    const T inv = recip(tfma(-a, chp, b));
    const T ai = a * inv;
    chp = c * inv;
    ahp = -ai * ahp;
    dhp = tfma(-ai, dhp, sm.D[i] * inv);
    uhp = tfma(-ai, uhp, sm.U[i] * inv);
    vhp = tfma(-ai, vhp, cs.V[i] * inv);
    if constexpr (REGQ) {
      rc[q] = chp; ra[q] = ahp; rd[q] = dhp; ru[q] = uhp; rv[q] = vhp;
    } else {
      sm.Cc[i] = chp;
      sm.A[i] = ahp;
      sm.D[i] = dhp;
      sm.U[i] = uhp;
      cs.V[i] = vhp;
    }
  }
  const T e_ch = chp, e_ah = ahp, e_dh = dhp, e_uh = uhp, e_vh = vhp;
  T cd = T(0), ca = T(0), cg_ = T(-1), cu = T(0), cv = T(0);
#pragma unroll
  for (int q = Q - 2; q >= 0; --q) {
    const int i = sk(r0 + q);
    if constexpr (REGQ) {
      const T ch = rc[q];
      cd = tfma(-ch, cd, rd[q]);
      ca = tfma(-ch, ca, ra[q]);
      cg_ = -ch * cg_;
      cu = tfma(-ch, cu, ru[q]);
      cv = tfma(-ch, cv, rv[q]);
      rd[q] = cd; ra[q] = ca; rc[q] = cg_; ru[q] = cu; rv[q] = cv;
    } else {
      const T ch = sm.Cc[i];
      cd = tfma(-ch, cd, sm.D[i]);
      ca = tfma(-ch, ca, sm.A[i]);
      cg_ = -ch * cg_;
      cu = tfma(-ch, cu, sm.U[i]);
      cv = tfma(-ch, cv, cs.V[i]);
      sm.D[i] = cd;
      sm.A[i] = ca;
      sm.Cc[i] = cg_;
      sm.U[i] = cu;
      cs.V[i] = cv;
    }
  }
  T nd = shfl_down(cd, 1), na = shfl_down(ca, 1), ng = shfl_down(cg_, 1);
  T nu = shfl_down(cu, 1), nv = shfl_down(cv, 1);
  if (lane == 31) { nd = T(0); na = T(0); ng = T(0); nu = T(0); nv = T(0); }
  T a32 = e_ah, b32 = T(1) - e_ch * na, c32 = -e_ch * ng;
  T d32 = tfma(-e_ch, nd, e_dh), u32 = tfma(-e_ch, nu, e_uh), v32 = tfma(-e_ch, nv, e_vh);
  {
    const T inv = recip(b32);
    a32 *= inv; c32 *= inv; d32 *= inv; u32 *= inv; v32 *= inv;
  }
#pragma unroll
  for (int k = 1; k < 32; k <<= 1) {
    T am = shfl_up(a32, k), cm = shfl_up(c32, k), dm = shfl_up(d32, k);
    T um = shfl_up(u32, k), vm = shfl_up(v32, k);
    T ap = shfl_down(a32, k), cp = shfl_down(c32, k), dp = shfl_down(d32, k);
    T up = shfl_down(u32, k), vp = shfl_down(v32, k);
    if (lane < k) { am = T(0); cm = T(0); dm = T(0); um = T(0); vm = T(0); }
    if (lane + k > 31) { ap = T(0); cp = T(0); dp = T(0); up = T(0); vp = T(0); }
    const T inv = recip(T(1) - a32 * cm - c32 * ap);
    const T na2 = -a32 * am * inv, nc2 = -c32 * cp * inv;
    d32 = (d32 - a32 * dm - c32 * dp) * inv;
    u32 = (u32 - a32 * um - c32 * up) * inv;
    v32 = (v32 - a32 * vm - c32 * vp) * inv;
    a32 = na2;
    c32 = nc2;
  }
  T YL = shfl_up(d32, 1), UL = shfl_up(u32, 1), VL = shfl_up(v32, 1);
  if (lane == 0) { YL = T(0); UL = T(0); VL = T(0); }
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int i = sk(r0 + q);
    T y = d32, z = u32, w = v32;
    if (q < Q - 1) {
      if constexpr (REGQ) {
        y = tfma(-rc[q], d32, tfma(-ra[q], YL, rd[q]));
        z = tfma(-rc[q], u32, tfma(-ra[q], UL, ru[q]));
        w = tfma(-rc[q], v32, tfma(-ra[q], VL, rv[q]));
      } else {
        y = tfma(-sm.Cc[i], d32, tfma(-sm.A[i], YL, sm.D[i]));
        z = tfma(-sm.Cc[i], u32, tfma(-sm.A[i], UL, sm.U[i]));
        w = tfma(-sm.Cc[i], v32, tfma(-sm.A[i], VL, cs.V[i]));
      }
    }
    sm.X[i] = y;
    sm.Z[i] = z;
    cs.Wg[i] = w;
  }
}

// One warp of every CTA: the cluster system in the interface values Y_k, one
// row per lane (lanes >= CS carry identity rows), from the contributions in
// slots[par], solved by cyclic reduction over the lanes; the cyclic corners
// are split off by Sherman-Morrison with the correction factor's denominator
// in extended precision (sm_factor, as in the CTA-level solve). Every CTA solves the same
// system with the same arithmetic and keeps, for itself (rank), its Y and P
// and the new values of the nodes next to its ends. Dirichlet rows have
// identity rows at the row's ends, so the first block has no left neighbour
// (P = 0) and the system is plain.
// mode 0: the step's new values u + delta (compensated); Picard and Newton iterations:
// 1 the next iterate's u + (e + delta), 2 (the last) u + (e + delta)
// compensated -- each the owner's arithmetic for its nodes.
template <typename T, int NT, int CS>
__device__ __forceinline__ void cluster_solve(ClusterShared<T, NT>& cs, bool per, int lane,
                                              int rank, int par, cg::cluster_group& cluster,
                                              int mode = 0) {
  const bool on = lane < CS;
  const int k = on ? lane : 0;
  // lane k reads CTA k's contribution (pushed into this CTA's memory before
  // the barrier), and the fields of CTA k + 1's that its row needs from lane
  // k + 1
  (void)cluster;
  const ClusterSlot<T> s = load_slot(&cs.slots[par][k]);
  struct {
    T ra0, rg0, rd0, a0, g0, y0;
    int ti;
  } sn;
  {
    const int kn = (k + 1) % CS;
    sn.ra0 = shfl(s.ra0, kn); sn.rg0 = shfl(s.rg0, kn); sn.rd0 = shfl(s.rd0, kn);
    sn.a0 = shfl(s.a0, kn); sn.g0 = shfl(s.g0, kn); sn.y0 = shfl(s.y0, kn);
    sn.ti = __shfl_sync(FULL_MASK, s.ti, kn);
  }
  T a = T(0), b = T(1), c = T(0), d = T(0), uu = T(0);
  if (on) {
    const T A = s.eah, B = T(1) - s.ech * sn.ra0, C = -s.ech * sn.rg0;
    const T D = tfma(-s.ech, sn.rd0, s.edh);
    T pa = A, pb = T(0), pd = T(0);
    if (s.ti > 0) { pa = -A * s.al; pb = -A * s.gl; pd = A * s.yl; }
    T qa = T(0), qb = C, qd = T(0);
    if (sn.ti > 0) { qa = -C * sn.a0; qb = -C * sn.g0; qd = C * sn.y0; }
    a = pa;
    b = B + pb + qa;
    c = qb;
    d = D - pd - qd;
  }
  // Sherman-Morrison split of the corners: gamma = -b_0, fa = a_0 / gamma
  T fa = T(0);
  if (per) {
    const T gam = -shfl(b, 0);
    fa = shfl(a, 0) * recip(gam);
    const T cl = shfl(c, CS - 1);
    if (lane == 0) { b -= gam; uu = gam; }
    if (lane == CS - 1) { b -= cl * fa; uu = cl; }
  }
  if (lane == 0) a = T(0);
  if (lane >= CS - 1) c = T(0);
  // cyclic reduction over the lanes (rows normalised to a unit diagonal)
  {
    const T inv = recip(b);
    a *= inv; c *= inv; d *= inv; uu *= inv;
  }
  // rows beyond CS are decoupled identities: log2(CS) levels decouple the rest
#pragma unroll
  for (int st = 1; st < CS; st <<= 1) {
    T am = shfl_up(a, st), cm = shfl_up(c, st), dm = shfl_up(d, st), um = shfl_up(uu, st);
    T ap = shfl_down(a, st), cp = shfl_down(c, st), dp = shfl_down(d, st), up = shfl_down(uu, st);
    if (lane < st) { am = T(0); cm = T(0); dm = T(0); um = T(0); }
    if (lane + st > 31) { ap = T(0); cp = T(0); dp = T(0); up = T(0); }
    const T inv = recip(T(1) - a * cm - c * ap);
    const T na = -a * am * inv, nc = -c * cp * inv;
    d = (d - a * dm - c * dp) * inv;
    uu = (uu - a * um - c * up) * inv;
    a = na;
    c = nc;
  }
  T Y = d;
  if (per) {
    const T fac = sm_factor(fa, shfl(d, 0), shfl(d, CS - 1), shfl(uu, 0), shfl(uu, CS - 1));
    Y = tfma(-fac, uu, d);
  }
  // P of block k is the interface before it; new first / last node values
  T P = shfl(Y, (lane + CS - 1) % CS);
  if (!per && lane == 0) P = T(0);
  T first = T(0), last = T(0);
  if (on) {
    const T X0 = s.ti > 0 ? tfma(-s.g0, Y, tfma(-s.a0, P, s.y0)) : Y;
    const T d0 = s.jf == 0 ? X0 : tfma(-s.rg0, X0, tfma(-s.ra0, P, s.rd0));
    T lf = s.lf, ll = s.ll;
    if (mode == 0) {
      first = comp_add(s.uf, d0, lf);
      last = comp_add(s.ul, Y, ll);
    } else if (mode == 1) {
      first = s.uf + (s.ef + d0);
      last = s.ul + (s.el + Y);
    } else {
      first = comp_add(s.uf, s.ef + d0, lf);
      last = comp_add(s.ul, s.el + Y, ll);
    }
  }
  const T last_prev = shfl(last, (lane + CS - 1) % CS);
  const T first_next = shfl(first, (lane + 1) % CS);
  const T myY = shfl(Y, rank), myP = shfl(P, rank);
  const T hl = shfl(last_prev, rank), hr = shfl(first_next, rank);
  if (lane == 0) {
    cs.reply.Y = myY;
    cs.reply.P = myP;
    cs.reply.halo_l = (rank > 0 || per) ? hl : T(0);
    cs.reply.halo_r = (rank + 1 < CS || per) ? hr : T(0);
  }
}

// One cluster per row (rows have (CS-1) W < n <= CS W, W = NT*C), FP32. The
// row's nodes are spread evenly over the CS CTAs, and each CTA's nk nodes over
// tk = ceil(nk / C) chunks of C or C - 1 nodes, the last bk = tk C - nk of
// them one node short; threads from tk on hold no nodes. Since nk > W/2 - 1,
// tk > NT/2 > C > bk, so every row length has such a split. A short chunk
// ends at a position known at compile time, so every warp runs the one sweep
// and a short chunk costs a few selects there (a chunk ending at an arbitrary
// node would need a select at every node, and the warp holding it would pace
// the CTA and, through the cluster barrier, every CTA of the row: 13-20%
// slower on ragged rows, measured).
//
// Each chunk is eliminated as two half-chunks on packed f32x2 pairs, as
// btcs_x2.cuh does for rows of one CTA (pair k holds nodes k and k + C/2 of
// the chunk; a chunk of C - 1 nodes ends its second half at pair C/2 - 2).
// Neighbour values are read directly (the edge values of the previous step,
// published before the barrier that ends it). Each thread folds its two
// halves into the relations of a one-piece chunk in its own end value
// X_t = X_B: with A's row X_A = pd - pa L - pc X_t,
//     first node  x_0 = (rd_A - rg_A pd) - (ra_A - rg_A pa) L + rg_A pc X_t,
//     end row     g x_e = (eB_d - eB_a pd) + eB_a pa L - eB_c x_next,
//                 g = 1 - eB_a pc,
// which the block rows, the block and cluster solves and the slots take. A
// chunk's first node is updated through its first-node relation, the
// arithmetic the cluster solve uses for a CTA's first node, so the halo
// values are bitwise the owners'. Increment form and Kahan-compensated FP32
// state as in btcs.cu.
template <int NT, int C, int CS, int VAR = VAR_BTCS>
__global__ void __cluster_dims__(CS, 1, 1)
__launch_bounds__(NT, NT <= 512 ? 512 / NT : 1)
    k_btcs_cluster_x2(float* __restrict__ u, const RowDesc* __restrict__ rows, int count,
                      int* __restrict__ counter) {
  (void)counter;
  constexpr int Q = NT / 32;
  constexpr int H = C / 2;
  static_assert(CS >= 2 && CS <= 16, "slots hold at most 16 CTAs");
  static_assert(C % 2 == 0 && C >= 4, "two half-chunks of at least two nodes");
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = int(cluster.block_rank());
  const int item = int(blockIdx.x) / CS;
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ ClusterShared<float, NT> cs;
  BtcsShared<float, NT>& sm = cs.sm;
  float2* us = reinterpret_cast<float2*>(dsm);  // H * NT pairs
  float2* lo = us + H * NT;                      // H * NT pairs
  float2* es = us + 2 * H * NT;                  // H * NT pairs (Picard, Newton: the iterate's e)
  constexpr bool ITER = VAR == VAR_PICARD || VAR == VAR_NEWTON;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool valid = item < count;  // grid is count * CS: always true
  const RowDesc rd = rows[valid ? item : 0];
  const int n = rd.n;
  const bool per = rd.bc == BC_PERIODIC;
  const bool lastcta = rank == CS - 1;
  const int nbase = n / CS, nrem = n % CS;
  const int nk = nbase + (rank < nrem ? 1 : 0);
  const int64_t kstart = int64_t(rank) * nbase + (rank < nrem ? rank : nrem);
  const int tk = (nk + C - 1) / C;
  const int bk = tk * C - nk;
  const int tl = tk - 1;
  const int ts = tk - bk;
  const bool active = tid < tk;
  const bool shrt = active && tid >= ts;
  const int cstart = tid * C - (shrt ? tid - ts : 0);
  const int clen = active ? (shrt ? C - 1 : C) : 0;
  float* row = u + rd.offset + kstart + cstart;
#pragma unroll
  for (int k = 0; k < H; ++k) {
    const float2 x = make_float2(k < clen ? row[k] : 0.f, k + H < clen ? row[k + H] : 0.f);
    us[k * NT + tid] = x;
    lo[k * NT + tid] = make_float2(0.f, 0.f);
    if (k == 0) cs.hfirst[tid] = x.x;
    if (k == H - 2 && shrt) cs.hlast[tid] = x.y;
    if (k == H - 1 && !shrt) cs.hlast[tid] = x.y;
  }
  __syncthreads();
  cluster.sync();  // every CTA of the cluster runs before any addresses another's memory
  if (tid == 0) {
    const int kl = rank > 0 ? rank - 1 : CS - 1, kr = rank + 1 < CS ? rank + 1 : 0;
    cluster.map_shared_rank(&cs.reply, kr)->halo_l = cs.hlast[tl];
    cluster.map_shared_rank(&cs.reply, kl)->halo_r = cs.hfirst[0];
  }
  cluster.sync();
  // matrix coefficients; Crank-Nicolson (VAR_CN): half of the step's r and s,
  // with the full step's explicit increment as right-hand side. Picard
  // (VAR_PICARD): `iters` solves a step, A(w) delta = Delta(w) - e with
  // w = u^n + e and e += delta (the rows of the current iterate w). Newton
  // (VAR_NEWTON, Eq. 10-14): `iters` solves J(w) delta = -F(w) of the
  // central-convection residual of Eq. 11, e += delta, with the Jacobian rows
  // l = -(r/2) w_i - s, d = 1 + (r/2)(w_{i+1} - w_{i-1}) + 2s,
  // c = (r/2) w_i - s (the operands and roundings of the resident kernel's
  // Newton rows)
  static_assert(VAR == VAR_BTCS || VAR == VAR_CN || VAR == VAR_PICARD || VAR == VAR_NEWTON,
                "lagged BTCS, Crank-Nicolson, Picard or Newton rows");
  const int nit = ITER ? rd.iters : 1;
  const float r = VAR == VAR_CN ? 0.5f * rd.rf : rd.rf, s = VAR == VAR_CN ? 0.5f * rd.sf : rd.sf;
  const float ds1 = 1.f + 2.f * s;
  const float2 R2 = make_float2(r, r), S2 = make_float2(s, s), DS1 = make_float2(ds1, ds1);
  const float hr = 0.5f * r;
  const float2 HR2 = make_float2(hr, hr), NS2 = make_float2(-s, -s);
  const bool dfirst = !per && rank == 0 && tid == 0;
  const bool dlast = !per && lastcta && tid == tl;
  const bool tlshort = bk > 0;
  float2 CH[H], AH[H], ND[H];  // forward: -ch, ah, -dh; backward: gamma, alpha, -delta
  int par = 0;
  for (int64_t step = 0; step < rd.nsteps; ++step) {
  if constexpr (ITER) {
#pragma unroll
    for (int k = 0; k < H; ++k) es[k * NT + tid] = make_float2(0.f, 0.f);
  }
  for (int it = 0; it < nit; ++it) {
    const bool lastit = it + 1 == nit;
    auto W = [&](int k) -> float2 {
      if constexpr (ITER) return add2(us[k * NT + tid], es[k * NT + tid]);
      else return us[k * NT + tid];
    };
    const float halo_l = cs.reply.halo_l, halo_r = cs.reply.halo_r;
    const float left = tid > 0 ? cs.hlast[tid - 1] : halo_l;
    const float right = tid < tl ? cs.hfirst[tid + 1] : halo_r;
    // ---- forward sweep of both halves (A's first row reads the left
    // neighbour, B's first row node C/2 - 1, A's end row node C/2, B's end
    // row the right neighbour), then the backward sweep
    float2 a = W(0);
    float2 ul = make_float2(left, W(H - 1).x);
    float2 DL = sub2(a, ul);  // a - u_l
    float2 chp = make_float2(0.f, 0.f), ahp = make_float2(-1.f, -1.f), ndhp = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < H; ++k) {
      float2 an = (k + 1 < H) ? W(k + 1) : make_float2(W(0).y, right);
      if (k == H - 2 && shrt) an.y = right;  // a short chunk's end row
      const float2 ER = sub2(an, a);         // u_r - a
      float2 nl, c, nc, d, nrhs;             // -l, c, -c, d, -rhs
      if constexpr (VAR == VAR_NEWTON) {
        const float2 ha = mul2(HR2, a);
        const float2 cdf = sub2(an, ul);  // w_{i+1} - w_{i-1}
        nl = add2(ha, S2);
        c = sub2(ha, S2);
        nc = sub2(S2, ha);
        d = fma2(HR2, cdf, DS1);
        // -rhs = F_i = e_i + (r/2) w_i (w_{i+1} - w_{i-1}) - s (w_{i+1} - 2 w_i + w_{i-1})
        nrhs = fma2(NS2, sub2(ER, DL), fma2(ha, cdf, es[k * NT + tid]));
      } else {
        const float2 ra = mul2(R2, a);
        const float2 M = make_float2(fmaxf(ra.x, 0.f), fmaxf(ra.y, 0.f));
        const float2 m = make_float2(fminf(ra.x, 0.f), fminf(ra.y, 0.f));
        nl = add2(S2, M);
        c = sub2(m, S2);
        nc = sub2(S2, m);
        d = add2(DS1, sub2(M, m));
        nrhs = fma2(nl, DL, mul2(c, ER));  // of the increment form
        if constexpr (VAR == VAR_CN) nrhs = mul2(make_float2(2.f, 2.f), nrhs);
        if constexpr (ITER) nrhs = add2(nrhs, es[k * NT + tid]);
      }
      if (k == 0 && dfirst) { nl.x = 0.f; c.x = 0.f; nc.x = 0.f; d.x = 1.f; nrhs.x = 0.f; }
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
    const float eAc = chp.x, eAa = ahp.x, eAd = -ndhp.x;
    float eBc = chp.y, eBa = ahp.y, eBd = -ndhp.y;
    if (shrt) { eBc = -CH[H - 2].y; eBa = AH[H - 2].y; eBd = -ND[H - 2].y; }
    if (dlast) { eBc = 0.f; eBa = 0.f; eBd = 0.f; }  // Dirichlet: an identity end row
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
        if (k == H - 2 && shrt) { ncd.y = 0.f; ca.y = 0.f; cg.y = -1.f; }
        ND[k] = ncd;
        AH[k] = ca;
        CH[k] = cg;
      }
    }
    // A's row divided by bA, then the one-piece relations of the chunk
    const float ib = 1.f / (1.f - eAc * AH[0].y);
    const float pa = eAa * ib, pc = (-eAc * CH[0].y) * ib;
    const float pd = tfma(-eAc, -ND[0].y, eAd) * ib;
    const float rgA = CH[0].x, raA = AH[0].x, rdA = -ND[0].x;
    const float frd = tfma(-rgA, pd, rdA), fra = tfma(-rgA, pa, raA), frg = -rgA * pc;
    const float ig = 1.f / tfma(-eBa, pc, 1.f);
    const float e_dh = tfma(-eBa, pd, eBd) * ig, e_ah = (-eBa * pa) * ig, e_ch = eBc * ig;
    sm.rd[sk(tid)] = frd;
    sm.ra[sk(tid)] = fra;
    sm.rg[sk(tid)] = frg;
    if (tid == tl) { cs.iface[0] = e_ah; cs.iface[1] = e_ch; cs.iface[2] = e_dh; }
    __syncthreads();
    {  // the block row of chunk t < tl, as in the scalar kernel
      const int t = tid, i = sk(t);
      float A = 0.f, B = 1.f, Cc = 0.f, D = 0.f, Uv = 0.f, Vv = 0.f;
      if (t < tl) {
        A = e_ah;
        B = 1.f - e_ch * sm.ra[sk(t + 1)];
        Cc = -e_ch * sm.rg[sk(t + 1)];
        D = tfma(-e_ch, sm.rd[sk(t + 1)], e_dh);
        if (t == 0) { Uv = A; A = 0.f; }
        if (t == tl - 1) { Vv = Cc; Cc = 0.f; }
      }
      sm.A[i] = A; sm.B[i] = B; sm.Cc[i] = Cc; sm.D[i] = D; sm.U[i] = Uv; cs.V[i] = Vv;
    }
    __syncthreads();
    if (warp == Q - 1) {
      block_solve3<float, NT>(cs, lane);
      __syncwarp();
      {
        ClusterSlot<float> sl;
        sl.eah = cs.iface[0]; sl.ech = cs.iface[1]; sl.edh = cs.iface[2];
        sl.rd0 = sm.rd[sk(0)]; sl.ra0 = sm.ra[sk(0)]; sl.rg0 = sm.rg[sk(0)];
        sl.yl = sm.X[sk(tl - 1)];
        sl.al = sm.Z[sk(tl - 1)];
        sl.gl = cs.Wg[sk(tl - 1)];
        sl.y0 = sm.X[sk(0)]; sl.a0 = sm.Z[sk(0)]; sl.g0 = cs.Wg[sk(0)];
        const int jl = tlshort ? H - 2 : H - 1;  // end pair of the interface chunk
        sl.uf = us[0].x;
        sl.lf = lo[0].x;
        sl.ul = us[jl * NT + tl].y;
        sl.ll = lo[jl * NT + tl].y;
        sl.ef = ITER ? es[0].x : 0.f;
        sl.el = ITER ? es[jl * NT + tl].y : 0.f;
        sl.ti = tl;
        sl.jf = C - 1;
        if (lane < CS) store_slot(cluster.map_shared_rank(&cs.slots[par][rank], lane), sl);
      }
    }
    // the step's cluster barrier: the last warp (the only one that writes to or
    // reads from another CTA's memory in the step loop) arrives with release
    // semantics, the others relaxed, without a fence of their own; every
    // thread waits (acquire)
    if (warp == Q - 1)
      asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    else
      asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
    if (warp == Q - 1)
      cluster_solve<float, NT, CS>(cs, per, lane, rank, par, cluster, ITER ? (lastit ? 2 : 1) : 0);
    __syncthreads();
    par ^= 1;
    // ---- chunk-end values, X_A, back-substitution of both halves
    const float Y = cs.reply.Y, P = cs.reply.P;
    if (tid <= tl) {
      auto xend = [&](int t) -> float {
        return t < tl ? tfma(-cs.Wg[sk(t)], Y, tfma(-sm.Z[sk(t)], P, sm.X[sk(t)])) : Y;
      };
      const float Xt = xend(tid);
      const float L = tid > 0 ? xend(tid - 1) : P;
      const float XA = tfma(-pc, Xt, tfma(-pa, L, pd));
      const float d0 = tfma(-frg, Xt, tfma(-fra, L, frd));  // the first node
      const float2 Lp = make_float2(L, XA), Xp = make_float2(XA, Xt);
#pragma unroll
      for (int k = 0; k < H; ++k) {
        float2 ndelta = fma2(CH[k], Xp, fma2(AH[k], Lp, ND[k]));
        if (k == 0) ndelta.x = -d0;
        if (k == H - 1 && shrt) ndelta.y = 0.f;  // the padding pair keeps its value
        const int o = k * NT + tid;
        float2 nv;
        if constexpr (ITER) {
          const float2 inc = sub2(es[o], ndelta);  // e + delta
          if (!lastit) {
            es[o] = inc;
            nv = add2(us[o], inc);  // the next iterate's value (edges below)
          } else {
            const float2 uo = us[o], l0 = lo[o];
            const float2 y = sub2(inc, l0);
            nv = add2(uo, y);
            lo[o] = sub2(sub2(nv, uo), y);
            us[o] = nv;
          }
        } else {
          const float2 uo = us[o], l0 = lo[o];
          const float2 ny = add2(ndelta, l0);
          nv = sub2(uo, ny);
          lo[o] = add2(sub2(nv, uo), ny);
          us[o] = nv;
        }
        if (k == 0) cs.hfirst[tid] = nv.x;
        if (k == H - 2 && shrt) cs.hlast[tid] = nv.y;
        if (k == H - 1 && !shrt) cs.hlast[tid] = nv.y;
      }
    }
    __syncthreads();
  }  // iterations
  }  // steps
#pragma unroll
  for (int k = 0; k < H; ++k) {
    const float2 x = us[k * NT + tid];
    if (k < clen) row[k] = x.x;
    if (k + H < clen) row[k + H] = x.y;
  }
  cluster.sync();  // no CTA leaves while another may still address its memory
}

// FP32 rows run the packed-pair form of the kernel (k_btcs_cluster_x2): the
// lagged BTCS, Crank-Nicolson, Picard and Newton rows (the iterating variants
// stage the iterate's e beside the state: a third array of dynamic shared
// memory)
#define REG_CLUSTER(T, DT, NT, C, CS)                                                       \
  reg.push_back({K_BTCS_CLUSTER, DT, NT, C, CS,                                             \
                 reinterpret_cast<const void*>(&k_btcs_cluster_x2<NT, C, CS, VAR_BTCS>),   \
                 sizeof(T) * size_t(NT) * C * 2});                                          \
  reg.push_back({K_CN_CLUSTER, DT, NT, C, CS,                                               \
                 reinterpret_cast<const void*>(&k_btcs_cluster_x2<NT, C, CS, VAR_CN>),     \
                 sizeof(T) * size_t(NT) * C * 2});                                          \
  reg.push_back({K_PICARD_CLUSTER, DT, NT, C, CS,                                           \
                 reinterpret_cast<const void*>(&k_btcs_cluster_x2<NT, C, CS, VAR_PICARD>), \
                 sizeof(T) * size_t(NT) * C * 3});                                          \
  reg.push_back({K_NEWTON_CLUSTER, DT, NT, C, CS,                                           \
                 reinterpret_cast<const void*>(&k_btcs_cluster_x2<NT, C, CS, VAR_NEWTON>), \
                 sizeof(T) * size_t(NT) * C * 3});
#define REG_CLUSTERS(T, DT, NT, C)                                                          \
  REG_CLUSTER(T, DT, NT, C, 2) REG_CLUSTER(T, DT, NT, C, 3) REG_CLUSTER(T, DT, NT, C, 4)    \
  REG_CLUSTER(T, DT, NT, C, 5) REG_CLUSTER(T, DT, NT, C, 6) REG_CLUSTER(T, DT, NT, C, 7)    \
  REG_CLUSTER(T, DT, NT, C, 8)
// cluster sizes above the portable 8 (launchable where the device can
// schedule them; the planner asks the occupancy API first)
#define REG_CLUSTERS_WIDE(T, DT, NT, C)                                                     \
  REG_CLUSTER(T, DT, NT, C, 9) REG_CLUSTER(T, DT, NT, C, 10) REG_CLUSTER(T, DT, NT, C, 11)  \
  REG_CLUSTER(T, DT, NT, C, 12) REG_CLUSTER(T, DT, NT, C, 13) REG_CLUSTER(T, DT, NT, C, 14) \
  REG_CLUSTER(T, DT, NT, C, 15) REG_CLUSTER(T, DT, NT, C, 16)

// FP32 only: FP64 rows are limited by the FP64 pipe, where the multi-level
// solver is as fast. 128-thread CTAs (4096 nodes each) in clusters of up to
// 16 cover rows up to 65536 nodes at half the padding granularity of the
// 256-thread shapes, which remain for devices (or modes) limited to 8.
void register_btcs_cluster(std::vector<KernelEntry>& reg) {
  REG_CLUSTERS(float, 0, 256, 32)
  REG_CLUSTERS(float, 0, 128, 32)
  REG_CLUSTERS_WIDE(float, 0, 128, 32)
}

}  // namespace burgers
