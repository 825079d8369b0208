// btcs_cluster.cu -- lagged upwind BTCS (Sec. 2.4, Eq. 23) for rows too long
// for one CTA but short enough for a thread-block cluster: the row stays in
// the shared memory of CS CTAs for all of its steps, as in the resident kernel.
//
// Three levels of the same partitioned elimination:
//   chunk   each thread eliminates its C (or C - 1) rows (as in btcs.cu) and
//           leaves one reduced row per chunk in its unknown X_t (the
//           chunk-end value);
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

#include <type_traits>

#include "btcs_common.cuh"
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
template <typename T, int NT, int CS>
__device__ __forceinline__ void cluster_solve(ClusterShared<T, NT>& cs, bool per, int lane,
                                              int rank, int par, cg::cluster_group& cluster) {
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
    first = comp_add(s.uf, d0, lf);
    last = comp_add(s.ul, Y, ll);
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

// One cluster per row (rows have (CS-1) W < n <= CS W, W = NT*C). The row's
// nodes are spread evenly over the CS CTAs, and each CTA's nk nodes over
// tk = ceil(nk / C) chunks of C or C - 1 nodes, the last bk = tk C - nk of
// them one node short; threads from tk on hold no nodes. Since nk > W/2 - 1,
// tk > NT/2 > C > bk, so every row length has such a split. A short chunk
// ends at node C - 2, a position known at compile time: every warp runs the
// one sweep, and a short chunk costs a few selects at that position (a chunk
// ending at an arbitrary node would need a select at every node, and the
// warp holding it would pace the CTA and, through the cluster barrier, every
// CTA of the row).
template <typename T, int NT, int C, int CS>
__global__ void __cluster_dims__(CS, 1, 1)
__launch_bounds__(NT, (sizeof(T) == 4 && NT <= 512) ? 512 / NT : 1)
    k_btcs_cluster(T* __restrict__ u, const RowDesc* __restrict__ rows, int count,
                   int* __restrict__ counter) {
  (void)counter;
  constexpr int Q = NT / 32;
  static_assert(CS >= 2 && CS <= 16, "slots hold at most 16 CTAs");
  static_assert(C >= 3, "a short chunk keeps at least two nodes");
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = int(cluster.block_rank());
  const int item = int(blockIdx.x) / CS;
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ ClusterShared<T, NT> cs;
  BtcsShared<T, NT>& sm = cs.sm;
  T* us = reinterpret_cast<T*>(dsm);  // C * NT values
  T* lo = us + C * NT;                // C * NT values (FP32)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool valid = item < count;    // grid is count * CS: always true
  const RowDesc rd = rows[valid ? item : 0];
  const int n = rd.n;
  const bool per = rd.bc == BC_PERIODIC;
  const bool lastcta = rank == CS - 1;
  const int nbase = n / CS, nrem = n % CS;
  const int nk = nbase + (rank < nrem ? 1 : 0);                    // nodes of this CTA
  const int64_t kstart = int64_t(rank) * nbase + (rank < nrem ? rank : nrem);
  const int tk = (nk + C - 1) / C;            // chunks holding nodes
  const int bk = tk * C - nk;                 // short chunks among them (the last ones)
  const int tl = tk - 1;                      // its last chunk (the interface)
  const int ts = tk - bk;                     // first short chunk
  const bool active = tid < tk;
  const bool shrt = active && tid >= ts;      // chunk of C - 1 nodes
  const int cstart = tid * C - (shrt ? tid - ts : 0);  // first node of the chunk in the CTA
  const int clen = active ? (shrt ? C - 1 : C) : 0;
  T* row = u + rd.offset + kstart;
  // ---- load, publish the chunk edges and this CTA's ends to its neighbours
#pragma unroll
  for (int j = 0; j < C; ++j) {
    const T x = j < clen ? row[cstart + j] : T(0);
    us[j * NT + tid] = x;
    if constexpr (Kahan<T>::on) lo[j * NT + tid] = T(0);
    if (j == 0) cs.hfirst[tid] = x;
    if (j == C - 2 && shrt) cs.hlast[tid] = x;
    if (j == C - 1 && !shrt) cs.hlast[tid] = x;
  }
  __syncthreads();
  cluster.sync();  // every CTA of the cluster runs before any addresses another's memory
  if (tid == 0) {
    const int kl = rank > 0 ? rank - 1 : CS - 1, kr = rank + 1 < CS ? rank + 1 : 0;
    cluster.map_shared_rank(&cs.reply, kr)->halo_l = cs.hlast[tl];
    cluster.map_shared_rank(&cs.reply, kl)->halo_r = cs.hfirst[0];
  }
  cluster.sync();
  const T r = T(rd.r), s = T(rd.s), ds1 = T(1) + T(2) * s;
  // Dirichlet identity rows: the row's first node is replaced at j = 0; its
  // last one (the end row of chunk tl of the last CTA) only sets that chunk's
  // end relation, which is zeroed after the sweep. Warps of chunks without
  // nodes skip the sweep; lanes without nodes in a mixed warp compute values
  // nobody reads.
  const bool dfirst = !per && rank == 0 && tid == 0;
  const bool dlast = !per && lastcta && tid == tl;
  const bool padwarp = __all_sync(FULL_MASK, !active);
  const bool tlshort = bk > 0;                // the interface chunk is short
  T ch[C], ah[C], dd[C];
  int par = 0;  // slot buffer of this step
  for (int64_t step = 0; step < rd.nsteps; ++step) {
    const T halo_l = cs.reply.halo_l, halo_r = cs.reply.halo_r;
    T left = tid > 0 ? cs.hlast[tid - 1] : halo_l;
    T right = tid < tl ? cs.hfirst[tid + 1] : halo_r;
    // ---- assembly fused with the forward sweep (rows as in btcs.cu), then
    // the backward sweep: (delta, alpha, gamma) into (dd, ah, ch)
    T e_ch = T(0), e_ah = T(0), e_dh = T(0);
    if (padwarp) {  // all rows identity
      dd[0] = T(0); ah[0] = T(0); ch[0] = T(0);
    } else {
      // a short chunk's end row reads its right neighbour from its last slot
      if (shrt) us[(C - 1) * NT + tid] = right;
      T chp = T(0), ahp = T(-1), dhp = T(0);
      T ul = left, a = us[tid];
#pragma unroll
      for (int j = 0; j < C; ++j) {
        const T an = (j + 1 < C) ? us[(j + 1) * NT + tid] : right;
        const T ur = an;
        const T ra = r * a;
        T l = -s - tmax(ra, T(0));
        T c = tmin(ra, T(0)) - s;
        T d = ds1 + tabs(ra);
        T rhs = tfma(l, a - ul, -c * (ur - a));
        if (j == 0 && dfirst) { l = T(0); c = T(0); d = T(1); rhs = T(0); }
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
      // the end row: node C - 1, or C - 2 of a short chunk
      e_ch = shrt ? ch[C - 2] : ch[C - 1];
      e_ah = shrt ? ah[C - 2] : ah[C - 1];
      e_dh = shrt ? dd[C - 2] : dd[C - 1];
      T cd = T(0), ca = T(0), cgm = T(-1);
      dd[C - 1] = T(0); ah[C - 1] = T(0); ch[C - 1] = T(-1);
#pragma unroll
      for (int j = C - 2; j >= 0; --j) {
        const T cj = ch[j];
        cd = tfma(-cj, cd, dd[j]);
        ca = tfma(-cj, ca, ah[j]);
        cgm = -cj * cgm;
        if (j == C - 2 && shrt) { cd = T(0); ca = T(0); cgm = T(-1); }  // a short chunk's end row
        dd[j] = cd; ah[j] = ca; ch[j] = cgm;
      }
      if (dlast) { e_ch = T(0); e_ah = T(0); e_dh = T(0); }
    }
    sm.rd[sk(tid)] = dd[0];
    sm.ra[sk(tid)] = ah[0];
    sm.rg[sk(tid)] = ch[0];
    if (tid == tl) { cs.iface[0] = e_ah; cs.iface[1] = e_ch; cs.iface[2] = e_dh; }
    __syncthreads();
    // ---- the block row of this thread's chunk t (chunks 0..tl-1; the
    // interface row tl is the cluster's): its end row with the first-row
    // relation of chunk t + 1 substituted, every thread its own
    {
      const int t = tid, i = sk(t);
      T A = T(0), B = T(1), Cc = T(0), D = T(0), Uv = T(0), Vv = T(0);
      if (t < tl) {
        const T ech = e_ch;
        A = e_ah;
        B = T(1) - ech * sm.ra[sk(t + 1)];
        Cc = -ech * sm.rg[sk(t + 1)];
        D = tfma(-ech, sm.rd[sk(t + 1)], e_dh);
        if (t == 0) { Uv = A; A = T(0); }
        if (t == tl - 1) { Vv = Cc; Cc = T(0); }
      }
      sm.A[i] = A; sm.B[i] = B; sm.Cc[i] = Cc; sm.D[i] = D; sm.U[i] = Uv; cs.V[i] = Vv;
    }
    __syncthreads();
    if (warp == Q - 1) {  // the last warp (warp 0 also carries the CTA's first node)
      block_solve3<T, NT>(cs, lane);
      __syncwarp();
      {
        ClusterSlot<T> sl;
        sl.eah = cs.iface[0]; sl.ech = cs.iface[1]; sl.edh = cs.iface[2];
        sl.rd0 = sm.rd[sk(0)]; sl.ra0 = sm.ra[sk(0)]; sl.rg0 = sm.rg[sk(0)];
        sl.yl = tl > 0 ? sm.X[sk(tl - 1)] : T(0);
        sl.al = tl > 0 ? sm.Z[sk(tl - 1)] : T(0);
        sl.gl = tl > 0 ? cs.Wg[sk(tl - 1)] : T(0);
        sl.y0 = sm.X[sk(0)]; sl.a0 = sm.Z[sk(0)]; sl.g0 = cs.Wg[sk(0)];
        const int jl = tlshort ? C - 2 : C - 1;  // end row of the interface chunk
        sl.uf = us[0];
        sl.ul = us[jl * NT + tl];
        sl.lf = T(0);
        sl.ll = T(0);
        if constexpr (Kahan<T>::on) { sl.lf = lo[0]; sl.ll = lo[jl * NT + tl]; }
        sl.ti = tl;
        sl.jf = C - 1;  // chunk 0 is never short (ts >= 1)
        // pushed into every CTA's memory (lane k writes CTA k's copy), so
        // after the cluster barrier each CTA reads its own shared memory
        if (lane < CS) store_slot(cluster.map_shared_rank(&cs.slots[par][rank], lane), sl);
      }
    }
    cluster.sync();
    if (warp == Q - 1) cluster_solve<T, NT, CS>(cs, per, lane, rank, par, cluster);
    __syncthreads();
    par ^= 1;
    // ---- chunk-end values from the block relations, back-substitution (a
    // short chunk's end row, restarted in the backward sweep, gives its X
    // exactly: delta = Xt - 0 L + 0)
    const T Y = cs.reply.Y, P = cs.reply.P;
    if (tid <= tl) {
      auto xend = [&](int t) -> T {
        return t < tl ? tfma(-cs.Wg[sk(t)], Y, tfma(-sm.Z[sk(t)], P, sm.X[sk(t)])) : Y;
      };
      const T Xt = xend(tid);
      const T L = tid > 0 ? xend(tid - 1) : P;
#pragma unroll
      for (int j = 0; j < C; ++j) {
        if (j < C - 1 || !shrt) {
          const T delta = (j == C - 1) ? Xt : tfma(-ch[j], Xt, tfma(-ah[j], L, dd[j]));
          const int o = j * NT + tid;
          T l0 = T(0);
          if constexpr (Kahan<T>::on) l0 = lo[o];
          const T nv = comp_add(us[o], delta, l0);
          us[o] = nv;
          if constexpr (Kahan<T>::on) lo[o] = l0;
          if (j == 0) cs.hfirst[tid] = nv;
          if (j == C - 2 && shrt) cs.hlast[tid] = nv;
          if (j == C - 1) cs.hlast[tid] = nv;
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < C; ++j)
    if (j < clen) row[cstart + j] = us[j * NT + tid];
  cluster.sync();  // no CTA leaves while another may still address its memory
}

#define REG_CLUSTER(T, DT, NT, C, CS)                                                       \
  reg.push_back({K_BTCS_CLUSTER, DT, NT, C, CS,                                             \
                 reinterpret_cast<const void*>(&k_btcs_cluster<T, NT, C, CS>),             \
                 sizeof(T) * size_t(NT) * C * (Kahan<T>::on ? 2 : 1)});
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
