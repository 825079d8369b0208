// multilevel.cu -- BTCS (Sec. 2.4, Eq. 23) for rows too long to stay resident
// in one CTA, e.g. the N = 2^24 periodic grid.
//
// The partitioned elimination of btcs.cu applied recursively through global
// memory. Level 0 holds the n nodes; every chunk of C consecutive rows of
// level l is eliminated by one thread and leaves six numbers: the forward
// outputs of its end row (ch, ah, dh) and the relation of its first row
// (delta, alpha, gamma). Chunk k of level l is row k of level l+1:
//     A_k = ah_k,  B_k = 1 - ch_k alpha_{k+1},  C_k = -ch_k gamma_{k+1},
//     D_k = dh_k - ch_k delta_{k+1}               (k+1 taken cyclically),
// so level l+1 has ceil(m_l / C) rows and is again (cyclic) tridiagonal. Once
// a level fits one CTA, k_ml_top solves it like the resident kernel
// (Sherman-Morrison split of the cyclic corners, extended-precision
// correction denominator). The recover sweeps then walk back down: each
// chunk repeats its elimination (nothing per row is stored, which halves the
// memory traffic) and forms
//     x_j = delta_j - alpha_j X_{k-1} - gamma_j X_k
// from the two solved chunk-end values. Level 0 reads u^n and writes u^{n+1}
// in place: each thread reads and writes only its own nodes.
//
// Per step: L reduce launches, one top launch per top shape, L recover
// launches; the host captures the whole step sequence in a CUDA graph.
#include <algorithm>

#include "api_internal.h"
#include "btcs_common.cuh"
#include "common.cuh"
#include "kernels.h"

namespace burgers {

constexpr int ML_MAXL = 6;

struct MLRow {
  int64_t offset;
  int64_t nsteps;
  double r, s;
  int32_t n, bc, levels;
  int32_t var;    // 0 lagged BTCS, 1 Crank-Nicolson, 2 Picard, 3 Newton (level-0 rows)
  int32_t iters;  // iterations per step (Picard, Newton; else 1)
  int32_t pad1, pad2, pad3;
  int64_t m[ML_MAXL + 1];   // rows per level, m[0] = n
  int64_t ef[ML_MAXL];      // workspace offset of the six chunk arrays of level l
  int64_t x[ML_MAXL + 1];   // workspace offset of the solution of level l >= 1
};

// Row j of level `level` (>= 1) from the chunk arrays of the level below.
template <typename T>
struct UpperRows {
  const T* E;
  int64_t M;
  int64_t base;
  int je;
  __device__ __forceinline__ void operator()(int j, T& l, T& d, T& c, T& rhs) const {
    if (j > je) { l = T(0); d = T(1); c = T(0); rhs = T(0); return; }
    const int64_t i = base + j;
    const int64_t i1 = (i + 1 == M) ? 0 : i + 1;
    const T ech = E[i], eah = E[M + i], edh = E[2 * M + i];
    const T fd = E[3 * M + i1], fa = E[4 * M + i1], fg = E[5 * M + i1];
    l = eah;
    d = T(1) - ech * fa;
    c = -ech * fg;
    rhs = tfma(-ech, fd, edh);
  }
};

// Upper-level tiles staged in shared memory: the CTA's TILE = NT*C rows of the
// six chunk arrays of the level below (the first-row relation one row
// further, for each row's right neighbour), loaded coalesced, each array
// skewed by one element per C rows so that the C consecutive rows of the 32
// threads of a warp fall in distinct banks (C + 1 is odd).
template <typename T, int NT, int C>
struct UpperSmem {
  static constexpr int TILE = NT * C;
  static constexpr int AS = TILE + TILE / C + 2;  // elements per array
  static constexpr size_t bytes() { return sizeof(T) * 6 * size_t(AS); }
  __device__ static __forceinline__ int sk(int p) { return p + p / C; }
};

// Row j of an upper level from the staged tile (the arithmetic of UpperRows).
template <typename T, int NT, int C>
struct UpperRowsSmem {
  const T* S;
  int lbase;  // the thread's first row within the tile
  int je;
  __device__ __forceinline__ void operator()(int j, T& l, T& d, T& c, T& rhs) const {
    using U = UpperSmem<T, NT, C>;
    if (j > je) { l = T(0); d = T(1); c = T(0); rhs = T(0); return; }
    const int p = U::sk(lbase + j), p1 = U::sk(lbase + j + 1);
    const T ech = S[p], eah = S[U::AS + p], edh = S[2 * U::AS + p];
    const T fd = S[3 * U::AS + p1], fa = S[4 * U::AS + p1], fg = S[5 * U::AS + p1];
    l = eah;
    d = T(1) - ech * fa;
    c = -ech * fg;
    rhs = tfma(-ech, fd, edh);
  }
};

// One sweep of an upper level (levels >= 1; level 0 runs k_ml_sweep0, whose
// recover sweep writes u^{n+1} into the other buffer of the step's parity).
template <typename T, int NT, int C, bool LVL0, bool RECOVER>
__global__ void __launch_bounds__(NT) k_ml_sweep(T* __restrict__ u, T* __restrict__ u2,
                                                 T* __restrict__ lo, T* __restrict__ ws,
                                                 const MLRow* __restrict__ rows,
                                                 const TileItem* __restrict__ items, int nitems,
                                                 int level, int64_t step, int iter,
                                                 T* __restrict__ ea, T* __restrict__ eb) {
  static_assert(!LVL0, "level 0 runs k_ml_sweep0");
  (void)iter; (void)ea; (void)eb;
  {
    // the tile staged in shared memory (UpperSmem); every thread passes the
    // barriers, those past the level's end with no rows
    using U = UpperSmem<T, NT, C>;
    extern __shared__ __align__(16) unsigned char ml_dsm[];
    T* S = reinterpret_cast<T*>(ml_dsm);
    (void)u; (void)u2; (void)lo;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
      const TileItem ti = items[it];
      const MLRow& R = rows[ti.row];
      if (step >= R.nsteps) continue;  // the whole CTA
      const int64_t M = R.m[level];
      const int64_t t0 = int64_t(ti.tile) * U::TILE;
      const int nrow = int(M - t0 < int64_t(U::TILE) ? M - t0 : int64_t(U::TILE));
      const T* E = ws + R.ef[level - 1];
      for (int q = threadIdx.x; q <= nrow; q += NT) {
        const int64_t i = t0 + q;
        const int pq = U::sk(q);
        if (q < nrow) {
          S[pq] = E[i];
          S[U::AS + pq] = E[M + i];
          S[2 * U::AS + pq] = E[2 * M + i];
        }
        const int64_t i1 = (i == M) ? 0 : i;  // row i - 1's right neighbour (cyclic)
        S[3 * U::AS + pq] = E[3 * M + i1];
        S[4 * U::AS + pq] = E[4 * M + i1];
        S[5 * U::AS + pq] = E[5 * M + i1];
      }
      __syncthreads();
      const int lbase = int(threadIdx.x) * C;
      const int64_t base = t0 + lbase;
      const bool active = base < M;
      const int je = !active ? -1
                             : int(M - 1 - base < int64_t(C - 1) ? M - 1 - base : int64_t(C - 1));
      T v[C], ah[C], ch[C];
      T e_ch, e_ah, e_dh;
      UpperRowsSmem<T, NT, C> rsrc{S, lbase, je};
      chunk_forward<T, C>(v, ah, ch, je, rsrc, e_ch, e_ah, e_dh);
      chunk_backward<T, C>(v, ah, ch, je);
      const int64_t k = base / C;
      const int64_t Mn = R.m[level + 1];
      if constexpr (!RECOVER) {
        if (active) {
          T* Eo = ws + R.ef[level];
          Eo[k] = e_ch;
          Eo[Mn + k] = e_ah;
          Eo[2 * Mn + k] = e_dh;
          Eo[3 * Mn + k] = v[0];
          Eo[4 * Mn + k] = ah[0];
          Eo[5 * Mn + k] = ch[0];
        }
      } else {
        // the solution of this thread's rows into its own slots of array 0
        // (only it reads them), then the tile stored coalesced
        if (active) {
          const T* Xn = ws + R.x[level + 1];
          const T L = k > 0 ? Xn[k - 1] : (R.bc == BC_PERIODIC ? Xn[Mn - 1] : T(0));
          const T Xk = Xn[k];
#pragma unroll
          for (int j = 0; j < C; ++j)
            if (j <= je) S[U::sk(lbase + j)] = tfma(-ch[j], Xk, tfma(-ah[j], L, v[j]));
        }
        __syncthreads();
        T* out = ws + R.x[level];
        for (int q = threadIdx.x; q < nrow; q += NT) out[t0 + q] = S[U::sk(q)];
      }
      __syncthreads();  // before the next tile is staged
    }
  }
}

// ---------------------------------------------------------------------------
// Level-0 sweeps with staged tiles. A CTA's tile of NT*C nodes and its two
// halo nodes are copied into shared memory with cp.async while the previous tile is being
// eliminated (two buffers), so the sweep streams instead of waiting on each
// thread's strided loads. Rows whose start is 16-byte aligned move in 16-byte
// vectors (the last one zero-filled past the row end); others move element
// by element. The buffer inserts 16 bytes after every 128, which keeps the
// threads' reads of their C consecutive nodes spread over the banks while
// leaving every vector slot 16-byte aligned. The recover sweep writes its
// results back into its own slots and stores the tile contiguously.
//
// Local index L of node t0 + i is VE + i (VE elements per vector); the slot
// L = VE - 1 holds the left neighbour of node t0 (periodic image for t0 = 0)
// and L = VE + TILE the right neighbour of the tile's last node (row[0] when
// that node is the row's last).
// ---------------------------------------------------------------------------
template <typename T, int NT, int C>
struct Sweep0Smem {
  static constexpr int TILE = NT * C;
  static constexpr int VE = 16 / int(sizeof(T));
  static constexpr int GRP = 128 / int(sizeof(T));
  __device__ __host__ static constexpr int idx(int L) { return L + VE * (L / GRP); }
  static constexpr int SSK = (idx(TILE + VE) / VE + 1) * VE;  // one buffer, elements
  // buffers: the state and the iterate's e (Picard, Newton), two of each
  static constexpr size_t bytes(bool recover, bool iterating = false) {
    (void)recover;
    return sizeof(T) * size_t(SSK) * 2 * (1 + (iterating ? 1 : 0));
  }
};

template <typename T>
__device__ __forceinline__ unsigned smem_addr(const T* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
// One element; src_bytes 0 zero-fills the slot without reading.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem, bool valid) {
  const int nb = valid ? int(sizeof(T)) : 0;
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(smem_addr(smem)),
                 "l"(gmem), "r"(nb)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(smem_addr(smem)),
                 "l"(gmem), "r"(nb)
                 : "memory");
}
// One 16-byte vector, of which the first nb bytes are read (rest zero-filled).
__device__ __forceinline__ void cp_async_vec(void* smem, const void* gmem, int nb) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_addr(smem)),
               "l"(gmem), "r"(nb)
               : "memory");
}
// A 16-byte shared-memory load the compiler may not merge with an earlier
// load of the same slot (so a value need not stay live in registers).
__device__ __forceinline__ float4 lds_fresh(const float* p) {
  float4 w;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n"
               : "=f"(w.x), "=f"(w.y), "=f"(w.z), "=f"(w.w)
               : "r"(smem_addr(p)));
  return w;
}
__device__ __forceinline__ double2 lds_fresh(const double* p) {
  double2 w;
  asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];\n" : "=d"(w.x), "=d"(w.y) : "r"(smem_addr(p)));
  return w;
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Copies nodes [t0, min(t0 + TILE, n)) of `row` to slots VE.. of `buf`.
template <typename T, int NT, int C>
__device__ __forceinline__ void stage_tile(T* buf, const T* row, int64_t t0, int64_t n) {
  using SM = Sweep0Smem<T, NT, C>;
  constexpr int VE = SM::VE;
  const int tid = threadIdx.x;
  const int64_t rem = n - t0;  // nodes left in the row from t0 (> 0)
  const int cnt = rem < SM::TILE ? int(rem) : SM::TILE;
  if ((reinterpret_cast<uintptr_t>(row) & 15) == 0) {
    const T* src = row + t0;
    for (int q = tid; q * VE < cnt; q += NT) {
      const int e = q * VE;
      const int left = cnt - e;
      cp_async_vec(buf + SM::idx(VE + e), src + e, (left < VE ? left : VE) * int(sizeof(T)));
    }
  } else {
    const T* src = row + t0;
    for (int i = tid; i < cnt; i += NT) cp_async_elem(buf + SM::idx(VE + i), src + i, true);
  }
}

// Level-0 row i of variant VAR from the iterate a = w_i and its neighbours
// (e: the iterate's e_i; unused by BTCS and CN). rm, sm, ds1 are the matrix
// coefficients (CN: r/2, s/2).
template <typename T, int VAR>
__device__ __forceinline__ void ml_row(T ul, T a, T ur, T e, T rm, T sm, T ds1, T hr, T& l,
                                       T& d, T& c, T& rhs) {
  if constexpr (VAR == 3) {  // Newton on the Eq. 11 residual (central convection)
    const T ha = hr * a;
    l = -ha - sm;
    c = ha - sm;
    d = tfma(hr, ur - ul, ds1);
    rhs = tfma(sm, (ur - a) - (a - ul), tfma(-ha, ur - ul, -e));
  } else {
    const T ra = rm * a;
    l = -sm - tmax(ra, T(0));
    c = tmin(ra, T(0)) - sm;
    d = ds1 + tabs(ra);
    rhs = tfma(l, a - ul, -c * (ur - a));  // explicit increment from the same coefficients
    if constexpr (VAR == 1) rhs = T(2) * rhs;
    if constexpr (VAR == 2) rhs = rhs - e;
  }
}

// Row i of A(u)^T (the lagged BTCS matrix of the state u transposed: sub
// c_{i-1}, diagonal d_i, super l_{i+1}; a Dirichlet end row of A is an
// identity row, so its coefficients enter as 0, 1, 0) with the right-hand
// side of the increment form lam - A^T lam, from u and lam at nodes i-1, i,
// i+1 and whether those rows are identity rows (the adjoint of the BTCS
// step: A^T nu = lam - A^T lam, mu = lam + nu).
template <typename T>
__device__ __forceinline__ void ml_row_t(T am, T a, T ap, T lm, T lam, T lp, bool idm, bool id,
                                         bool idp, T r, T s, T ds1, T& l, T& d, T& c, T& rhs) {
  const T cm = idm ? T(0) : tmin(r * am, T(0)) - s;   // c_{i-1}
  const T lpp = idp ? T(0) : -s - tmax(r * ap, T(0));  // l_{i+1}
  const T dm1 = id ? T(0) : tfma(r, tabs(a), T(2) * s);  // d_i - 1
  l = cm;
  d = T(1) + dm1;
  c = lpp;
  rhs = -tfma(cm, lm, tfma(dm1, lam, lpp * lp));
}

// The CTA handles items blockIdx.x + k * gridDim.x, k = 0, 1, ... Their
// (row, tile, row offset, row length) are gathered into shared memory KC at a
// time, so staging the next tile needs no dependent global loads; the row's
// record travels with the tile (cp.async into a per-buffer copy).
//
// VAR selects the level-0 rows: 0 lagged BTCS, 1 Crank-Nicolson, 2 Picard,
// 3 Newton (see ml_row and btcs_kernel.cuh). The iterating variants (2, 3)
// stage the iterate's e beside u^n (iteration `iter` reads e from ea or eb,
// none in the first) and, except in the step's last iteration, the recover
// sweep writes e + delta to the other buffer instead of updating u.
// (the iterating variants' six FP32 tile buffers allow two CTAs of 256
// threads per SM, so their register budget is that of two)
template <typename T, int NT, int C, bool RECOVER, int VAR = 0>
__global__ void __launch_bounds__(NT, ((sizeof(T) == 4 && VAR < 2) ? 768 : 512) / NT)
    k_ml_sweep0(T* __restrict__ u, T* __restrict__ u2, T* __restrict__ lo, T* __restrict__ ws,
                const MLRow* __restrict__ rows, const TileItem* __restrict__ items, int nitems,
                int level, int64_t step, int iter, T* __restrict__ ea, T* __restrict__ eb) {
  constexpr bool ITV = VAR == 2 || VAR == 3;
  constexpr bool TR = VAR == 4;  // transposed system of the adjoint: lam in ea, nu to eb
  constexpr bool STAGE_E = ITV || TR;
  const T* ecur = TR ? ea : ((ITV && iter > 0) ? ((iter & 1) ? ea : eb) : nullptr);
  T* enext = TR ? eb : ((iter & 1) ? eb : ea);
  if constexpr (!STAGE_E) { (void)ecur; (void)enext; }
  using SM = Sweep0Smem<T, NT, C>;
  constexpr int TILE = SM::TILE, VE = SM::VE, SSK = SM::SSK;
  // FP32 recover sweeps: the Kahan term of u lives in `lo` as one byte per
  // node (lo8_encode against the value it compensates), read and written in
  // place by each thread for its own nodes (16 contiguous bytes: no staging)
  constexpr bool KL = RECOVER && Kahan<T>::on;
  constexpr int EBUF = 2;  // first buffer of e
  constexpr int RV = int(sizeof(MLRow) / 16);
  static_assert(sizeof(MLRow) % 16 == 0, "row record moves in 16-byte pieces");
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ __align__(16) MLRow srow[2];
  __shared__ int stile[2];
  constexpr int KC = 64;  // cached item descriptors
  static_assert(NT >= KC, "one thread per cached descriptor");
  __shared__ int64_t coff[KC];
  __shared__ int crow[KC], ctile[KC], cn[KC];
  T* sbase = reinterpret_cast<T*>(dsm);
  (void)level;
  T* src = (step & 1) ? u2 : u;
  T* dst = (step & 1) ? u : u2;
  const int tid = threadIdx.x;
  const int G = gridDim.x;
  const int nk = int(blockIdx.x) < nitems ? (nitems - int(blockIdx.x) + G - 1) / G : 0;
  if (nk == 0) return;

  auto fill = [&](int k0) {  // descriptors of items k0 .. k0 + KC - 1
    const int k = k0 + tid;
    if (tid < KC && k < nk) {
      const TileItem ti = items[int(blockIdx.x) + k * G];
      crow[tid] = ti.row;
      ctile[tid] = ti.tile;
      coff[tid] = rows[ti.row].offset;
      cn[tid] = rows[ti.row].n;
    }
  };
  auto prefetch = [&](int k, int b) {
    const int slot = k % KC;
    const int rowi = crow[slot];
    const int64_t n = cn[slot];
    const int64_t t0 = int64_t(ctile[slot]) * TILE;
    const T* row = src + coff[slot];
    T* su = sbase + b * SSK;
    stage_tile<T, NT, C>(su, row, t0, n);
    if (tid == 0) {
      cp_async_elem(su + SM::idx(VE - 1), row + (t0 == 0 ? n - 1 : t0 - 1), true);
      stile[b] = ctile[slot];
    }
    if (tid == NT - 1) {
      const int64_t gr = t0 + TILE < n ? t0 + TILE : 0;
      cp_async_elem(su + SM::idx(VE + TILE), row + gr, true);
    }
    if (tid >= 32 && tid < 32 + RV)
      cp_async_vec(reinterpret_cast<char*>(&srow[b]) + 16 * (tid - 32),
                   reinterpret_cast<const char*>(rows + rowi) + 16 * (tid - 32), 16);
    if constexpr (STAGE_E) {
      if (ecur) {  // e (lam) of the tile and of its two neighbours
        const T* erow = ecur + coff[slot];
        T* se = sbase + (EBUF + b) * SSK;
        stage_tile<T, NT, C>(se, erow, t0, n);
        if (tid == 0) cp_async_elem(se + SM::idx(VE - 1), erow + (t0 == 0 ? n - 1 : t0 - 1), true);
        if (tid == NT - 1)
          cp_async_elem(se + SM::idx(VE + TILE), erow + (t0 + TILE < n ? t0 + TILE : 0), true);
      }
    }
    cp_async_commit();
  };

  fill(0);
  __syncthreads();
  prefetch(0, 0);
  int b = 0;
  for (int k = 0; k < nk; ++k, b ^= 1) {
    if (k + 1 < nk) {
      if ((k + 1) % KC == 0) {
        __syncthreads();  // every thread is past its last read of the cache
        fill(k + 1);
        __syncthreads();
      }
      prefetch(k + 1, b ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const MLRow& R = srow[b];
    const int64_t M = R.m[0];
    const int64_t t0 = int64_t(stile[b]) * TILE;
    const int64_t base = t0 + int64_t(tid) * C;
    T* su = sbase + b * SSK;
    const int lb = VE + tid * C;  // local index of this thread's first node
    using V = typename Vec16<T>::type;
    constexpr int NV = C / VE;
    static_assert(C % VE == 0, "a chunk is whole vectors");
    const bool lastit = !ITV || iter + 1 == R.iters;
    if (base < M && iter < R.iters) {
      const bool active = step < R.nsteps;
      // the chunk and its two neighbours: a[0] = w_{base-1}, a[1 + j] = w_{base+j}
      // (w = u^n, plus e for the iterating variants)
      T a[C + 2], ev[C + 2];
      a[0] = su[SM::idx(lb - 1)];
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const V w = *reinterpret_cast<const V*>(su + SM::idx(lb + q * VE));
        const T* wp = reinterpret_cast<const T*>(&w);
#pragma unroll
        for (int e = 0; e < VE; ++e) a[1 + q * VE + e] = wp[e];
      }
      a[C + 1] = su[SM::idx(lb + C)];
#pragma unroll
      for (int j = 0; j < C + 2; ++j) ev[j] = T(0);
      T ehr = T(0);
      if constexpr (STAGE_E) {
        if (ecur) {
          const T* se = sbase + (EBUF + b) * SSK;
          ev[0] = se[SM::idx(lb - 1)];
#pragma unroll
          for (int q = 0; q < NV; ++q) {
            const V w = *reinterpret_cast<const V*>(se + SM::idx(lb + q * VE));
            const T* wp = reinterpret_cast<const T*>(&w);
#pragma unroll
            for (int e = 0; e < VE; ++e) ev[1 + q * VE + e] = wp[e];
          }
          ev[C + 1] = se[SM::idx(lb + C)];
          ehr = se[SM::idx(VE + TILE)];
          if constexpr (ITV) {
#pragma unroll
            for (int j = 0; j < C + 2; ++j) a[j] = a[j] + ev[j];
          }
        }
      }
      const int64_t kk = base / C;
      const int64_t Mn = R.m[1];
      T L = T(0), Xk = T(0);
      if constexpr (RECOVER) {  // issue the coarse solution loads before the sweep
        if (active) {
          const T* Xn = ws + R.x[1];
          L = kk > 0 ? Xn[kk - 1] : (R.bc == BC_PERIODIC ? Xn[Mn - 1] : T(0));
          Xk = Xn[kk];
        }
      }
      const T r = T(R.r), s = T(R.s);
      // matrix coefficients of the variant (CN: half the step's r and s)
      const T rm = VAR == 1 ? T(0.5) * r : r, smv = VAR == 1 ? T(0.5) * s : s;
      const T ds1 = T(1) + T(2) * smv, hrv = T(0.5) * r;
      const bool dir = R.bc == BC_DIRICHLET;
      T v[C], ah[C], ch[C];
      T e_ch = T(0), e_ah = T(0), e_dh = T(0);
      int je = C - 1;
      if (!active) {
        // rows already done: copied through by the last recover sweep only
      } else if (base + C < M && !dir) {
        // interior chunk of a periodic row: no row end
        auto rowsrc = [&](int j, T& l, T& d, T& c, T& rhs) {
          if constexpr (TR)
            ml_row_t<T>(a[j], a[j + 1], a[j + 2], ev[j], ev[j + 1], ev[j + 2], false, false, false,
                        r, s, ds1, l, d, c, rhs);
          else
            ml_row<T, VAR>(a[j], a[j + 1], a[j + 2], ev[j + 1], rm, smv, ds1, hrv, l, d, c, rhs);
        };
        chunk_forward<T, C>(v, ah, ch, C - 1, rowsrc, e_ch, e_ah, e_dh);
        chunk_backward<T, C>(v, ah, ch, C - 1);
      } else if (!TR && base + C < M && !(dir && base == 0)) {
        // interior chunk: no row end, no Dirichlet end row
        auto rowsrc = [&](int j, T& l, T& d, T& c, T& rhs) {
          ml_row<T, VAR>(a[j], a[j + 1], a[j + 2], ev[j + 1], rm, smv, ds1, hrv, l, d, c, rhs);
        };
        chunk_forward<T, C>(v, ah, ch, C - 1, rowsrc, e_ch, e_ah, e_dh);
        chunk_backward<T, C>(v, ah, ch, C - 1);
      } else {
        je = int(M - 1 - base < int64_t(C - 1) ? M - 1 - base : int64_t(C - 1));
        const int jend = int(M - 1 - base);  // local index of the row's last node, if here
        // right neighbour of the row's last node
        const T hr = ITV ? su[SM::idx(VE + TILE)] + ehr : su[SM::idx(VE + TILE)];
        auto rowsrc = [&](int j, T& l, T& d, T& c, T& rhs) {
          const int64_t gi = base + j;
          if (j > je) { l = T(0); d = T(1); c = T(0); rhs = T(0); return; }
          const T ur = j == jend ? hr : a[j + 2];
          if constexpr (TR) {
            const T lr = j == jend ? ehr : ev[j + 2];
            // Dirichlet: rows 0 and M-1 are identity rows of A, and there is
            // no row beyond either end
            auto ident = [&](int64_t g) { return dir && (g <= 0 || g >= M - 1); };
            ml_row_t<T>(a[j], a[j + 1], ur, ev[j], ev[j + 1], lr, ident(gi - 1), ident(gi),
                        ident(gi + 1), r, s, ds1, l, d, c, rhs);
          } else {
            ml_row<T, VAR>(a[j], a[j + 1], ur, ev[j + 1], rm, smv, ds1, hrv, l, d, c, rhs);
            if (dir && (gi == 0 || gi == M - 1)) { l = T(0); c = T(0); d = T(1); rhs = T(0); }
          }
        };
        chunk_forward<T, C>(v, ah, ch, je, rowsrc, e_ch, e_ah, e_dh);
        chunk_backward<T, C>(v, ah, ch, je);
      }
      if constexpr (!RECOVER) {
        if (active) {
          T* Eo = ws + R.ef[0];
          Eo[kk] = e_ch;
          Eo[Mn + kk] = e_ah;
          Eo[2 * Mn + kk] = e_dh;
          Eo[3 * Mn + kk] = v[0];
          Eo[4 * Mn + kk] = ah[0];
          Eo[5 * Mn + kk] = ch[0];
        }
      } else if (TR || (ITV && !lastit)) {
        // an iteration before the step's last: e + delta for the next one
        // (the transposed system: nu itself)
        if (active) {
          T* erow = enext + R.offset + base;
#pragma unroll
          for (int j = 0; j < C; ++j)
            if (j <= je) {
              const T delta = tfma(-ch[j], Xk, tfma(-ah[j], L, v[j]));
              erow[j] = (!TR && ecur) ? ev[j + 1] + delta : delta;
            }
        }
      } else {
        // u^{n+1} = u^n + delta (FP32: compensated; the iterating variants
        // add e + delta), one vector at a time, stored straight from
        // registers; rows already done are copied through
        T* drow = dst + R.offset + base;
        signed char* lrow = reinterpret_cast<signed char*>(lo) + R.offset + base;
        const int cnt = M - base < C ? int(M - base) : C;
        const bool vec = cnt == C && (reinterpret_cast<uintptr_t>(drow) & 15) == 0;
        // the chunk's compensation bytes, four to a word (registers)
        static_assert(C % 4 == 0, "whole words of compensation bytes");
        unsigned lw[C / 4], nw[C / 4];
#pragma unroll
        for (int k = 0; k < C / 4; ++k) { lw[k] = 0u; nw[k] = 0u; }
        const bool lvec = cnt == C && (reinterpret_cast<uintptr_t>(lrow) & 15) == 0 && C % 16 == 0;
        if constexpr (KL) {
          if (active) {
            if (lvec) {
#pragma unroll
              for (int k = 0; k < C / 16; ++k) {
                const uint4 w = reinterpret_cast<const uint4*>(lrow)[k];
                lw[4 * k] = w.x; lw[4 * k + 1] = w.y; lw[4 * k + 2] = w.z; lw[4 * k + 3] = w.w;
              }
            } else {
#pragma unroll
              for (int j = 0; j < C; ++j)
                if (j < cnt) lw[j >> 2] |= unsigned(static_cast<unsigned char>(lrow[j])) << (8 * (j & 3));
            }
          }
        }
#pragma unroll
        for (int q = 0; q < NV; ++q) {
          V w = lds_fresh(su + SM::idx(lb + q * VE));  // u^n again, not kept live
          T* wp = reinterpret_cast<T*>(&w);
          if (active) {
#pragma unroll
            for (int e = 0; e < VE; ++e) {
              const int j = q * VE + e;
              if (j <= je) {
                T delta = tfma(-ch[j], Xk, tfma(-ah[j], L, v[j]));
                if constexpr (ITV) {
                  if (ecur) delta = ev[j + 1] + delta;
                }
                if constexpr (KL) {
                  const signed char q0 = static_cast<signed char>(lw[j >> 2] >> (8 * (j & 3)));
                  T l0 = T(lo8_decode(float(wp[e]), q0));
                  wp[e] = comp_add(wp[e], delta, l0);
                  nw[j >> 2] |= unsigned(static_cast<unsigned char>(lo8_encode(float(wp[e]), float(l0))))
                                << (8 * (j & 3));
                } else {
                  wp[e] = wp[e] + delta;
                }
              }
            }
          }
          if (vec) {
            *reinterpret_cast<V*>(drow + q * VE) = w;
          } else {
#pragma unroll
            for (int e = 0; e < VE; ++e)
              if (q * VE + e < cnt) drow[q * VE + e] = wp[e];
          }
        }
        if constexpr (KL) {  // rows already done keep their terms
          if (active) {
            if (lvec) {
#pragma unroll
              for (int k = 0; k < C / 16; ++k)
                reinterpret_cast<uint4*>(lrow)[k] =
                    make_uint4(nw[4 * k], nw[4 * k + 1], nw[4 * k + 2], nw[4 * k + 3]);
            } else {
#pragma unroll
              for (int j = 0; j < C; ++j)
                if (j < cnt) lrow[j] = static_cast<signed char>(nw[j >> 2] >> (8 * (j & 3)));
            }
          }
        }
      }
    }
    __syncthreads();  // buffer b is refilled two iterations later
  }
}

// Copies the rows of the level-0 items from u2 back into u (after an odd
// number of steps).
template <typename T, int NT, int C>
__global__ void __launch_bounds__(NT) k_ml_copy(T* __restrict__ u, T* __restrict__ u2,
                                                T* __restrict__ lo, T* __restrict__ ws,
                                                const MLRow* __restrict__ rows,
                                                const TileItem* __restrict__ items, int nitems,
                                                int level, int64_t step, int iter,
                                                T* __restrict__ ea, T* __restrict__ eb) {
  (void)lo; (void)ws; (void)level; (void)step; (void)iter; (void)ea; (void)eb;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const TileItem ti = items[it];
    const MLRow& R = rows[ti.row];
    const int64_t lo_i = int64_t(ti.tile) * (NT * C);
    const int64_t hi_i = min(lo_i + NT * C, R.m[0]);
    for (int64_t g = lo_i + threadIdx.x; g < hi_i; g += NT) u[R.offset + g] = u2[R.offset + g];
  }
}

// Solves the top level of each row (one CTA per row) into X_top.
template <typename T, int NT, int C>
__global__ void __launch_bounds__(NT) k_ml_top(T* __restrict__ u, T* __restrict__ u2,
                                               T* __restrict__ lo, T* __restrict__ ws,
                                               const MLRow* __restrict__ rows,
                                               const TileItem* __restrict__ items, int nitems,
                                               int level, int64_t step, int iter,
                                               T* __restrict__ ea, T* __restrict__ eb) {
  __shared__ BtcsShared<T, NT> sm;
  // tops of 2048 rows or more stage their rows as the upper-level sweeps
  // stage a tile (512 x 32768 one-level rows 7% faster, the 2^24-node row 3%;
  // the smaller tops read them directly: staging made them 2-4% slower)
  constexpr bool STAGE = NT * C >= 2048;
  using U = UpperSmem<T, NT, C>;
  extern __shared__ __align__(16) unsigned char ml_dsm[];
  T* S = reinterpret_cast<T*>(ml_dsm);
  (void)u; (void)u2; (void)lo; (void)iter; (void)ea; (void)eb;
  (void)level;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const MLRow& R = rows[items[it].row];
    if (step >= R.nsteps) continue;
    const int L = R.levels;
    const int64_t M = R.m[L];
    const int base = tid * C;
    const int tl = int((M - 1) / C);
    const int je = base < M ? int(M - 1 - base < int64_t(C - 1) ? M - 1 - base : int64_t(C - 1)) : -1;
    if constexpr (STAGE) {
      const T* E = ws + R.ef[L - 1];
      const int nrow = int(M);  // at most NT * C
      for (int q = tid; q <= nrow; q += NT) {
        const int pq = U::sk(q);
        if (q < nrow) {
          S[pq] = E[q];
          S[U::AS + pq] = E[M + q];
          S[2 * U::AS + pq] = E[2 * M + q];
        }
        const int64_t i1 = (q == nrow) ? 0 : q;  // row q - 1's right neighbour (cyclic)
        S[3 * U::AS + pq] = E[3 * M + i1];
        S[4 * U::AS + pq] = E[4 * M + i1];
        S[5 * U::AS + pq] = E[5 * M + i1];
      }
      __syncthreads();
    }
    T v[C], ah[C], ch[C];
    T e_ch, e_ah, e_dh;
    if constexpr (STAGE) {
      UpperRowsSmem<T, NT, C> src{S, base, je};
      chunk_forward<T, C>(v, ah, ch, je, src, e_ch, e_ah, e_dh);
    } else {
      UpperRows<T> src{ws + R.ef[L - 1], M, base, je};
      chunk_forward<T, C>(v, ah, ch, je, src, e_ch, e_ah, e_dh);
    }
    chunk_backward<T, C>(v, ah, ch, je);
    sm.rd[sk(tid)] = v[0];
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
    if (warp == 0) {
      if (R.bc == BC_PERIODIC) reduced_solve<T, NT, true>(sm, tl, lane);
      else reduced_solve<T, NT, false>(sm, tl, lane);
    }
    __syncthreads();
    if (tid <= tl) {
      T Lv = T(0);
      if (tid > 0) Lv = sm.X[sk(tid - 1)];
      else if (R.bc == BC_PERIODIC) Lv = sm.X[sk(tl)];
      const T Xt = sm.X[sk(tid)];
      if constexpr (STAGE) {  // into this thread's own slots of array 0 (only it reads them)
#pragma unroll
        for (int j = 0; j < C; ++j)
          if (j <= je) S[U::sk(base + j)] = tfma(-ch[j], Xt, tfma(-ah[j], Lv, v[j]));
      } else {
        T* out = ws + R.x[L];
#pragma unroll
        for (int j = 0; j < C; ++j)
          if (j <= je) out[base + j] = tfma(-ch[j], Xt, tfma(-ah[j], Lv, v[j]));
      }
    }
    __syncthreads();
    if constexpr (STAGE) {
      T* out = ws + R.x[L];
      for (int q = tid; q < int(M); q += NT) out[q] = S[U::sk(q)];
      __syncthreads();
    }
  }
}

#define REG_SWEEP(T, DT, NT, C)                                                               \
  reg.push_back({K_BTCS_REDUCE, DT, NT, C, 1,                                                 \
                 reinterpret_cast<const void*>(&k_ml_sweep0<T, NT, C, false>),               \
                 Sweep0Smem<T, NT, C>::bytes(false)});                                        \
  reg.push_back({K_BTCS_REDUCE, DT, NT, C, 0,                                                 \
                 reinterpret_cast<const void*>(&k_ml_sweep<T, NT, C, false, false>),         \
                 UpperSmem<T, NT, C>::bytes()});                                              \
  reg.push_back({K_BTCS_RECOVER, DT, NT, C, 1,                                                \
                 reinterpret_cast<const void*>(&k_ml_sweep0<T, NT, C, true>),                \
                 Sweep0Smem<T, NT, C>::bytes(true)});                                         \
  reg.push_back({K_BTCS_RECOVER, DT, NT, C, 0,                                                \
                 reinterpret_cast<const void*>(&k_ml_sweep<T, NT, C, false, true>),          \
                 UpperSmem<T, NT, C>::bytes()});
// level-0 sweeps of the implicit variants: exact = 2 + variant (1 CN, 2
// Picard, 3 Newton)
#define REG_SWEEPV1(T, DT, NT, C, VAR)                                                         \
  reg.push_back({K_BTCS_REDUCE, DT, NT, C, 2 + VAR,                                           \
                 reinterpret_cast<const void*>(&k_ml_sweep0<T, NT, C, false, VAR>),          \
                 Sweep0Smem<T, NT, C>::bytes(false, VAR >= 2)});                              \
  reg.push_back({K_BTCS_RECOVER, DT, NT, C, 2 + VAR,                                          \
                 reinterpret_cast<const void*>(&k_ml_sweep0<T, NT, C, true, VAR>),           \
                 Sweep0Smem<T, NT, C>::bytes(true, VAR >= 2)});
#define REG_SWEEPV(T, DT, NT, C)                                                         \
  REG_SWEEPV1(T, DT, NT, C, 1) REG_SWEEPV1(T, DT, NT, C, 2) REG_SWEEPV1(T, DT, NT, C, 3) \
  REG_SWEEPV1(T, DT, NT, C, 4)
#define REG_TOP(T, DT, NT, C) \
  reg.push_back({K_BTCS_TOP, DT, NT, C, 0, reinterpret_cast<const void*>(&k_ml_top<T, NT, C>), \
                 (NT * C >= 2048) ? UpperSmem<T, NT, C>::bytes() : 0});
#define REG_COPY(T, DT, NT, C) \
  reg.push_back({K_BTCS_TOP, DT, NT, C, 1, reinterpret_cast<const void*>(&k_ml_copy<T, NT, C>), 0});

void register_multilevel(std::vector<KernelEntry>& reg) {
  REG_SWEEP(float, 0, 256, 16) REG_SWEEP(float, 0, 128, 8)
  REG_SWEEP(double, 1, 256, 8) REG_SWEEP(double, 1, 128, 4)
  REG_SWEEPV(float, 0, 256, 16) REG_SWEEPV(double, 1, 256, 8)
  REG_TOP(float, 0, 32, 1) REG_TOP(float, 0, 32, 4) REG_TOP(float, 0, 128, 8)
  REG_TOP(float, 0, 256, 16)
  REG_TOP(double, 1, 32, 1) REG_TOP(double, 1, 32, 4) REG_TOP(double, 1, 128, 8)
  REG_TOP(double, 1, 256, 8)
  REG_COPY(float, 0, 256, 16) REG_COPY(double, 1, 256, 8)
}

// ---------------------------------------------------------------------------
// host planning
// ---------------------------------------------------------------------------
namespace {
struct TopShape {
  int nt, c;
};
const TopShape kTop32[] = {{32, 1}, {32, 4}, {128, 8}, {256, 16}};
const TopShape kTop64[] = {{32, 1}, {32, 4}, {128, 8}, {256, 8}};
}  // namespace

static int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

burgers_status plan_multilevel(burgers_ctx* ctx, const burgers_batch* batch,
                               const std::vector<int64_t>& longs, Plan* p, int var, int iters) {
  const int dtype = batch->dtype;
  const int nit = (var == 2 || var == 3) ? iters : 1;
  const int snt = 256, sc = dtype == 0 ? 16 : 8;  // sweep shape
  const TopShape* tops = dtype == 0 ? kTop32 : kTop64;
  const int64_t top_cap = int64_t(tops[3].nt) * tops[3].c;
  // level 0: the staged BTCS sweeps, or the implicit variants' own rows
  const KernelEntry* red0 = find_kernel(K_BTCS_REDUCE, dtype, snt, sc, var ? 2 + var : 1);
  const KernelEntry* red1 = find_kernel(K_BTCS_REDUCE, dtype, snt, sc, 0);
  const KernelEntry* rec0 = find_kernel(K_BTCS_RECOVER, dtype, snt, sc, var ? 2 + var : 1);
  const KernelEntry* rec1 = find_kernel(K_BTCS_RECOVER, dtype, snt, sc, 0);
  if (!red0 || !red1 || !rec0 || !rec1) return set_error(BURGERS_EINVAL, "multi-level kernels missing");
  std::vector<MLRow> mrows;
  int64_t ws = 0;
  int Lmax = 0;
  int64_t smax = 0;
  auto al = [](int64_t x) { return (x + 63) & ~int64_t(63); };
  for (int64_t b : longs) {
    const burgers_instance& in = batch->inst[b];
    MLRow R;
    memset(&R, 0, sizeof R);
    R.offset = in.offset;
    R.nsteps = in.nsteps;
    R.r = in.dt / in.dx;
    R.s = in.nu * in.dt / (in.dx * in.dx);
    R.n = in.n;
    R.bc = in.bc;
    R.var = var;
    R.iters = nit;
    R.m[0] = in.n;
    int L = 0;
    while (L == 0 || R.m[L] > top_cap) {
      if (L == ML_MAXL) return set_error(BURGERS_EINVAL, "row too long for the multi-level solver");
      R.m[L + 1] = cdiv(R.m[L], sc);
      ++L;
    }
    if (R.m[L] < 2) return set_error(BURGERS_EINVAL, "row too short for the multi-level solver");
    R.levels = L;
    for (int l = 0; l < L; ++l) {
      R.ef[l] = ws;
      ws = al(ws + 6 * R.m[l + 1]);
    }
    for (int l = 1; l <= L; ++l) {
      R.x[l] = ws;
      ws = al(ws + R.m[l]);
    }
    Lmax = std::max(Lmax, L);
    smax = std::max<int64_t>(smax, in.nsteps);
    mrows.push_back(R);
  }
  p->ml_ws_elems = ws;
  p->ml_rows = int(mrows.size());
  int64_t span = 0;
  for (const MLRow& R : mrows) span = std::max<int64_t>(span, R.offset + R.n);
  span = (span + 63) & ~int64_t(63);  // aligned start of the Kahan buffer
  p->ml_span = span;
  // ping-pong copy of the rows (+ the Kahan terms for FP32, one byte a node in
  // a region of span elements), then for the
  // iterating variants two planes of e = w - u^n (read by one iteration,
  // written by it for the next)
  p->ml_e_off = dtype == 0 ? 2 * span : span;
  p->scratch_elems =
      std::max<int64_t>(p->scratch_elems, p->ml_e_off + ((nit > 1 || var == 4) ? 2 * span : 0));
  p->ml_bytes.resize(mrows.size() * sizeof(MLRow));
  memcpy(p->ml_bytes.data(), mrows.data(), p->ml_bytes.size());
  // item lists: sweeps of each level, then one list per top shape
  const int64_t tile = int64_t(snt) * sc;
  std::vector<std::pair<int, int>> level_items(static_cast<size_t>(Lmax));  // (begin, count)
  for (int l = 0; l < Lmax; ++l) {
    int begin = int(p->items.size());
    for (size_t q = 0; q < mrows.size(); ++q)
      if (mrows[q].levels > l) {
        int64_t tiles = cdiv(mrows[q].m[l], tile);
        for (int64_t t = 0; t < tiles; ++t) p->items.push_back(TileItem{int32_t(q), int32_t(t)});
      }
    level_items[size_t(l)] = {begin, int(p->items.size()) - begin};
  }
  struct TopGroup {
    const KernelEntry* k;
    int begin, count;
  };
  std::vector<TopGroup> tgroups;
  for (int ts = 0; ts < 4; ++ts) {
    int begin = int(p->items.size());
    for (size_t q = 0; q < mrows.size(); ++q) {
      const int64_t mt = mrows[q].m[mrows[q].levels];
      int pick = 0;
      while (pick < 3 && !(int64_t(tops[pick].nt) * tops[pick].c >= mt && tops[pick].c < mt)) ++pick;
      if (pick == ts) p->items.push_back(TileItem{int32_t(q), 0});
    }
    int cnt = int(p->items.size()) - begin;
    if (cnt > 0) {
      const KernelEntry* k = find_kernel(K_BTCS_TOP, dtype, tops[ts].nt, tops[ts].c, 0);
      if (!k) return set_error(BURGERS_EINVAL, "top kernel missing");
      tgroups.push_back(TopGroup{k, begin, cnt});
    }
  }
  auto grid_for = [&](const KernelEntry* k, int nitems) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k->fn, k->nt, k->dyn_smem) != cudaSuccess ||
        b < 1)
      b = 1;
    return std::max(1, std::min(nitems, ctx->sm_count * b));
  };
  for (int64_t s = 0; s < smax; ++s)
  for (int it = 0; it < nit; ++it) {
    for (int l = 0; l < Lmax; ++l) {
      Launch L;
      L.type = LAUNCH_ML;
      L.k = l == 0 ? red0 : red1;
      L.item_begin = level_items[size_t(l)].first;
      L.item_count = level_items[size_t(l)].second;
      L.grid = grid_for(L.k, L.item_count);
      L.level = l;
      L.step_base = s;
      L.iter = it;
      p->launches.push_back(L);
    }
    for (const TopGroup& g : tgroups) {
      Launch L;
      L.type = LAUNCH_ML;
      L.k = g.k;
      L.item_begin = g.begin;
      L.item_count = g.count;
      L.grid = g.count;
      L.level = 0;
      L.step_base = s;
      L.iter = it;
      p->launches.push_back(L);
    }
    for (int l = Lmax - 1; l >= 0; --l) {
      Launch L;
      L.type = LAUNCH_ML;
      L.k = l == 0 ? rec0 : rec1;
      L.item_begin = level_items[size_t(l)].first;
      L.item_count = level_items[size_t(l)].second;
      L.grid = grid_for(L.k, L.item_count);
      L.level = l;
      L.step_base = s;
      L.iter = it;
      p->launches.push_back(L);
    }
  }
  if (smax % 2 == 1 && var != 4) {  // the result is in the scratch copy (the transposed
                                    // solve writes only nu)
    Launch L;
    L.type = LAUNCH_ML;
    L.k = find_kernel(K_BTCS_TOP, dtype, snt, sc, 1);
    if (!L.k) return set_error(BURGERS_EINVAL, "copy kernel missing");
    L.item_begin = level_items[0].first;
    L.item_count = level_items[0].second;
    L.grid = grid_for(L.k, L.item_count);
    L.level = 0;
    L.step_base = smax;
    p->launches.push_back(L);
  }
  return BURGERS_OK;
}

cudaError_t enqueue_multilevel_launch(burgers_ctx* ctx, Plan* p, const Launch& L, void* u,
                                      cudaStream_t st) {
  char* base = static_cast<char*>(p->dev);
  void* ws = ctx->mlws.ptr;
  const size_t esz = p->dtype == 0 ? 4 : 8;
  void* u2 = ctx->scratch.ptr;
  void* lo = p->dtype == 0 ? static_cast<char*>(ctx->scratch.ptr) + size_t(p->ml_span) * esz : nullptr;
  const MLRow* rows = reinterpret_cast<const MLRow*>(base + p->ml_off);
  const TileItem* items = reinterpret_cast<const TileItem*>(base + p->items_off) + L.item_begin;
  // the staged sweeps copy row records in 16-byte pieces
  if (reinterpret_cast<uintptr_t>(rows) & 15) return cudaErrorMisalignedAddress;
  int ni = L.item_count, level = L.level, iter = L.iter;
  int64_t step = L.step_base;
  // e planes of the iterating variants (unused by the other launches)
  void* ea = static_cast<char*>(ctx->scratch.ptr) + size_t(p->ml_e_off) * esz;
  void* eb = static_cast<char*>(ea) + size_t(p->ml_span) * esz;
  void* args[] = {&u, &u2, &lo, &ws, &rows, &items, &ni, &level, &step, &iter, &ea, &eb};
  return cudaLaunchKernel(L.k->fn, dim3(L.grid), dim3(L.k->nt), args, L.k->dyn_smem, st);
}

}  // namespace burgers
