// btcs_thomas.cu -- lagged BTCS steps (Sec. 2.4, Eq. 23) of many short rows,
// one thread per row, each solving its tridiagonal system with the plain
// Thomas elimination (cyclic rows through Sherman-Morrison, Eq. 18).
//
// The partitioned resident kernel pays, every step, a reduced solve on one
// warp (parallel cyclic reduction and the Sherman-Morrison factor) and
// three CTA barriers, whatever the row length; for rows of a few hundred
// nodes that fixed cost dominates. Here a CTA of NT threads takes NT rows
// (rows are cost-sorted, so neighbours have similar lengths and step counts)
// and each thread runs its own row's steps with no barrier and no exchange.
//
// Layout: at entry the CTA transposes its rows from the caller's buffer
// (row-major, coalesced reads) into an interleaved layout [i][t] (node i of
// the CTA's thread t at i * NT + t), so that at every step the warp's 32
// threads touch one contiguous line per node index; the sweep coefficients
// (ch, dh and zh, the eliminated super-diagonal and the two right-hand sides)
// use the same layout. MODE (below) says which of these live in shared memory
// and which in a context workspace (L2 resident). At exit the rows are
// transposed back.
//
// One thread per row exposes only as many elimination chains as there are
// rows, so this kernel is the faster one for many short rows (thousands of
// rows of up to 64 nodes FP32, 128 FP64); the partitioned kernel keeps the
// rest (pick_thomas in api.cu has the measured crossover).
//
// A step, in the increment form of the resident kernel (A(u^n) delta =
// Delta(u^n), u += delta): one forward pass that assembles row i from
// u_{i-1}, u_i, u_{i+1} and eliminates it; one backward pass that forms the
// increment and adds it, Kahan-compensated in FP32. Periodic rows split the
// corners off as in Eq. 18 (gamma = -d_0, v = e_0 + (l_0/gamma) e_{n-1}) and
// solve T y = rhs and T z = u together; the correction factor
// (v.y)/(1 + v.z) needs y_0 and z_0 before the backward pass, which the
// forward pass accumulates as y_0 = sum_k prod_{j<k} (-ch_j) dh_k (the
// back-substitution unrolled), so the backward pass applies x = y - fac z
// directly. The denominator is formed in extended precision (sm_factor).
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "btcs_common.cuh"
#include "common.cuh"
#include "kernels.h"

namespace burgers {

// Where a CTA keeps its rows during the steps (PLANE = NMAX * NT values):
//   MODE 0: state (and FP32 Kahan terms) in the workspace, the three
//           coefficient planes in shared memory;
//   MODE 1: everything in the workspace (L2 resident), shared memory only
//           for the transposes;
//   MODE 2: everything in shared memory (no global traffic between the
//           transposes at entry and exit; fewest rows per SM).
template <typename T>
constexpr int thomas_state_planes() { return Kahan<T>::on ? 2 : 1; }
template <typename T, int NT, int NMAX, int MODE>
constexpr size_t thomas_ws_per_cta() {
  return MODE == 2 ? 0
                   : size_t(NMAX) * NT * (thomas_state_planes<T>() + (MODE == 1 ? 3 : 0));
}
template <typename T, int NT, int NMAX, int MODE>
constexpr size_t thomas_dsm() {
  return MODE == 1   ? size_t(NT / 32) * 32 * 33 * sizeof(T)
         : MODE == 0 ? size_t(3) * NMAX * NT * sizeof(T)
                     : size_t(3 + thomas_state_planes<T>()) * NMAX * NT * sizeof(T);
}

// Row i of the lagged BTCS system (Sec. 2.4): l, d, c from a = u_i and the
// explicit increment of Eq. 21 with the same coefficients as right-hand side.
template <typename T>
struct ThomasRow {
  T l, d, c, rhs;
};
template <typename T>
__device__ __forceinline__ ThomasRow<T> thomas_row(T am, T a, T ap, T r, T s, T ds1) {
  const T ra = r * a;
  ThomasRow<T> w;
  w.l = -s - tmax(ra, T(0));
  w.c = tmin(ra, T(0)) - s;
  w.d = ds1 + tabs(ra);
  w.rhs = tfma(w.l, a - am, -w.c * (ap - a));
  return w;
}

// One step of one row, thread-private. pu, plo: the row's state and Kahan
// terms; pch, pdh, pzh: its coefficient planes; all with node stride NT.
// Rows 0 and n-1 (the corner split of periodic rows, the held ends of
// Dirichlet rows) are peeled off; rows 1 .. n-2 run in register blocks whose
// loads are issued one block ahead.
template <typename T, int NT, int BCT>
__device__ __forceinline__ void thomas_step(T* __restrict__ pu, T* __restrict__ plo,
                                            T* __restrict__ pch, T* __restrict__ pdh,
                                            T* __restrict__ pzh, int n, T r, T s) {
  constexpr bool KL = Kahan<T>::on;
  constexpr bool PER = BCT == BC_PERIODIC;
  constexpr int BF = sizeof(T) == 4 ? 8 : 4;  // forward block
  constexpr int BB = sizeof(T) == 4 ? 4 : 2;  // backward block
  const T ds1 = T(1) + T(2) * s;
  const int last = n - 1;
  // ---- forward
  T chp, dhp, zhp = T(0), fa = T(0), sy = T(0), sz = T(0), pr = T(1);
  T am = pu[0];
  {
    const T a = am, ap = pu[NT];
    if constexpr (PER) {
      // gamma = -d_0: T has 2 d_0 and no corner; u_sm = gamma e_0 + c_{n-1} e_{n-1}
      const ThomasRow<T> w = thomas_row(pu[size_t(last) * NT], a, ap, r, s, ds1);
      const T gam = -w.d;
      fa = w.l * recip(gam);
      const T inv = recip(w.d - gam);
      chp = w.c * inv;
      dhp = w.rhs * inv;
      zhp = gam * inv;
      pzh[0] = zhp;
      sy = dhp;
      sz = zhp;
      pr = -chp;
    } else {  // held end: identity row, zero increment
      chp = T(0);
      dhp = T(0);
    }
    pch[0] = chp;
    pdh[0] = dhp;
  }
  // rows 1 .. n-2
  {
    T cur[BF + 1], nxt[BF + 1];
    const int i_end = last;  // exclusive
#pragma unroll
    for (int j = 0; j <= BF; ++j) cur[j] = pu[size_t(min(1 + j, last)) * NT];
    for (int i0 = 1; i0 < i_end; i0 += BF) {
      if (i0 + BF < i_end) {
#pragma unroll
        for (int j = 0; j <= BF; ++j) nxt[j] = pu[size_t(min(i0 + BF + j, last)) * NT];
      }
      auto body = [&](auto full_tag) {
        constexpr bool FULL = decltype(full_tag)::value;
        T* bch = pch + size_t(i0) * NT;
        T* bdh = pdh + size_t(i0) * NT;
        T* bzh = pzh + size_t(i0) * NT;
#pragma unroll
        for (int j = 0; j < BF; ++j) {
          if (!FULL && i0 + j >= i_end) break;
          const ThomasRow<T> w = thomas_row(am, cur[j], cur[j + 1], r, s, ds1);
          const T inv = recip(tfma(-w.l, chp, w.d));
          const T ch = w.c * inv;
          const T dh = tfma(-w.l, dhp, w.rhs) * inv;
          bch[j * NT] = ch;
          bdh[j * NT] = dh;
          if constexpr (PER) {
            const T zh = (-w.l * zhp) * inv;
            bzh[j * NT] = zh;
            sy = tfma(pr, dh, sy);  // y_0 and z_0: the back-substitution unrolled
            sz = tfma(pr, zh, sz);
            pr = -ch * pr;
            zhp = zh;
          }
          chp = ch;
          dhp = dh;
          am = cur[j];
        }
      };
      if (i0 + BF <= i_end) body(std::true_type{});
      else body(std::false_type{});
#pragma unroll
      for (int j = 0; j <= BF; ++j) cur[j] = nxt[j];
    }
  }
  {  // row n-1
    const T a = pu[size_t(last) * NT];
    if constexpr (PER) {  // T has d - c l_0 / gamma and no corner
      const ThomasRow<T> w = thomas_row(am, a, pu[0], r, s, ds1);
      const T inv = recip(tfma(-w.l, chp, w.d - w.c * fa));
      dhp = tfma(-w.l, dhp, w.rhs) * inv;
      zhp = tfma(-w.l, zhp, w.c) * inv;
      pzh[size_t(last) * NT] = zhp;
      sy = tfma(pr, dhp, sy);
      sz = tfma(pr, zhp, sz);
    } else {
      dhp = T(0);
    }
    pch[size_t(last) * NT] = T(0);
    pdh[size_t(last) * NT] = dhp;
  }
  // y_{n-1} = dh_{n-1}, z_{n-1} = zh_{n-1}: the correction (v.y)/(1 + v.z)
  const T fac = PER ? sm_factor(fa, sy, dhp, sz, zhp) : T(0);
  // ---- backward: x = y - fac z added to the state (Kahan in FP32)
  auto add = [&](T* u, T* lo, T x) {
    T l0 = KL ? *lo : T(0);
    *u = comp_add(*u, x, l0);
    if constexpr (KL) *lo = l0;
  };
  T yn = dhp, zn = zhp;  // row n-1
  if constexpr (PER) add(pu + size_t(last) * NT, plo + size_t(last) * NT, tfma(-fac, zn, yn));
  {
    // rows n-2 .. 1 in blocks [i0 - BB + 1, i0]
    T bch[BB], bdh[BB], bzh[BB], bu[BB], blo[BB];
    T nch[BB], ndh[BB], nzh[BB], nu[BB], nlo[BB];
    auto load = [&](int i0, T (&ch)[BB], T (&dh)[BB], T (&zh)[BB], T (&uu)[BB], T (&ll)[BB]) {
#pragma unroll
      for (int j = 0; j < BB; ++j) {
        const size_t o = size_t(max(i0 - j, 1)) * NT;
        ch[j] = pch[o];
        dh[j] = pdh[o];
        zh[j] = PER ? pzh[o] : T(0);
        uu[j] = pu[o];
        ll[j] = KL ? plo[o] : T(0);
      }
    };
    if (last - 1 >= 1) load(last - 1, bch, bdh, bzh, bu, blo);
    for (int i0 = last - 1; i0 >= 1; i0 -= BB) {
      if (i0 - BB >= 1) load(i0 - BB, nch, ndh, nzh, nu, nlo);
      auto body = [&](auto full_tag) {
        constexpr bool FULL = decltype(full_tag)::value;
        T* bpu = pu + size_t(i0) * NT;
        T* bplo = plo + size_t(i0) * NT;
#pragma unroll
        for (int j = 0; j < BB; ++j) {
          if (!FULL && i0 - j < 1) break;
          const T y = tfma(-bch[j], yn, bdh[j]);
          T x = y;
          if constexpr (PER) {
            const T z = tfma(-bch[j], zn, bzh[j]);
            x = tfma(-fac, z, y);
            zn = z;
          }
          T l0 = blo[j];
          const T nv = comp_add(bu[j], x, l0);
          bpu[-j * NT] = nv;
          if constexpr (KL) bplo[-j * NT] = l0;
          yn = y;
        }
      };
      if (i0 - BB + 1 >= 1) body(std::true_type{});
      else body(std::false_type{});
#pragma unroll
      for (int j = 0; j < BB; ++j) {
        bch[j] = nch[j]; bdh[j] = ndh[j]; bzh[j] = nzh[j]; bu[j] = nu[j]; blo[j] = nlo[j];
      }
    }
  }
  if constexpr (PER) {  // row 0
    const T y = tfma(-pch[0], yn, pdh[0]);
    const T z = tfma(-pch[0], zn, pzh[0]);
    add(pu, plo, tfma(-fac, z, y));
  }
}

template <typename T, int NT, int NMAX, int MODE>
__global__ void __launch_bounds__(NT) k_btcs_thomas(T* __restrict__ u,
                                                    const RowDesc* __restrict__ rows, int count,
                                                    T* __restrict__ ws) {
  constexpr bool KL = Kahan<T>::on;
  constexpr size_t PLANE = size_t(NMAX) * NT;
  extern __shared__ __align__(16) unsigned char dsm[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int SP = thomas_state_planes<T>();
  T* wsb = ws + size_t(blockIdx.x) * thomas_ws_per_cta<T, NT, NMAX, MODE>();
  T* sm0 = reinterpret_cast<T*>(dsm);
  T* su = MODE == 2 ? sm0 : wsb;  // state, [i][t]
  T* slo = su + PLANE;             // FP32 Kahan terms, [i][t]
  T* cb = MODE == 1 ? wsb + SP * PLANE : (MODE == 2 ? sm0 + SP * PLANE : sm0);
  T* sch = cb;
  T* sdh = cb + PLANE;
  T* szh = cb + 2 * PLANE;
  const int row = int(blockIdx.x) * NT + tid;
  const bool active = row < count;
  RowDesc rd{};
  if (active) rd = rows[row];
  const int n = active ? rd.n : 0;
  const int64_t off = active ? rd.offset : 0;
  int nw = n;  // longest row of the warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nw = max(nw, __shfl_xor_sync(FULL_MASK, nw, o));
  // transposes go through a 32 x 33 tile per warp in the coefficient planes
  // (free before and after the steps), or at the start of shared memory
  T* tile = (MODE == 1 ? sm0 : cb) + warp * 32 * 33;

  // ---- rows -> interleaved workspace (through a 32 x 33 tile per warp)
  for (int j0 = 0; j0 < nw; j0 += 32) {
    for (int r = 0; r < 32; ++r) {
      const int64_t ro = shfl(off, r);
      const int rn = shfl(n, r);
      tile[r * 33 + lane] = j0 + lane < rn ? u[ro + j0 + lane] : T(0);
    }
    __syncwarp();
    for (int j = 0; j < 32 && j0 + j < NMAX; ++j) {
      su[size_t(j0 + j) * NT + tid] = tile[lane * 33 + j];
      if constexpr (KL) slo[size_t(j0 + j) * NT + tid] = T(0);
    }
    __syncwarp();
  }
  __syncthreads();  // the tiles share shared memory with the coefficient planes

  if (active && n >= 3) {
    const RowCoefs<T> cf = row_coefs(rd, T(0));
    for (int64_t st = 0; st < rd.nsteps; ++st) {
      if (rd.bc == BC_PERIODIC)
        thomas_step<T, NT, BC_PERIODIC>(su + tid, slo + tid, sch + tid, sdh + tid, szh + tid, n,
                                        cf.r, cf.s);
      else
        thomas_step<T, NT, BC_DIRICHLET>(su + tid, slo + tid, sch + tid, sdh + tid, szh + tid, n,
                                         cf.r, cf.s);
    }
  }
  __syncthreads();

  // ---- interleaved workspace -> rows
  for (int j0 = 0; j0 < nw; j0 += 32) {
    for (int j = 0; j < 32 && j0 + j < NMAX; ++j) tile[lane * 33 + j] = su[size_t(j0 + j) * NT + tid];
    __syncwarp();
    for (int r = 0; r < 32; ++r) {
      const int64_t ro = shfl(off, r);
      const int rn = shfl(n, r);
      if (j0 + lane < rn) u[ro + j0 + lane] = tile[r * 33 + lane];
    }
    __syncwarp();
  }
}

#define REG_THOMAS(T, DT, NT, NMAX, M)                                                  \
  reg.push_back({K_BTCS_THOMAS, DT, NT, NMAX, M,                                       \
                 reinterpret_cast<const void*>(&k_btcs_thomas<T, NT, NMAX, M>),        \
                 thomas_dsm<T, NT, NMAX, M>()});

// kind K_BTCS_THOMAS: nt threads (rows) per CTA, c = NMAX (the longest row a
// thread holds), exact = MODE (where the rows live during the steps)
void register_btcs_thomas(std::vector<KernelEntry>& reg) {
  REG_THOMAS(float, 0, 256, 32, 0) REG_THOMAS(float, 0, 256, 64, 0)
  REG_THOMAS(float, 0, 128, 128, 0) REG_THOMAS(float, 0, 64, 256, 0)
  REG_THOMAS(float, 0, 64, 128, 1) REG_THOMAS(float, 0, 64, 256, 1)
  REG_THOMAS(float, 0, 64, 512, 1) REG_THOMAS(float, 0, 64, 1024, 1)
  REG_THOMAS(float, 0, 64, 2048, 1)
  REG_THOMAS(float, 0, 256, 32, 2) REG_THOMAS(float, 0, 128, 64, 2)
  REG_THOMAS(float, 0, 64, 128, 2) REG_THOMAS(float, 0, 32, 256, 2)
  REG_THOMAS(double, 1, 128, 32, 0) REG_THOMAS(double, 1, 128, 64, 0)
  REG_THOMAS(double, 1, 64, 128, 0) REG_THOMAS(double, 1, 64, 64, 1)
  REG_THOMAS(double, 1, 64, 128, 1) REG_THOMAS(double, 1, 64, 256, 1)
  REG_THOMAS(double, 1, 64, 512, 1) REG_THOMAS(double, 1, 64, 1024, 1)
  REG_THOMAS(double, 1, 128, 32, 2) REG_THOMAS(double, 1, 64, 64, 2)
  REG_THOMAS(double, 1, 32, 128, 2)
}

size_t thomas_ws_values(int dtype, int nt, int nmax, int mode) {
  return mode == 2 ? 0 : size_t(nmax) * nt * ((dtype == 0 ? 2 : 1) + (mode == 1 ? 3 : 0));
}

}  // namespace burgers
