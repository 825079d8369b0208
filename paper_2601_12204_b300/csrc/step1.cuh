// step1.cuh -- the one-step-per-HBM-pass explicit update of one tile (K = 1
// streaming), shared by the per-tile kernel k_explicit_step1 (explicit.cu)
// and the bulk-copy kernel k_explicit_step1_bulk (step1_bulk.cu), plus the
// packing of the FP32 compensation bytes.
#pragma once

#include <stdint.h>

#include "common.cuh"
#include "kernels.h"

namespace burgers {

// C compensation bytes from p: the widest aligned vector loads (16, 8 or 4
// bytes), else byte by byte. STREAM: evict-first loads of data read once.
template <int C, bool STREAM>
__device__ __forceinline__ void load_bytes(signed char (&q)[C], const signed char* p) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  auto unpack = [&](int at, unsigned w) {
#pragma unroll
    for (int e = 0; e < 4; ++e) q[at + e] = static_cast<signed char>(w >> (8 * e));
  };
  if (C % 16 == 0 && (a & 15) == 0) {
#pragma unroll
    for (int k = 0; k < C / 16; ++k) {
      const uint4* vp = reinterpret_cast<const uint4*>(p) + k;
      const uint4 w = STREAM ? __ldcs(vp) : __ldg(vp);
      unpack(16 * k, w.x); unpack(16 * k + 4, w.y); unpack(16 * k + 8, w.z); unpack(16 * k + 12, w.w);
    }
  } else if (C % 8 == 0 && (a & 7) == 0) {
#pragma unroll
    for (int k = 0; k < C / 8; ++k) {
      const uint2* vp = reinterpret_cast<const uint2*>(p) + k;
      const uint2 w = STREAM ? __ldcs(vp) : __ldg(vp);
      unpack(8 * k, w.x); unpack(8 * k + 4, w.y);
    }
  } else if (C % 4 == 0 && (a & 3) == 0) {
#pragma unroll
    for (int k = 0; k < C / 4; ++k) {
      const unsigned* vp = reinterpret_cast<const unsigned*>(p) + k;
      unpack(4 * k, STREAM ? __ldcs(vp) : __ldg(vp));
    }
  } else {
#pragma unroll
    for (int j = 0; j < C; ++j) q[j] = p[j];
  }
}

// Packs 4 compensation bytes into a word (byte e at bits 8e..8e+7).
__device__ __forceinline__ unsigned pack4(signed char a, signed char b, signed char c,
                                          signed char d) {
  return (unsigned(a) & 0xffu) | ((unsigned(b) & 0xffu) << 8) | ((unsigned(c) & 0xffu) << 16) |
         ((unsigned(d) & 0xffu) << 24);
}

// Stores C compensation bytes to p with the widest aligned vector stores.
template <int C, bool STREAM>
__device__ __forceinline__ void store_bytes(signed char* p, const signed char (&q)[C]) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  if (C % 16 == 0 && (a & 15) == 0) {
#pragma unroll
    for (int k = 0; k < C / 16; ++k) {
      const int b = 16 * k;
      const uint4 w = make_uint4(pack4(q[b], q[b + 1], q[b + 2], q[b + 3]),
                                 pack4(q[b + 4], q[b + 5], q[b + 6], q[b + 7]),
                                 pack4(q[b + 8], q[b + 9], q[b + 10], q[b + 11]),
                                 pack4(q[b + 12], q[b + 13], q[b + 14], q[b + 15]));
      if (STREAM) __stcs(reinterpret_cast<uint4*>(p) + k, w);
      else reinterpret_cast<uint4*>(p)[k] = w;
    }
  } else if (C % 8 == 0 && (a & 7) == 0) {
#pragma unroll
    for (int k = 0; k < C / 8; ++k) {
      const int b = 8 * k;
      const uint2 w = make_uint2(pack4(q[b], q[b + 1], q[b + 2], q[b + 3]),
                                 pack4(q[b + 4], q[b + 5], q[b + 6], q[b + 7]));
      if (STREAM) __stcs(reinterpret_cast<uint2*>(p) + k, w);
      else reinterpret_cast<uint2*>(p)[k] = w;
    }
  } else if (C % 4 == 0 && (a & 3) == 0) {
#pragma unroll
    for (int k = 0; k < C / 4; ++k) {
      const unsigned w = pack4(q[4 * k], q[4 * k + 1], q[4 * k + 2], q[4 * k + 3]);
      if (STREAM) __stcs(reinterpret_cast<unsigned*>(p) + k, w);
      else reinterpret_cast<unsigned*>(p)[k] = w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < C; ++j) p[j] = q[j];
  }
}

// One forward-Euler step (Eq. 21) of tile ti.tile of row ti.row, NT*C nodes,
// from src into dst: a thread updates C consecutive nodes read and written as
// 16-byte vectors when the row's start allows it. The two neighbours of a
// thread's nodes come from the adjacent lanes by shuffle, and from memory at
// warp and row edges. FP32 moves 4 bytes of state and 1 byte of compensation
// per node each way (10 bytes per cell-update). Rows with step_base >= nsteps
// are copied through.
template <typename T, int NT, int C>
__device__ __forceinline__ void step1_tile(const T* __restrict__ src, T* __restrict__ dst,
                                           const signed char* __restrict__ lo_src,
                                           signed char* __restrict__ lo_dst,
                                           const RowDesc* __restrict__ rows, const TileItem ti,
                                           int64_t step_base) {
  using V = typename Vec16<T>::type;
  constexpr int VE = 16 / int(sizeof(T));
  static_assert(C % VE == 0, "whole vectors per thread");
  constexpr bool KL = Kahan<T>::on;
  const int lane = threadIdx.x & 31;
  {
    const RowDesc rd = rows[ti.row];
    const int64_t n = rd.n;
    const int64_t g0 = int64_t(ti.tile) * (NT * C) + int64_t(threadIdx.x) * C;
    const int cnt = g0 >= n ? 0 : (n - g0 < C ? int(n - g0) : C);
    const T* srow = src + rd.offset;
    T* drow = dst + rd.offset;
    const signed char* lsrc = KL ? lo_src + rd.offset : nullptr;
    signed char* ldst = KL ? lo_dst + rd.offset : nullptr;
    // vector path: 16-byte state vectors, the compensation bytes as the widest
    // aligned words
    const bool vec = cnt == C && (reinterpret_cast<uintptr_t>(srow + g0) & 15) == 0 &&
                     (reinterpret_cast<uintptr_t>(drow + g0) & 15) == 0;
    T v[C], lo[C];
    signed char q[C];
    if (vec) {
#pragma unroll
      for (int qv = 0; qv < C / VE; ++qv) {
        const V w = __ldcs(reinterpret_cast<const V*>(srow + g0) + qv);
        const T* wp = reinterpret_cast<const T*>(&w);
#pragma unroll
        for (int e = 0; e < VE; ++e) v[qv * VE + e] = wp[e];
      }
      if constexpr (KL) load_bytes<C, true>(q, lsrc + g0);
    } else {
#pragma unroll
      for (int j = 0; j < C; ++j) {
        v[j] = j < cnt ? srow[g0 + j] : T(0);
        q[j] = (KL && j < cnt) ? lsrc[g0 + j] : static_cast<signed char>(0);
      }
    }
#pragma unroll
    for (int j = 0; j < C; ++j) lo[j] = KL ? T(lo8_decode(float(v[j]), q[j])) : T(0);
    // neighbours: the adjacent lane's edge node when it is the adjacent node
    T left = shfl_up(v[C - 1], 1);
    T right = shfl_down(v[0], 1);
    const bool per = rd.bc == BC_PERIODIC;
    if (cnt > 0) {
      if (lane == 0 || g0 == 0) left = g0 > 0 ? srow[g0 - 1] : (per ? srow[n - 1] : T(0));
      if (lane == 31 || cnt < C || g0 + C == n)
        right = g0 + cnt < n ? srow[g0 + cnt] : (per ? srow[0] : T(0));
    }
    if (cnt == 0) return;
    if (step_base < rd.nsteps) {
      const RowCoefs<T> cf = row_coefs(rd, T(0));
      // node-by-node tests only where the thread holds the row's end or a
      // Dirichlet end node
      const bool plain = cnt == C && (per || (g0 != 0 && g0 + C < n));
      T prev = left;
#pragma unroll
      for (int j = 0; j < C; ++j) {
        const T cur = v[j];
        const T ur = (plain || j + 1 < cnt) ? (j + 1 < C ? v[j + 1] : right) : right;
        T l0 = lo[j];
        const T nv = explicit_update(cur, prev, ur, cf.r, cf.h, cf.s, l0);
        const int64_t gi = g0 + j;
        const bool keep = !plain && (j >= cnt || (!per && (gi == 0 || gi == n - 1)));
        if (!keep) { v[j] = nv; lo[j] = l0; }
        prev = cur;
      }
    }
    if constexpr (KL) {
#pragma unroll
      for (int j = 0; j < C; ++j) q[j] = lo8_encode(float(v[j]), float(lo[j]));
    }
    if (vec) {
#pragma unroll
      for (int qv = 0; qv < C / VE; ++qv) {
        V w;
        T* wp = reinterpret_cast<T*>(&w);
#pragma unroll
        for (int e = 0; e < VE; ++e) wp[e] = v[qv * VE + e];
        __stcs(reinterpret_cast<V*>(drow + g0) + qv, w);
      }
      if constexpr (KL) store_bytes<C, true>(ldst + g0, q);
    } else {
#pragma unroll
      for (int j = 0; j < C; ++j)
        if (j < cnt) {
          drow[g0 + j] = v[j];
          if constexpr (KL) ldst[g0 + j] = q[j];
        }
    }
  }
}

}  // namespace burgers
