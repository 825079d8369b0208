// step1_bulk.cu -- one explicit step per HBM pass (K = 1 streaming, Eq. 21)
// over whole tiles moved by the tensor memory accelerator.
//
// A persistent CTA walks its tiles (items blockIdx.x, blockIdx.x + gridDim.x,
// ...) through a ring of S shared-memory stages. One thread issues the 1D bulk
// copies (cp.async.bulk) of a tile's state (W values) and, for FP32, its W
// compensation bytes into a stage, completing on the stage's mbarrier; the
// CTA computes the tile in place in shared memory and the same thread writes
// the stage back with bulk stores. Loads for the next S - 1 tiles are in flight
// while a tile computes, so a CTA keeps tens of kilobytes of HBM traffic
// outstanding with a handful of instructions. Tiles that are not whole, or
// rows whose start is not 16-byte aligned, go through step1_tile after the
// ring has drained (the plan puts those items last).
//
// Thread t owns vectors t, t + NT, ..., t + (G-1) NT of the tile (VE values
// each, 16 bytes), so a warp's shared-memory accesses are consecutive 16-byte
// words; a vector's neighbour values come from the adjacent lanes by shuffle
// and, at warp edges, from shared memory (all reads finish before the writes
// start); the two values beyond the tile come from global memory.
//
// Every wait is bounded: an mbarrier that has not completed after about two
// seconds sets bit 0 of *err, the CTA stops issuing copies, waits (bounded)
// for those it has in flight and for its stores, and returns.
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "common.cuh"
#include "kernels.h"
#include "step1.cuh"

namespace burgers {

namespace {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Waits for phase `parity` of *bar for at most limit_ns; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}
// 1D bulk copy global -> this CTA's shared memory, completing on *bar.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// 1D bulk copy shared -> global (bulk async-group completion).
__device__ __forceinline__ void bulk_store(void* dst, const void* src, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
               "r"(smem_addr(src)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// Waits until at most one committed store group still reads shared memory.
__device__ __forceinline__ void bulk_wait_read1() {
  asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}
// Waits until every committed store group has completed.
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}
// Orders this thread's generic-proxy shared-memory writes before later
// async-proxy (bulk copy) reads of them.
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;

}  // namespace

// Stage bytes of one tile: W values plus (FP32) W compensation bytes.
template <typename T, int NT, int G>
constexpr size_t bulk_stage_bytes() {
  return size_t(NT) * G * (16 / sizeof(T)) * (sizeof(T) + (Kahan<T>::on ? 1 : 0));
}

template <typename T, int NT, int G, int S>
__global__ void __launch_bounds__(NT) k_explicit_step1_bulk(
    const T* __restrict__ src, T* __restrict__ dst, const signed char* __restrict__ lo_src,
    signed char* __restrict__ lo_dst, const RowDesc* __restrict__ rows,
    const TileItem* __restrict__ items, int nbulk, int nitems, int64_t step_base,
    int* __restrict__ err) {
  using V = typename Vec16<T>::type;
  constexpr int VE = 16 / int(sizeof(T));
  constexpr int C = G * VE;  // values a thread updates
  constexpr int W = NT * C;  // values a tile holds
  constexpr bool KL = Kahan<T>::on;
  constexpr unsigned UB = unsigned(W * sizeof(T)), LB = KL ? unsigned(W) : 0u;
  constexpr size_t SB = bulk_stage_bytes<T, NT, G>();
  static_assert(UB % 16 == 0 && SB % 16 == 0, "bulk copies move multiples of 16 bytes");
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ __align__(8) uint64_t bar[S];
  const int tid = threadIdx.x, lane = tid & 31;
  auto stage_u = [&](int s) { return reinterpret_cast<T*>(dsm + size_t(s) * SB); };
  auto stage_lo = [&](int s) { return reinterpret_cast<signed char*>(dsm + size_t(s) * SB + UB); };

  if (tid == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
    mbar_init_fence();
  }
  __syncthreads();
  const int M = nbulk > int(blockIdx.x) ? (nbulk - 1 - int(blockIdx.x)) / int(gridDim.x) + 1 : 0;
  auto issue = [&](int m) {  // thread 0: tile m of this CTA into stage m % S
    const TileItem ti = items[blockIdx.x + int64_t(m) * gridDim.x];
    const int64_t g = rows[ti.row].offset + int64_t(ti.tile) * W;
    const int s = m % S;
    mbar_expect_tx(&bar[s], UB + LB);
    bulk_load(stage_u(s), src + g, UB, &bar[s]);
    if constexpr (KL) bulk_load(stage_lo(s), lo_src + g, LB, &bar[s]);
  };
  int issued = 0;
  if (tid == 0)
    for (; issued < S && issued < M; ++issued) issue(issued);

  bool failed = false;
  int m = 0;
  for (; m < M; ++m) {
    const int s = m % S;
    const bool ok = mbar_wait(&bar[s], unsigned(m / S) & 1u, WAIT_LIMIT_NS);
    if (__syncthreads_or(!ok)) { failed = true; break; }
    const TileItem ti = items[blockIdx.x + int64_t(m) * gridDim.x];
    const RowDesc rd = rows[ti.row];
    const int64_t n = rd.n, t0 = int64_t(ti.tile) * W;
    const bool per = rd.bc == BC_PERIODIC;
    T* su = stage_u(s);
    signed char* sl = stage_lo(s);
    T v[G][VE], lo[G][VE], left[G], right[G];
    // reads: the thread's vectors, their compensation bytes, the edge values
#pragma unroll
    for (int k = 0; k < G; ++k) {
      const int vi = tid + NT * k;  // vector index in the tile
      const V w = reinterpret_cast<const V*>(su)[vi];
      const T* wp = reinterpret_cast<const T*>(&w);
#pragma unroll
      for (int e = 0; e < VE; ++e) v[k][e] = wp[e];
      if constexpr (KL) {
        const unsigned q4 = reinterpret_cast<const unsigned*>(sl)[vi];
#pragma unroll
        for (int e = 0; e < VE; ++e)
          lo[k][e] = T(lo8_decode(float(v[k][e]), static_cast<signed char>(q4 >> (8 * e))));
      } else {
#pragma unroll
        for (int e = 0; e < VE; ++e) lo[k][e] = T(0);
      }
      left[k] = shfl_up(v[k][VE - 1], 1);
      right[k] = shfl_down(v[k][0], 1);
      const int first = VE * vi;  // tile index of the vector's first value
      if (lane == 0) {
        if (first > 0) left[k] = su[first - 1];
        else left[k] = t0 > 0 ? src[rd.offset + t0 - 1] : (per ? src[rd.offset + n - 1] : T(0));
      }
      if (lane == 31) {
        if (first + VE < W) right[k] = su[first + VE];
        else right[k] = t0 + W < n ? src[rd.offset + t0 + W] : (per ? src[rd.offset] : T(0));
      }
    }
    __syncthreads();  // every read of the stage is done before it is overwritten
    if (step_base < rd.nsteps) {
      const RowCoefs<T> cf = row_coefs(rd, T(0));
      // a Dirichlet row's held end nodes lie only in its first and last tile
      const bool ends = !per && (t0 == 0 || t0 + W >= n);
      auto update = [&](auto ends_tag) {
        constexpr bool E = decltype(ends_tag)::value;
#pragma unroll
        for (int k = 0; k < G; ++k) {
          const int first = VE * (tid + NT * k);
          T prev = left[k];
#pragma unroll
          for (int e = 0; e < VE; ++e) {
            const T cur = v[k][e];
            const T ur = e + 1 < VE ? v[k][e + 1] : right[k];
            T l0 = lo[k][e];
            const T nv = explicit_update(cur, prev, ur, cf.r, cf.h, cf.s, l0);
            bool held = false;
            if constexpr (E) {
              const int64_t gi = t0 + first + e;
              held = gi == 0 || gi == n - 1;
            }
            if (!held) { v[k][e] = nv; lo[k][e] = l0; }
            prev = cur;
          }
        }
      };
      if (ends) update(std::true_type{});
      else update(std::false_type{});
    }
#pragma unroll
    for (int k = 0; k < G; ++k) {
      const int vi = tid + NT * k;
      V w;
      T* wp = reinterpret_cast<T*>(&w);
#pragma unroll
      for (int e = 0; e < VE; ++e) wp[e] = v[k][e];
      reinterpret_cast<V*>(su)[vi] = w;
      if constexpr (KL) {
        unsigned q4 = 0;
#pragma unroll
        for (int e = 0; e < VE; ++e)
          q4 |= (unsigned(lo8_encode(float(v[k][e]), float(lo[k][e]))) & 0xffu) << (8 * e);
        reinterpret_cast<unsigned*>(sl)[vi] = q4;
      }
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      const int64_t g = rd.offset + t0;
      bulk_store(dst + g, su, UB);
      if constexpr (KL) bulk_store(lo_dst + g, sl, LB);
      bulk_commit();
      // the stage of the previous tile is free once its stores have read it
      if (m >= 1 && issued < M) {
        bulk_wait_read1();
        issue(issued);
        ++issued;
      }
    }
  }
  if (failed) {
    // stop; wait (bounded) for the loads this CTA still has in flight
    if (tid == 0) {
      atomicOr(err, 1);
      for (int q = m; q < issued; ++q) (void)mbar_wait(&bar[q % S], unsigned(q / S) & 1u, WAIT_LIMIT_NS);
    }
  }
  if (tid == 0) bulk_wait_all();
  __syncthreads();
  if (failed) return;
  // tiles that are not whole (row tails) or not bulk-aligned
  for (int it = nbulk + int(blockIdx.x); it < nitems; it += int(gridDim.x))
    step1_tile<T, NT, C>(src, dst, lo_src, lo_dst, rows, items[it], step_base);
}

#define REG_STEP1_BULK(T, DT, NT, G, S)                                                       \
  reg.push_back({K_EXPLICIT_STEP1_BULK, DT, NT, G * int(16 / sizeof(T)), S,                  \
                 reinterpret_cast<const void*>(&k_explicit_step1_bulk<T, NT, G, S>),          \
                 size_t(S) * bulk_stage_bytes<T, NT, G>()});

// kind K_EXPLICIT_STEP1_BULK: c = values a thread updates (the tile is nt * c,
// as for K_EXPLICIT_STEP1), `exact` holds the number of stages
void register_step1_bulk(std::vector<KernelEntry>& reg) {
  REG_STEP1_BULK(float, 0, 256, 4, 4)
  REG_STEP1_BULK(float, 0, 128, 4, 6)
  REG_STEP1_BULK(float, 0, 512, 2, 4)
  REG_STEP1_BULK(float, 0, 512, 2, 3)
  REG_STEP1_BULK(double, 1, 256, 2, 4)
}

}  // namespace burgers
