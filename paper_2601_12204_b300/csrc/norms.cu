// norms.cu -- FP64 reductions over rows: relative L2 / RMS error norms
// (Nomenclature "L2", Sec. 2.7.4) and the per-row max|u| of the CFL time step
// (Eq. 7-8). Two deterministic passes: every (row, chunk) item reduces its
// nodes in a fixed order into one partial, then one thread per row combines
// that row's partials in item order.
#include "common.cuh"
#include "kernels.h"
#include "norms.h"

namespace burgers {

constexpr int RED_NT = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int k = 16; k > 0; k >>= 1) v += __shfl_xor_sync(FULL_MASK, v, k);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int k = 16; k > 0; k >>= 1) v = fmax(v, __shfl_xor_sync(FULL_MASK, v, k));
  return v;
}

template <typename TU, typename TR>
__global__ void __launch_bounds__(RED_NT) k_l2_partial(const TU* __restrict__ u,
                                                       const TR* __restrict__ ref,
                                                       const RowDesc* __restrict__ rows,
                                                       const TileItem* __restrict__ items,
                                                       int chunk, double2* __restrict__ partial) {
  __shared__ double s_num[RED_NT / 32], s_den[RED_NT / 32];
  const TileItem ti = items[blockIdx.x];
  const RowDesc rd = rows[ti.row];
  const int64_t lo = int64_t(ti.tile) * chunk;
  const int64_t hi = min(lo + chunk, int64_t(rd.n));
  const TU* pu = u + rd.offset;
  const TR* pr = ref + rd.offset;
  double num = 0.0, den = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += RED_NT) {
    const double rv = double(pr[i]);
    const double e = double(pu[i]) - rv;
    num = fma(e, e, num);
    den = fma(rv, rv, den);
  }
  num = warp_sum(num);
  den = warp_sum(den);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { s_num[w] = num; s_den[w] = den; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < RED_NT / 32; ++k) { a += s_num[k]; b += s_den[k]; }
    partial[blockIdx.x] = make_double2(a, b);
  }
}

__global__ void k_l2_final(const double2* __restrict__ partial,
                           const int32_t* __restrict__ first_item, const RowDesc* __restrict__ rows,
                           int count, double* __restrict__ rel, double* __restrict__ rms) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count) return;
  double num = 0.0, den = 0.0;
  for (int k = first_item[b]; k < first_item[b + 1]; ++k) {
    num += partial[k].x;
    den += partial[k].y;
  }
  rel[b] = den > 0.0 ? sqrt(num / den) : (num == 0.0 ? 0.0 : INFINITY);
  rms[b] = sqrt(num / double(rows[b].n));
}

template <typename T>
__global__ void __launch_bounds__(RED_NT) k_absmax_partial(const T* __restrict__ u,
                                                           const RowDesc* __restrict__ rows,
                                                           const TileItem* __restrict__ items,
                                                           int chunk, double* __restrict__ partial) {
  __shared__ double s_m[RED_NT / 32];
  const TileItem ti = items[blockIdx.x];
  const RowDesc rd = rows[ti.row];
  const int64_t lo = int64_t(ti.tile) * chunk;
  const int64_t hi = min(lo + chunk, int64_t(rd.n));
  const T* pu = u + rd.offset;
  double m = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += RED_NT) m = fmax(m, fabs(double(pu[i])));
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int k = 0; k < RED_NT / 32; ++k) a = fmax(a, s_m[k]);
    partial[blockIdx.x] = a;
  }
}

// Eq. 7-8 with safety factor cfl; -1 where neither limit is finite.
__global__ void k_cfl_final(const double* __restrict__ partial,
                            const int32_t* __restrict__ first_item, const double2* __restrict__ dxnu,
                            int count, double cfl, double* __restrict__ dt) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count) return;
  double m = 0.0;
  for (int k = first_item[b]; k < first_item[b + 1]; ++k) m = fmax(m, partial[k]);
  const double dx = dxnu[b].x, nu = dxnu[b].y;
  const double dconv = m > 0.0 ? dx / m : INFINITY;
  const double ddiff = nu > 0.0 ? dx * dx / (2.0 * nu) : INFINITY;
  const double d = fmin(dconv, ddiff);
  dt[b] = isinf(d) ? -1.0 : cfl * d;
}

cudaError_t launch_rel_l2(int dtype_u, int dtype_ref, const void* u, const void* ref,
                          const RowDesc* rows, const TileItem* items, int nitems,
                          const int32_t* first_item, int count, int chunk, double2* partial,
                          double* rel, double* rms, cudaStream_t st) {
  if (nitems > 0) {
    if (dtype_u == 0 && dtype_ref == 0)
      k_l2_partial<float, float><<<nitems, RED_NT, 0, st>>>(
          (const float*)u, (const float*)ref, rows, items, chunk, partial);
    else if (dtype_u == 0 && dtype_ref == 1)
      k_l2_partial<float, double><<<nitems, RED_NT, 0, st>>>(
          (const float*)u, (const double*)ref, rows, items, chunk, partial);
    else if (dtype_u == 1 && dtype_ref == 0)
      k_l2_partial<double, float><<<nitems, RED_NT, 0, st>>>(
          (const double*)u, (const float*)ref, rows, items, chunk, partial);
    else
      k_l2_partial<double, double><<<nitems, RED_NT, 0, st>>>(
          (const double*)u, (const double*)ref, rows, items, chunk, partial);
  }
  k_l2_final<<<(count + 127) / 128, 128, 0, st>>>(partial, first_item, rows, count, rel, rms);
  return cudaGetLastError();
}

cudaError_t launch_cfl(int dtype, const void* u, const RowDesc* rows, const TileItem* items,
                       int nitems, const int32_t* first_item, const double2* dxnu, int count,
                       int chunk, double cfl, double* partial, double* dt, cudaStream_t st) {
  if (nitems > 0) {
    if (dtype == 0)
      k_absmax_partial<float><<<nitems, RED_NT, 0, st>>>((const float*)u, rows, items, chunk,
                                                         partial);
    else
      k_absmax_partial<double><<<nitems, RED_NT, 0, st>>>((const double*)u, rows, items, chunk,
                                                          partial);
  }
  k_cfl_final<<<(count + 127) / 128, 128, 0, st>>>(partial, first_item, dxnu, count, cfl, dt);
  return cudaGetLastError();
}

}  // namespace burgers
