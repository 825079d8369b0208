// adjoint_long.cu -- discrete adjoint of the explicit solve (Eq. 21, upwind
// side by sign, H(0) = 0; Sec. 2.7.1 / 2.7.3) for rows longer than one CTA
// holds.
//
// The forward trajectory advances one step per HBM pass with the single-step
// kernel (k_explicit_step1, FP32 with its one-byte compensation term) and
// stores the state (and compensation) every k steps in HBM; the reverse pass
// walks the segments backwards, recomputes a segment's k states into HBM
// with the same kernel from its checkpoint (so the recomputed states are
// bitwise those of the checkpoint pass), and applies the transposed step
// Jacobian to lambda one step per pass over the same tiles:
//   lambda_i <- lambda_i - c_i lambda_i + (s + r u_{i+1}^+) lambda_{i+1}
//               + (s - r u_{i-1}^-) lambda_{i-1},
//   c_i = 2s + r (H_i (u_i - u_{i-1}) + (1 - H_i)(u_{i+1} - u_i) + |u_i|),
// the neighbour terms only from rows that are not Dirichlet identity rows,
// and dJ/dnu accumulates (dt/dx^2) lambda_i (u_{i+1} - 2u_i + u_{i-1}) over
// those rows in FP64: per tile and step into a per-tile sum (each tile has
// one owner per launch, so the order is fixed), summed per row at the end.
// FP32 lambda carries a Kahan term across the steps. Rows are aligned at their
// first step: a row with fewer steps than the longest is copied through by
// both kernels until its own steps begin (reverse) or after they end (forward).
//
// BTCS (Sec. 2.4): the forward states come from the library's own BTCS plan
// one step per call (checkpoints every k steps, a segment's k + 1 states
// recomputed the same way), and each reverse step solves the transposed
// system A(u^n)^T nu = lam - A(u^n)^T lam through the multi-level solver
// (its level-0 rows transposed, transposed_btcs_solve), then updates lambda
// from mu = lam + nu and u^{n+1} per tile (k_adjoint_btcs_update).
#include <math.h>
#include <string.h>

#include <algorithm>

#include "adjoint.h"
#include "api_internal.h"
#include "common.cuh"
#include "kernels.h"

namespace burgers {

// One reverse step of every tile: lam (after step `step`) -> lam2 (before it),
// from the state u = u^step.
template <typename T, int NT, int C>
__global__ void __launch_bounds__(NT) k_adjoint_step1(const T* __restrict__ u,
                                                      const T* __restrict__ lam, T* __restrict__ lam2,
                                                      const T* __restrict__ lc, T* __restrict__ lc2,
                                                      const RowDesc* __restrict__ rows,
                                                      const TileItem* __restrict__ items, int nitems,
                                                      int64_t step, double* __restrict__ gtile) {
  constexpr bool KL = Kahan<T>::on;
  __shared__ double wsum[NT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const TileItem ti = items[it];
    const RowDesc& rd = rows[ti.row];
    const int64_t n = rd.n;
    const int64_t g0 = int64_t(ti.tile) * (NT * C) + int64_t(threadIdx.x) * C;
    const int cnt = g0 >= n ? 0 : (n - g0 < C ? int(n - g0) : C);
    double part = 0.0;
    if (cnt > 0) {
      const T* urow = u + rd.offset;
      const T* lrow = lam + rd.offset;
      T* drow = lam2 + rd.offset;
      const T* crow = KL ? lc + rd.offset : nullptr;
      T* c2row = KL ? lc2 + rd.offset : nullptr;
      const bool per = rd.bc == BC_PERIODIC;
      // the thread's nodes and their two neighbours: v[0] = u_{g0-1},
      // v[1 + j] = u_{g0+j}, v[cnt + 1] = u_{g0+cnt} (likewise w for lambda)
      T v[C + 2], w[C + 2], kc[C];
#pragma unroll
      for (int j = 0; j < C + 2; ++j) { v[j] = T(0); w[j] = T(0); }
#pragma unroll
      for (int j = 0; j < C; ++j) {
        if (j < cnt) {
          v[1 + j] = urow[g0 + j];
          w[1 + j] = lrow[g0 + j];
        }
        kc[j] = (KL && j < cnt) ? crow[g0 + j] : T(0);
      }
      const int64_t il = g0 > 0 ? g0 - 1 : (per ? n - 1 : -1);
      const int64_t ir = g0 + cnt < n ? g0 + cnt : (per ? 0 : -1);
      if (il >= 0) { v[0] = urow[il]; w[0] = lrow[il]; }
      if (ir >= 0) {
#pragma unroll
        for (int j = 1; j <= C; ++j)
          if (j == cnt) { v[j + 1] = urow[ir]; w[j + 1] = lrow[ir]; }
      }
      if (step < rd.nsteps) {
        const RowCoefs<T> cf = row_coefs(rd, T(0));
        const T r = cf.r, s = cf.s;
#pragma unroll
        for (int j = 0; j < C; ++j) {
          if (j < cnt) {
            const int64_t gi = g0 + j;
            const T uu = v[1 + j], ul = v[j], ur = v[2 + j];
            const T ll = w[j], lr = w[2 + j], wj = w[1 + j];
            const bool upI = per || (gi > 0 && gi < n - 1);
            const bool upR = per || (gi + 1 < n - 1);
            const bool upL = per || (gi - 1 > 0);
            const T dl = uu - ul, dr = ur - uu;
            const T cI = upI ? tfma(r, (uu > T(0) ? dl : dr) + tabs(uu), T(2) * s) : T(0);
            T inc = -cI * wj;
            if (upR) inc = tfma(tfma(r, tmax(ur, T(0)), s), lr, inc);
            if (upL) inc = tfma(tfma(-r, tmin(ul, T(0)), s), ll, inc);
            if (upI) part = fma(double(wj), double(dr - dl), part);
            T out;
            if constexpr (KL) {
              const T y = inc - kc[j];
              out = wj + y;
              kc[j] = (out - wj) - y;
            } else {
              out = wj + inc;
            }
            drow[gi] = out;
            if constexpr (KL) c2row[gi] = kc[j];
          }
        }
      } else {  // the row's steps have not begun (reverse order): copied through
#pragma unroll
        for (int j = 0; j < C; ++j)
          if (j < cnt) {
            drow[g0 + j] = w[1 + j];
            if constexpr (KL) c2row[g0 + j] = kc[j];
          }
      }
    }
    // the tile's dJ/dnu part (FP64, fixed order)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(FULL_MASK, part, o);
    if (lane == 0) wsum[warp] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
#pragma unroll
      for (int q = 0; q < NT / 32; ++q) t += wsum[q];
      gtile[it] += t;
    }
    __syncthreads();
  }
}

// The BTCS step's reverse update of every tile, given nu from the transposed
// solve A(u^n)^T nu = lam - A(u^n)^T lam (mu = lam + nu) and x = u^{n+1}:
//   lam_i <- mu_i - mu_i r (-H_i x_{i-1} + (2H_i - 1) x_i + (1 - H_i) x_{i+1}),
// H_i = [u^n_i > 0], zero for Dirichlet identity rows, and dJ/dnu += (dt/dx^2)
// mu_i (x_{i+1} - 2x_i + x_{i-1}) over the other rows (FP64 per tile).
template <typename T, int NT, int C>
__global__ void __launch_bounds__(NT) k_adjoint_btcs_update(
    const T* __restrict__ un, const T* __restrict__ x, const T* __restrict__ lam,
    T* __restrict__ lam2, const T* __restrict__ lc, T* __restrict__ lc2, const T* __restrict__ nu,
    const RowDesc* __restrict__ rows, const TileItem* __restrict__ items, int nitems,
    int64_t step, double* __restrict__ gtile) {
  constexpr bool KL = Kahan<T>::on;
  __shared__ double wsum[NT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const TileItem ti = items[it];
    const RowDesc& rd = rows[ti.row];
    const int64_t n = rd.n;
    const int64_t g0 = int64_t(ti.tile) * (NT * C) + int64_t(threadIdx.x) * C;
    const int cnt = g0 >= n ? 0 : (n - g0 < C ? int(n - g0) : C);
    double part = 0.0;
    if (cnt > 0) {
      const T* arow = un + rd.offset;
      const T* xrow = x + rd.offset;
      const T* lrow = lam + rd.offset;
      const T* nrow = nu + rd.offset;
      T* drow = lam2 + rd.offset;
      const bool per = rd.bc == BC_PERIODIC;
      const bool active = step < rd.nsteps;
      const RowCoefs<T> cf = row_coefs(rd, T(0));
      const T r = cf.r;
#pragma unroll
      for (int j = 0; j < C; ++j) {
        if (j < cnt) {
          const int64_t gi = g0 + j;
          const T w = lrow[gi];
          T kc = KL ? lc[rd.offset + gi] : T(0);
          T out = w;
          if (active) {
            const bool ident = !per && (gi == 0 || gi == n - 1);
            const T nv = nrow[gi];
            const T mu = w + nv;
            T inc = nv;
            if (!ident) {
              const int64_t il = gi > 0 ? gi - 1 : n - 1, ir = gi + 1 < n ? gi + 1 : 0;
              const T xl = xrow[il], xc = xrow[gi], xr = xrow[ir];
              const bool H = arow[gi] > T(0);
              const T drw = r * (H ? (xc - xl) : (xr - xc));
              inc = tfma(-mu, drw, nv);
              part = fma(double(mu), double((xr - xc) - (xc - xl)), part);
            }
            if constexpr (KL) {
              const T y = inc - kc;
              out = w + y;
              kc = (out - w) - y;
            } else {
              out = w + inc;
            }
          }
          drow[gi] = out;
          if constexpr (KL) lc2[rd.offset + gi] = kc;
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(FULL_MASK, part, o);
    if (lane == 0) wsum[warp] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
#pragma unroll
      for (int q = 0; q < NT / 32; ++q) t += wsum[q];
      gtile[it] += t;
    }
    __syncthreads();
  }
}

// dJ/dnu of each long row: ds/dnu times the sum of its tiles' parts.
__global__ void k_adj_long_gnu(const double* __restrict__ gtile, const AdjLongRow* __restrict__ lr,
                               int nrows, double* __restrict__ gnu) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nrows) return;
  double s = 0.0;
  for (int t = lr[q].tile_begin; t < lr[q].tile_end; ++t) s += gtile[t];
  gnu[lr[q].out_index] = lr[q].ds_dnu * s;
}

void register_adjoint_long(std::vector<KernelEntry>& reg) {
  reg.push_back({K_ADJ_EXPLICIT, 0, 512, 8, 2,
                 reinterpret_cast<const void*>(&k_adjoint_step1<float, 512, 8>), 0});
  reg.push_back({K_ADJ_EXPLICIT, 1, 256, 4, 2,
                 reinterpret_cast<const void*>(&k_adjoint_step1<double, 256, 4>), 0});
  reg.push_back({K_ADJ_BTCS, 0, 512, 8, 2,
                 reinterpret_cast<const void*>(&k_adjoint_btcs_update<float, 512, 8>), 0});
  reg.push_back({K_ADJ_BTCS, 1, 256, 4, 2,
                 reinterpret_cast<const void*>(&k_adjoint_btcs_update<double, 256, 4>), 0});
}

burgers_status adjoint_long_run(burgers_ctx* ctx, int scheme, const burgers_batch* batch,
                                const std::vector<int64_t>& longs, const void* u0, const void* gT,
                                void* gu0, double* gnu, int64_t stride, cudaStream_t st) {
  const int dtype = batch->dtype;
  const size_t esz = dtype == 0 ? 4 : 8;
  const bool btcs = scheme == BURGERS_BTCS;
  const int nt = dtype == 0 ? 512 : 256, c = dtype == 0 ? 8 : 4;
  const KernelEntry* kf = find_kernel(K_EXPLICIT_STEP1, dtype, nt, c, 0);
  const KernelEntry* ka = find_kernel(btcs ? K_ADJ_BTCS : K_ADJ_EXPLICIT, dtype, nt, c, 2);
  if (!kf || !ka) return set_error(BURGERS_EINVAL, "long-row adjoint kernels missing");
  // BTCS: the forward steps and the transposed solves go through the
  // library's own plans on a batch of the long rows, one step per call
  std::vector<burgers_instance> one;
  for (int64_t b : longs) {
    burgers_instance in = batch->inst[b];
    in.nsteps = 1;
    one.push_back(in);
  }
  burgers_batch b1;
  b1.dtype = dtype;
  b1.reserved = 0;
  b1.count = int64_t(one.size());
  b1.inst = one.data();
  const int64_t tile = int64_t(nt) * c;
  std::vector<RowDesc> rows;
  std::vector<TileItem> items;
  std::vector<AdjLongRow> lrows;
  int64_t nmax = 0, span = 0;
  for (int64_t b : longs) {
    const burgers_instance& in = batch->inst[b];
    RowDesc d;
    d.offset = in.offset;
    d.nsteps = in.nsteps;
    d.r = in.dt / in.dx;
    d.s = in.nu * in.dt / (in.dx * in.dx);
    d.ds_dnu = in.dt / (in.dx * in.dx);
    d.n = in.n;
    d.bc = in.bc;
    set_fp32_coefs(d);
    AdjLongRow a;
    a.tile_begin = int32_t(items.size());
    const int64_t tiles = (in.n + tile - 1) / tile;
    for (int64_t t = 0; t < tiles; ++t)
      items.push_back(TileItem{int32_t(rows.size()), int32_t(t)});
    a.tile_end = int32_t(items.size());
    a.out_index = int32_t(b);
    a.pad = 0;
    a.ds_dnu = d.ds_dnu;
    rows.push_back(d);
    lrows.push_back(a);
    nmax = std::max<int64_t>(nmax, in.nsteps);
    span = std::max<int64_t>(span, in.offset + in.n);
  }
  const int64_t k = stride > 0 ? stride : std::max<int64_t>(1, int64_t(ceil(sqrt(double(std::max<int64_t>(nmax, 1))))));
  const int64_t nck = nmax > 0 ? (nmax + k - 1) / k : 0;
  // segment states: u^{s0} .. u^{s1-1} (explicit), .. u^{s1} (BTCS: its
  // reverse update also reads u^{n+1})
  const int64_t seg = std::min<int64_t>(k, std::max<int64_t>(nmax, 1)) + (btcs ? 1 : 0);
  const int64_t span_rows = span;  // elements of the caller's buffers the rows cover
  span = (span + 63) & ~int64_t(63);
  const int nitems = int(items.size());
  // workspace: forward state ping-pong, checkpoints, segment states, lambda
  // ping-pong (+ FP32 compensation: one byte per node for the state, the
  // element type for lambda), per-tile dJ/dnu sums
  const bool fp32 = dtype == 0;
  const size_t sb = size_t(span) * esz, lb = fp32 ? size_t(span) : 0;
  const size_t o_x0 = 0, o_x1 = o_x0 + sb, o_l0 = o_x1 + sb, o_l1 = o_l0 + lb;
  const size_t o_ck = (o_l1 + lb + 255) & ~size_t(255);
  const size_t ckb = ((sb + lb + 255) & ~size_t(255));
  const size_t o_seg = o_ck + size_t(nck) * ckb;
  const size_t o_la = o_seg + size_t(seg) * sb, o_lb = o_la + sb;
  const size_t o_ca = o_lb + sb, o_cb = o_ca + (fp32 ? sb : 0);
  const size_t o_nu = (o_cb + (fp32 ? sb : 0) + 255) & ~size_t(255);
  const size_t o_gt = (o_nu + (btcs ? sb : 0) + 255) & ~size_t(255);
  const size_t total = o_gt + size_t(std::max(nitems, 1)) * sizeof(double);
  cudaError_t e = ctx->adjlong.ensure(total);
  if (e != cudaSuccess) return set_error(BURGERS_ENOMEM, "long-row adjoint workspace: out of device memory");
  // descriptors: rows | items | per-row sums, staged through page-locked memory
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t d_rows = 0, d_items = al(rows.size() * sizeof(RowDesc));
  const size_t d_lr = al(d_items + items.size() * sizeof(TileItem));
  const size_t dtotal = al(d_lr + lrows.size() * sizeof(AdjLongRow));
  e = ctx->adjldesc.ensure(dtotal);
  if (e == cudaSuccess) e = ctx->adjlhost.ensure_host(dtotal);
  if (e != cudaSuccess) return set_error(BURGERS_ENOMEM, "long-row adjoint descriptors");
  if (ctx->adjl_event) {
    e = cudaEventSynchronize(ctx->adjl_event);
    if (e != cudaSuccess) return cuda_error(e, "adjoint staging");
  } else {
    e = cudaEventCreateWithFlags(&ctx->adjl_event, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_error(e, "cudaEventCreate");
  }
  char* h = static_cast<char*>(ctx->adjlhost.hptr);
  memcpy(h + d_rows, rows.data(), rows.size() * sizeof(RowDesc));
  memcpy(h + d_items, items.data(), items.size() * sizeof(TileItem));
  memcpy(h + d_lr, lrows.data(), lrows.size() * sizeof(AdjLongRow));
  char* dd = static_cast<char*>(ctx->adjldesc.ptr);
  e = cudaMemcpyAsync(dd, h, dtotal, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->adjl_event, st);
  if (e != cudaSuccess) return cuda_error(e, "adjoint upload");
  const RowDesc* drows = reinterpret_cast<const RowDesc*>(dd + d_rows);
  const TileItem* ditems = reinterpret_cast<const TileItem*>(dd + d_items);
  const AdjLongRow* dlr = reinterpret_cast<const AdjLongRow*>(dd + d_lr);
  char* w = static_cast<char*>(ctx->adjlong.ptr);
  void* X[2] = {w + o_x0, w + o_x1};
  void* LO[2] = {fp32 ? w + o_l0 : nullptr, fp32 ? w + o_l1 : nullptr};
  void* LAM[2] = {w + o_la, w + o_lb};
  void* LC[2] = {fp32 ? w + o_ca : nullptr, fp32 ? w + o_cb : nullptr};
  double* gt = reinterpret_cast<double*>(w + o_gt);
  auto grid_of = [&](const KernelEntry* kk) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kk->fn, kk->nt, kk->dyn_smem) != cudaSuccess ||
        b < 1)
      b = 1;
    return std::max(1, std::min(nitems, ctx->sm_count * b));
  };
  const int gf = grid_of(kf), ga = grid_of(ka);
  auto fwd = [&](const void* src, void* dst, const void* ls, void* ldst, int64_t step) {
    int ni = nitems, K = 1;
    int64_t sb_ = step;
    void* args[] = {(void*)&src, &dst, (void*)&ls, &ldst, (void*)&drows, (void*)&ditems, &ni, &K, &sb_};
    ctx->launches += 1;
    return cudaLaunchKernel(kf->fn, dim3(gf), dim3(kf->nt), args, kf->dyn_smem, st);
  };
  // ---- forward pass with checkpoints (rows laid out as in the batch)
  e = cudaMemcpyAsync(X[0], u0, size_t(span_rows) * esz, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && fp32) e = cudaMemsetAsync(LO[0], 0, lb, st);
  // checkpoint c holds u^{c k}; the steps after the last checkpoint are
  // recomputed in the reverse pass
  int cur = 0;
  const int64_t s_last = nck > 0 ? (nck - 1) * k : 0;
  burgers_status bs = BURGERS_OK;
  for (int64_t s = 0; s <= s_last && nck > 0 && e == cudaSuccess && bs == BURGERS_OK; ++s) {
    if (s % k == 0) {
      char* ck = w + o_ck + size_t(s / k) * ckb;
      e = cudaMemcpyAsync(ck, X[cur], sb, cudaMemcpyDeviceToDevice, st);
      if (e == cudaSuccess && fp32 && !btcs)
        e = cudaMemcpyAsync(ck + sb, LO[cur], lb, cudaMemcpyDeviceToDevice, st);
    }
    if (e == cudaSuccess && s < s_last) {
      if (btcs) {  // in place, one step (every long row; the reverse pass ignores
                   // the steps past a row's own count)
        bs = advance(ctx, BURGERS_BTCS, &b1, X[cur], st);
      } else {
        e = fwd(X[cur], X[cur ^ 1], LO[cur], LO[cur ^ 1], s);
        cur ^= 1;
      }
    }
  }
  if (bs != BURGERS_OK) return bs;
  // ---- reverse pass
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(LAM[0], gT, size_t(span_rows) * esz, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && fp32) e = cudaMemsetAsync(LC[0], 0, sb, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(gt, 0, size_t(std::max(nitems, 1)) * sizeof(double), st);
  int lcur = 0;
  for (int64_t cidx = nck - 1; cidx >= 0 && e == cudaSuccess; --cidx) {
    const int64_t s0 = cidx * k, s1 = std::min<int64_t>(s0 + k, nmax);
    const char* ck = w + o_ck + size_t(cidx) * ckb;
    char* S0 = w + o_seg;
    e = cudaMemcpyAsync(S0, ck, sb, cudaMemcpyDeviceToDevice, st);
    if (btcs) {  // u^{s0} .. u^{s1} through the BTCS plan, one step a call
      if (e == cudaSuccess) e = cudaMemcpyAsync(X[0], ck, sb, cudaMemcpyDeviceToDevice, st);
      for (int64_t j = 1; j <= s1 - s0 && e == cudaSuccess; ++j) {
        bs = advance(ctx, BURGERS_BTCS, &b1, X[0], st);
        if (bs != BURGERS_OK) return bs;
        e = cudaMemcpyAsync(S0 + size_t(j) * sb, X[0], sb, cudaMemcpyDeviceToDevice, st);
      }
    } else {
      if (e == cudaSuccess && fp32)
        e = cudaMemcpyAsync(LO[0], ck + sb, lb, cudaMemcpyDeviceToDevice, st);
      int lo = 0;
      for (int64_t j = 1; j < s1 - s0 && e == cudaSuccess; ++j) {
        e = fwd(S0 + size_t(j - 1) * sb, S0 + size_t(j) * sb, LO[lo], LO[lo ^ 1], s0 + j - 1);
        lo ^= 1;
      }
    }
    for (int64_t s = s1 - 1; s >= s0 && e == cudaSuccess; --s) {
      if (btcs) {
        const void* un = S0 + size_t(s - s0) * sb;
        const void* xn = S0 + size_t(s - s0 + 1) * sb;
        void* nuv = w + o_nu;
        bs = transposed_btcs_solve(ctx, &b1, un, LAM[lcur], nuv, st);
        if (bs != BURGERS_OK) return bs;
        const void* ls = LAM[lcur];
        void* ld = LAM[lcur ^ 1];
        const void* cs = LC[lcur];
        void* cd = LC[lcur ^ 1];
        const void* nuc = nuv;
        int ni = nitems;
        int64_t sv = s;
        void* args[] = {(void*)&un, (void*)&xn, (void*)&ls, &ld, (void*)&cs, &cd, (void*)&nuc,
                        (void*)&drows, (void*)&ditems, &ni, &sv, &gt};
        ctx->launches += 1;
        e = cudaLaunchKernel(ka->fn, dim3(ga), dim3(ka->nt), args, 0, st);
        lcur ^= 1;
        continue;
      }
      const void* us = S0 + size_t(s - s0) * sb;
      const void* ls = LAM[lcur];
      void* ld = LAM[lcur ^ 1];
      const void* cs = LC[lcur];
      void* cd = LC[lcur ^ 1];
      int ni = nitems;
      int64_t sv = s;
      void* args[] = {(void*)&us, (void*)&ls, &ld, (void*)&cs, &cd, (void*)&drows, (void*)&ditems,
                      &ni, &sv, &gt};
      ctx->launches += 1;
      e = cudaLaunchKernel(ka->fn, dim3(ga), dim3(ka->nt), args, 0, st);
      lcur ^= 1;
    }
  }
  if (e != cudaSuccess) return cuda_error(e, "long-row adjoint");
  // ---- results: dJ/du0 of each long row, dJ/dnu
  for (size_t q = 0; q < rows.size() && e == cudaSuccess; ++q)
    e = cudaMemcpyAsync(static_cast<char*>(gu0) + size_t(rows[q].offset) * esz,
                        static_cast<const char*>(LAM[lcur]) + size_t(rows[q].offset) * esz,
                        size_t(rows[q].n) * esz, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_error(e, "long-row adjoint result");
  const int nr = int(lrows.size());
  k_adj_long_gnu<<<(nr + 127) / 128, 128, 0, st>>>(gt, dlr, nr, gnu);
  ctx->launches += 1;
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "long-row adjoint dJ/dnu");
  return BURGERS_OK;
}

}  // namespace burgers
