// api.cu -- the C ABI of libburgers (include/burgers.h): context, argument
// checks, launch planning, plan and CUDA-graph caches, dispatch.
//
// A call turns its batch into a Plan: rows short enough to stay resident are
// grouped by kernel shape (smallest register capacity >= n), each group sorted
// by cost (n * nsteps, longest first) so the persistent CTAs of one launch
// drain it with little tail; longer rows become tiled work items of the
// streaming explicit kernel or of the multi-level BTCS solver. The packed
// descriptors live in device memory owned by the plan, so a repeated batch
// costs no host-to-device copy, and a plan with several launches is captured
// once into a CUDA graph and replayed.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <list>
#include <memory>
#include <string>
#include <vector>

#include "../../include/burgers.h"
#include "api_internal.h"
#include "kernels.h"
#include "norms.h"

using namespace burgers;

namespace burgers {

thread_local std::string g_last_error;

burgers_status set_error(burgers_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

burgers_status cuda_error(cudaError_t e, const char* where) {
  return set_error(BURGERS_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------
// device buffers
// ---------------------------------------------------------------------------
DevBuf::~DevBuf() {
  if (ptr) cudaFree(ptr);
}

cudaError_t DevBuf::ensure(size_t need) {
  if (need <= bytes) return cudaSuccess;
  if (ptr) {
    cudaError_t e = cudaDeviceSynchronize();  // the old buffer may still be in use
    if (e != cudaSuccess) return e;
    cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
  }
  size_t want = std::max(need, size_t(1) << 16);
  cudaError_t e = cudaMalloc(&ptr, want);
  if (e != cudaSuccess) {
    ptr = nullptr;
    return e;
  }
  bytes = want;
  ++generation;
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// shapes
// ---------------------------------------------------------------------------
struct Shape {
  int nt, c;
};

// Default resident shapes per (kind, dtype), ascending capacity; the first
// entry of a capacity is the default, later entries are autotuning
// alternatives of the same capacity. The defaults are the shapes the
// autotuner picks on a B300 for full batches of that capacity class (FP32
// BTCS and the implicit variants: 128 x 16, 128 x 32 and 256 x 32 for 2048,
// 4096 and 8192 nodes, 1.5-1.8x the 256 x 8, 256 x 16 and 512 x 16 shapes).
static const std::vector<Shape>& resident_shapes(int kind, int dtype) {
  static const std::vector<Shape> ex32 = {{32, 1},   {32, 2},    {32, 4},   {32, 8},  {64, 8},
                                          {128, 8},  {64, 16},   {128, 16}, {256, 8}, {256, 16},
                                          {128, 32}, {512, 16},  {256, 32}, {512, 8}, {1024, 16}};
  static const std::vector<Shape> ex64 = {{32, 1},  {32, 2},   {32, 4},  {32, 8},   {64, 8},
                                          {128, 8}, {256, 8},  {128, 16}, {512, 8}, {256, 16},
                                          {1024, 8}, {512, 16}};
  static const std::vector<Shape> bt32 = {{32, 1},   {32, 2},   {32, 4},   {32, 8},    {64, 8},
                                          {128, 8},  {128, 16}, {256, 8},  {64, 32},   {128, 32},
                                          {256, 16}, {512, 8},  {256, 32}, {512, 16},  {1024, 8}};
  static const std::vector<Shape> bt64 = {{32, 1},  {32, 2},  {32, 4},   {32, 8},   {64, 8},
                                          {128, 8}, {256, 8}, {128, 16}, {512, 8}, {256, 16}};
  static const std::vector<Shape> rk32 = {{32, 1},   {32, 2},  {32, 4},   {32, 8},  {64, 8},
                                          {128, 8},  {64, 16}, {128, 16}, {256, 8}, {512, 8},
                                          {256, 16}, {512, 16}};
  static const std::vector<Shape> rk64 = {{32, 1},  {32, 2},   {32, 4},   {32, 8},  {64, 8},
                                          {128, 4}, {128, 8},  {256, 4},  {256, 8}, {512, 4},
                                          {512, 8}, {1024, 4}};
  // Crank-Nicolson, Picard and Newton share the BTCS kernel shape
  static const std::vector<Shape> im32 = {{32, 1},   {32, 2},   {32, 4},   {32, 8},
                                          {64, 8},   {128, 8},  {128, 16}, {256, 8},
                                          {128, 32}, {256, 16}, {256, 32}};
  static const std::vector<Shape> im64 = {{32, 1},  {32, 2},   {32, 4},   {32, 8},  {64, 8},
                                          {128, 8}, {256, 8},  {128, 16}, {512, 8}};
  // Crank-Nicolson and Picard also have the packed kernel at 64 x 32 (Newton
  // has the scalar kernel only)
  static const std::vector<Shape> cp32 = {{32, 1},   {32, 2},   {32, 4},   {32, 8},
                                          {64, 8},   {128, 8},  {128, 16}, {256, 8},
                                          {64, 32},  {128, 32}, {256, 16}, {256, 32}};
  if (kind == K_EXPLICIT_RESIDENT) return dtype == 0 ? ex32 : ex64;
  if (kind == K_RK4_RESIDENT) return dtype == 0 ? rk32 : rk64;
  if (kind == K_CN_RESIDENT || kind == K_PICARD_RESIDENT || kind == K_NEWTON_RESIDENT)
    return dtype == 0 ? cp32 : im64;
  return dtype == 0 ? bt32 : bt64;
}

// A capacity class needs at least this many rows in a call to take the
// per-thread Thomas kernel by default (pick_thomas).
constexpr int64_t THOMAS_DEFAULT_MIN_ROWS = 8192;

static int64_t max_resident(int kind, int dtype) {
  int64_t m = 0;
  for (const Shape& s : resident_shapes(kind, dtype)) m = std::max<int64_t>(m, int64_t(s.nt) * s.c);
  return m;
}

}  // namespace burgers

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
burgers_ctx::burgers_ctx() = default;
burgers_ctx::~burgers_ctx() {
  for (auto& kv : redcache)
    if (kv.second.dev) cudaFree(kv.second.dev);
}

namespace burgers {

static int64_t resident_limit(const burgers_ctx* ctx, int kind, int dtype) {
  int64_t m = max_resident(kind, dtype);
  if (ctx->resident_max > 0) m = std::min<int64_t>(m, ctx->resident_max);
  if (ctx->resident_override) m = 0;
  return m;
}

int64_t resident_capacity(const burgers_ctx* ctx, int kind, int dtype) {
  return resident_limit(ctx, kind, dtype);
}

int64_t resident_class(int kind, int dtype, int64_t n) {
  int64_t cap = -1;
  for (const Shape& s : resident_shapes(kind, dtype)) {
    int64_t c = int64_t(s.nt) * s.c;
    if (c >= n && s.c < n && (cap < 0 || c < cap)) cap = c;
  }
  return cap;
}

std::vector<std::pair<int, int>> resident_shape_list(int kind, int dtype) {
  std::vector<std::pair<int, int>> out;
  for (const Shape& s : resident_shapes(kind, dtype)) out.emplace_back(s.nt, s.c);
  return out;
}

// Shape for a resident row of n nodes: the tuned choice for its capacity class
// if there is one, else the default (first smallest capacity >= n).
static Shape pick_resident(const burgers_ctx* ctx, int kind, int dtype, int64_t n) {
  const auto& list = resident_shapes(kind, dtype);
  int64_t cap = -1;
  Shape best{0, 0};
  for (const Shape& s : list) {
    int64_t c = int64_t(s.nt) * s.c;
    if (c >= n && s.c < n && (cap < 0 || c < cap)) {
      cap = c;
      best = s;
    }
  }
  if (cap > 0) {
    auto it = ctx->tuned.find(tune_key(kind, dtype, cap, cap == n));
    if (it != ctx->tuned.end()) return Shape{it->second.nt, it->second.c};
  }
  // ragged FP32 explicit rows of up to 4096 nodes: 128 x 32 leaves fewer
  // warps on the general path than 256 x 16 (about 10% faster; exact rows
  // keep 256 x 16)
  if (kind == K_EXPLICIT_RESIDENT && dtype == 0 && cap == 4096 && n < cap) return Shape{128, 32};
  // ragged FP32 BTCS rows of up to 2048 nodes: the packed kernel at 64 x 32
  // (longer chains, a 64-row reduced system) measured 6.5e11 against 5.4e11
  // cell-updates/s at 128 x 16 on 2000-node rows (100 steps at 10x the CFL
  // step); Crank-Nicolson, Picard and Newton take the same shape (one Picard
  // iteration is then bitwise the BTCS step)
  if ((kind == K_BTCS_RESIDENT || kind == K_CN_RESIDENT || kind == K_PICARD_RESIDENT ||
       kind == K_NEWTON_RESIDENT) &&
      dtype == 0 && cap == 2048 && n < cap)
    return Shape{64, 32};
  return best;
}

// BTCS rows of a capacity class whose tuning-table entry has k >= 1 take the
// per-thread Thomas kernel (k - 1: its layout mode, btcs_thomas.cu); an
// entry with k = 0 keeps the partitioned kernel. Without an entry, a class
// takes it when its rows are short and many (class_rows rows in the call):
// one thread per row needs thousands of rows to fill the GPU, and its
// elimination chain grows with the row. Measured on a B300 (100 steps at
// 10x the CFL step, cell-updates/s): FP32 16384 x 32 7.3e10 against 3.6e10
// partitioned, 65536 x 64 1.2e11 against 7.5e10, but 4096 x 64 4.1e10
// against 6.9e10 and 16384 x 128 1.1e11 against 1.5e11; FP64 16384 x 32
// 9.6e9 against 3.0e9, 65536 x 64 1.2e10 against 5.2e9, 16384 x 128 1.2e10
// against 8.2e9, 4096 x 64 3.5e9 against 5.1e9.
const KernelEntry* pick_thomas(const burgers_ctx* ctx, int dtype, int64_t n, int64_t class_rows) {
  if (ctx->plain) return nullptr;
  const int64_t cap = resident_class(K_BTCS_RESIDENT, dtype, n);
  if (cap <= 0) return nullptr;
  auto it = ctx->tuned.find(tune_key(K_BTCS_RESIDENT, dtype, cap, cap == n));
  if (it != ctx->tuned.end()) {
    if (it->second.k <= 0) return nullptr;
    const KernelEntry* k = find_kernel(K_BTCS_THOMAS, dtype, it->second.nt, it->second.c,
                                       it->second.k - 1);
    return k && k->c >= n ? k : nullptr;
  }
  if (class_rows < THOMAS_DEFAULT_MIN_ROWS) return nullptr;
  struct Def { int dtype, cap, nt, mode; };
  static const Def defs[] = {{0, 32, 256, 2}, {0, 64, 256, 0},
                             {1, 32, 128, 0}, {1, 64, 64, 1}, {1, 128, 64, 1}};
  for (const Def& d : defs)
    if (d.dtype == dtype && d.cap == cap) return find_kernel(K_BTCS_THOMAS, dtype, d.nt, d.cap, d.mode);
  return nullptr;
}

// FNV-1a over 64-bit words (then the tail bytes): the plan key hashes every
// instance record of a batch on each call, 48 bytes per row.
static uint64_t fnv1a(const void* data, size_t len, uint64_t h = 1469598103934665603ull) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  size_t i = 0;
  for (; i + 8 <= len; i += 8) {
    uint64_t w;
    memcpy(&w, p + i, 8);
    h ^= w;
    h *= 1099511628211ull;
  }
  for (; i < len; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

burgers_status validate_batch(const burgers_batch* batch, bool allow_empty) {
  if (!batch) return set_error(BURGERS_EINVAL, "batch is NULL");
  if (batch->dtype != BURGERS_F32 && batch->dtype != BURGERS_F64)
    return set_error(BURGERS_EINVAL, "bad dtype");
  if (batch->count < 0) return set_error(BURGERS_EINVAL, "negative count");
  if (batch->count > 0 && !batch->inst) return set_error(BURGERS_EINVAL, "inst is NULL");
  if (batch->count == 0 && !allow_empty) return BURGERS_OK;
  if (batch->count > (int64_t(1) << 30)) return set_error(BURGERS_EINVAL, "count too large");
  std::vector<std::pair<int64_t, int64_t>> spans;
  spans.reserve(size_t(batch->count));
  for (int64_t b = 0; b < batch->count; ++b) {
    const burgers_instance& in = batch->inst[b];
    char msg[160];
    if (in.n < 3) {
      snprintf(msg, sizeof msg, "row %lld: n = %d < 3", (long long)b, in.n);
      return set_error(BURGERS_EINVAL, msg);
    }
    if (in.bc != BURGERS_PERIODIC && in.bc != BURGERS_DIRICHLET) {
      snprintf(msg, sizeof msg, "row %lld: bad bc %d", (long long)b, in.bc);
      return set_error(BURGERS_EINVAL, msg);
    }
    if (!(in.dx > 0.0) || !(in.nu >= 0.0) || !(in.dt > 0.0) || in.nsteps < 0 ||
        in.offset < 0) {
      snprintf(msg, sizeof msg, "row %lld: need dx > 0, nu >= 0, dt > 0, nsteps >= 0, offset >= 0",
               (long long)b);
      return set_error(BURGERS_EINVAL, msg);
    }
    spans.emplace_back(in.offset, in.offset + in.n);
  }
  std::sort(spans.begin(), spans.end());
  for (size_t i = 1; i < spans.size(); ++i)
    if (spans[i].first < spans[i - 1].second)
      return set_error(BURGERS_EINVAL, "rows overlap");
  return BURGERS_OK;
}

static RowDesc make_row(const burgers_instance& in, int iters = 1) {
  RowDesc d;
  d.iters = iters;
  d.offset = in.offset;
  d.nsteps = in.nsteps;
  d.r = in.dt / in.dx;
  d.s = in.nu * in.dt / (in.dx * in.dx);
  d.ds_dnu = in.dt / (in.dx * in.dx);
  d.n = in.n;
  d.bc = in.bc;
  set_fp32_coefs(d);
  return d;
}

static int blocks_per_sm(const KernelEntry* k) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k->fn, k->nt, k->dyn_smem) != cudaSuccess ||
      b < 1)
    b = 1;
  return b;
}

// Streaming shape for a long explicit (kind K_EXPLICIT_STREAM) or RK4
// (K_RK4_STREAM) row: the largest registered window that fits the row, with K
// steps per pass such that the stale edges (K nodes per side, 4K for RK4)
// take at most a quarter of the window. Untuned FP32 defaults: forward Euler
// in windows of 8192 nodes with K = 64, or K = 128 where the shortest row
// spans 32 windows or more (its last window's padding and the wider halo are
// then small), RK4 in windows of 4096 with K = 32 (a window's load,
// compensation decode and encode and store cost about as much as 11 of its
// steps: on a 2^24-node row 256 x 16 with K = 32 ran 2.87e12 cell-updates/s,
// 256 x 32 with K = 64 / 128 3.42e12 / 3.73e12; rows of 40000 nodes 2.33e12
// at the old default, 2.86e12 at K = 64; RK4 K = 8 / 32 6.2e11 / 8.3e11).
static bool pick_stream(const burgers_ctx* ctx, int kind, int dtype, int64_t n_min, Shape* sh,
                        int* K) {
  static const Shape s32[] = {{256, 32}, {256, 16}, {128, 16}, {32, 4}};
  static const Shape s32rk[] = {{256, 16}, {128, 16}, {32, 4}};
  static const Shape s64[] = {{256, 8}, {128, 8}, {32, 4}};
  const int per_step = kind == K_RK4_STREAM ? 4 : 1;
  const Shape* list = dtype != 0 ? s64 : (per_step == 4 ? s32rk : s32);
  const int nlist = dtype == 0 && per_step == 1 ? 4 : 3;
  auto it = ctx->tuned.find(tune_key(kind, dtype, 0, 0));
  if (ctx->stream_k == 0 && it != ctx->tuned.end() &&
      int64_t(it->second.nt) * it->second.c <= n_min) {
    *sh = Shape{it->second.nt, it->second.c};
    *K = int(std::max<int64_t>(1, std::min<int64_t>(it->second.k, int64_t(sh->nt) * sh->c /
                                                                      (4 * per_step))));
    return true;
  }
  for (int i = 0; i < nlist; ++i) {
    int64_t W = int64_t(list[i].nt) * list[i].c;
    if (W <= n_min) {
      *sh = list[i];
      int k = ctx->stream_k > 0 ? ctx->stream_k
                                : (dtype == 0 ? (per_step == 4 ? 32 : (n_min >= 32 * W ? 128 : 64))
                                              : 16 / per_step);
      *K = int(std::max<int64_t>(1, std::min<int64_t>(k, W / (4 * per_step))));
      return true;
    }
  }
  return false;
}

// Builds the plan of one advance call.
static burgers_status build_plan(burgers_ctx* ctx, int scheme, const burgers_batch* batch,
                                 Plan* p, PlanScratch* ext, cudaStream_t ext_stream,
                                 int iters = 1) {
  const int dtype = batch->dtype;
  p->dtype = dtype;
  p->scheme = scheme;
  const int rkind = resident_kind(scheme);
  const bool stencil = scheme == BURGERS_EXPLICIT || scheme == BURGERS_RK4;
  // (the adjoint's transposed solves have only the multi-level path)
  const int64_t rlim = scheme == SCHEME_BTCS_T ? 0 : resident_limit(ctx, rkind, dtype);
  struct Grp {
    Shape sh;
    int exact;
    std::vector<std::pair<double, int64_t>> rows;  // (cost, index)
  };
  std::vector<Grp> groups;
  struct TGrp {
    const KernelEntry* k;
    std::vector<std::pair<double, int64_t>> rows;
  };
  std::vector<TGrp> tgroups;
  std::vector<int64_t> longs;
  // rows per BTCS capacity class (the per-thread Thomas kernel needs many)
  std::map<int64_t, int64_t> class_rows;
  if (scheme == BURGERS_BTCS)
    for (int64_t b = 0; b < batch->count; ++b)
      if (batch->inst[b].nsteps > 0 && batch->inst[b].n <= rlim)
        ++class_rows[resident_class(K_BTCS_RESIDENT, dtype, batch->inst[b].n)];
  for (int64_t b = 0; b < batch->count; ++b) {
    const burgers_instance& in = batch->inst[b];
    if (in.nsteps == 0) continue;
    // long rows: streaming explicit windows / multi-level BTCS (which needs at
    // least a few chunks; shorter rows stay resident whatever the limit)
    const int64_t min_long = stencil ? 128 : 64;
    if (in.n > rlim && in.n >= min_long && in.n > 0) {
      if (!has_long_path(scheme))
        return set_error(BURGERS_EINVAL, "row longer than the resident capacity of this scheme");
      longs.push_back(b);
      continue;
    }
    if (scheme == BURGERS_BTCS) {
      const int64_t cap = resident_class(K_BTCS_RESIDENT, dtype, in.n);
      auto cr = class_rows.find(cap);
      if (const KernelEntry* kt =
              pick_thomas(ctx, dtype, in.n, cr == class_rows.end() ? 0 : cr->second)) {
        TGrp* g = nullptr;
        for (TGrp& x : tgroups)
          if (x.k == kt) g = &x;
        if (!g) {
          tgroups.push_back(TGrp{kt, {}});
          g = &tgroups.back();
        }
        g->rows.emplace_back(double(in.n) * double(in.nsteps), b);
        continue;
      }
    }
    Shape sh = pick_resident(ctx, rkind, dtype, in.n);
    if (sh.nt == 0) return set_error(BURGERS_EINVAL, "no resident kernel shape fits the row");
    int exact = int64_t(sh.nt) * sh.c == in.n ? 1 : 0;
    // ragged FP32 rows of the packed kernels are cut into t = ceil(n / C)
    // chunks of C or C - 1 nodes, which needs t C - n <= t (true for every
    // row of its capacity class; a tuning table could name another shape)
    if (!exact && dtype == 0 && sh.c >= 4 && sh.c % 2 == 0 &&
        (rkind == K_EXPLICIT_RESIDENT || rkind == K_BTCS_RESIDENT || rkind == K_CN_RESIDENT ||
         rkind == K_PICARD_RESIDENT || rkind == K_NEWTON_RESIDENT ||
         (rkind == K_RK4_RESIDENT && sh.c >= 16))) {
      const int64_t t = (int64_t(in.n) + sh.c - 1) / sh.c;
      if (t * sh.c - in.n > t || t > sh.nt)
        return set_error(BURGERS_EINVAL, "row length has no split into chunks of C or C - 1 "
                                         "nodes for its launch shape");
    }
    Grp* g = nullptr;
    for (Grp& x : groups)
      if (x.sh.nt == sh.nt && x.sh.c == sh.c && x.exact == exact) g = &x;
    if (!g) {
      groups.push_back(Grp{sh, exact, {}});
      g = &groups.back();
    }
    g->rows.emplace_back(double(in.n) * double(in.nsteps), b);
  }
  // per-thread Thomas groups: one CTA per nt cost-sorted rows
  for (TGrp& g : tgroups) {
    std::stable_sort(g.rows.begin(), g.rows.end(),
                     [](const auto& a, const auto& b) { return a.first > b.first; });
    const int begin = int(p->rows.size());
    for (auto& pr : g.rows) {
      p->rows.push_back(make_row(batch->inst[pr.second], iters));
      p->row_inst.push_back(int32_t(pr.second));
    }
    Launch L;
    L.k = g.k;
    L.type = LAUNCH_THOMAS;
    L.row_begin = begin;
    L.row_count = int(g.rows.size());
    L.grid = (L.row_count + g.k->nt - 1) / g.k->nt;
    L.ws_elems = int64_t(L.grid) * int64_t(thomas_ws_values(dtype, g.k->nt, g.k->c, g.k->exact));
    p->launches.push_back(L);
  }
  // resident groups
  for (Grp& g : groups) {
    std::stable_sort(g.rows.begin(), g.rows.end(),
                     [](const auto& a, const auto& b) { return a.first > b.first; });
    const KernelEntry* k = find_kernel(rkind, dtype, g.sh.nt, g.sh.c, g.exact);
    if (!k) return set_error(BURGERS_EINVAL, "kernel shape not instantiated");
    int begin = int(p->rows.size());
    for (auto& pr : g.rows) {
      p->rows.push_back(make_row(batch->inst[pr.second], iters));
      p->row_inst.push_back(int32_t(pr.second));
    }
    int cnt = int(g.rows.size());
    if (ctx->plain) {
      for (int i = 0; i < cnt; ++i) {
        Launch L;
        L.k = k;
        L.type = LAUNCH_RESIDENT;
        L.grid = 1;
        L.row_begin = begin + i;
        L.row_count = 1;
        L.counter = p->ncounters++;
        p->launches.push_back(L);
      }
    } else {
      Launch L;
      L.k = k;
      L.type = LAUNCH_RESIDENT;
      L.grid = std::min(cnt, ctx->sm_count * blocks_per_sm(k));
      L.row_begin = begin;
      L.row_count = cnt;
      L.counter = p->ncounters++;
      p->launches.push_back(L);
    }
  }
  if (!longs.empty()) {
    if (stencil) {
      const int skind = scheme == BURGERS_RK4 ? K_RK4_STREAM : K_EXPLICIT_STREAM;
      int64_t nmin = INT64_MAX, smax = 0, span = 0;
      for (int64_t b : longs) {
        nmin = std::min<int64_t>(nmin, batch->inst[b].n);
        smax = std::max<int64_t>(smax, batch->inst[b].nsteps);
        span = std::max<int64_t>(span, batch->inst[b].offset + batch->inst[b].n);
      }
      Shape sh;
      int K;
      if (!pick_stream(ctx, skind, dtype, nmin, &sh, &K))
        return set_error(BURGERS_EINVAL, "row too short for the streaming kernel");
      const KernelEntry* k = nullptr;
      const bool step1 = K == 1 && scheme == BURGERS_EXPLICIT;
      const KernelEntry* kbulk = nullptr;
      if (step1) {  // one Euler step per pass: the bandwidth-bound single-step kernel
        // tile shape from the tuning table if it names one (its k: the stage
        // count of the bulk-copy kernel for the whole tiles, 0 = the per-tile
        // kernel only), else the per-tile kernel with 512 threads of 8 nodes
        // (FP32; measured on a B300 at 0.63 of the HBM copy rate in the method's
        // 8 bytes per cell-update, the bulk-copy ring at 0.60) or 256 of 4 (FP64)
        sh = Shape{dtype == 0 ? 512 : 256, dtype == 0 ? 8 : 4};
        int stages = 0;
        auto it1 = ctx->tuned.find(tune_key(K_EXPLICIT_STEP1, dtype, 0, 0));
        if (it1 != ctx->tuned.end() &&
            find_kernel(K_EXPLICIT_STEP1, dtype, it1->second.nt, it1->second.c, 0)) {
          sh = Shape{it1->second.nt, it1->second.c};
          stages = it1->second.k;
        }
        k = find_kernel(K_EXPLICIT_STEP1, dtype, sh.nt, sh.c, 0);
        // whole tiles move by bulk copies when every row starts 16-byte aligned in
        // the state and in the one-byte compensation buffers (offsets multiple of 16)
        bool aligned = true;
        for (int64_t b : longs) aligned = aligned && batch->inst[b].offset % 16 == 0;
        if (aligned && stages > 0)
          for (const KernelEntry& e : kernel_registry())
            if (e.kind == K_EXPLICIT_STEP1_BULK && e.dtype == dtype && e.nt == sh.nt &&
                e.c == sh.c && e.exact == stages && e.dyn_smem <= ctx->smem_optin)
              kbulk = &e;
      } else {
        k = find_kernel(skind, dtype, sh.nt, sh.c, 0);
      }
      if (!k) return set_error(BURGERS_EINVAL, "streaming shape not instantiated");
      const int64_t H = int64_t(K) * (scheme == BURGERS_RK4 ? 4 : 1);  // stale nodes per side
      const int64_t W = int64_t(sh.nt) * sh.c, O = step1 ? W : W - 2 * H;
      int rbegin = int(p->rows.size());
      int ibegin = int(p->items.size());
      for (size_t q = 0; q < longs.size(); ++q) {
        const burgers_instance& in = batch->inst[longs[q]];
        p->rows.push_back(make_row(in));
        p->row_inst.push_back(int32_t(longs[q]));
      }
      // items: the bulk-copy kernel takes the whole tiles first, the tails last
      int nbulk = -1;
      for (int pass = kbulk ? 0 : 1; pass < 2; ++pass) {
        for (size_t q = 0; q < longs.size(); ++q) {
          const int64_t n = batch->inst[longs[q]].n;
          const int64_t tiles = (n + O - 1) / O;
          for (int64_t t = 0; t < tiles; ++t) {
            const bool whole = (t + 1) * O <= n;
            if (!kbulk || whole == (pass == 0)) p->items.push_back(TileItem{int32_t(q), int32_t(t)});
          }
        }
        if (pass == 0) nbulk = int(p->items.size()) - ibegin;
      }
      int nitems = int(p->items.size()) - ibegin;
      // the per-tile single-step kernel streams with one CTA per tile, so the
      // scheduler overlaps the tiles' memory traffic; the bulk-copy kernel is
      // persistent (its stages keep the traffic in flight)
      int grid = step1 ? std::min(nitems, 1 << 20)
                       : std::min(nitems, ctx->sm_count * blocks_per_sm(k));
      const int grid_bulk = kbulk ? std::max(1, std::min(nitems, ctx->sm_count * blocks_per_sm(kbulk)))
                                  : 0;
      int64_t passes = (smax + K - 1) / K;
      for (int64_t ps = 0; ps < passes; ++ps) {
        Launch L;
        L.k = k;
        L.type = LAUNCH_STREAM;
        L.grid = grid;
        L.row_begin = rbegin;
        L.row_count = int(longs.size());
        L.item_begin = ibegin;
        L.item_count = nitems;
        L.K = K;
        L.step_base = ps * K;
        L.to_scratch = (ps % 2) == 0;
        if (kbulk) { L.k_fallback = k; L.k = kbulk; L.nbulk = nbulk; L.grid = grid_bulk; }
        p->launches.push_back(L);
      }
      if (passes % 2 == 1) {  // result sits in the scratch buffer: copy it back
        Launch L;
        L.k = k;
        L.type = LAUNCH_STREAM;
        L.grid = grid;
        L.row_begin = rbegin;
        L.row_count = int(longs.size());
        L.item_begin = ibegin;
        L.item_count = nitems;
        L.K = K;
        L.step_base = smax;  // every row done: copy-through
        L.to_scratch = false;
        if (kbulk) { L.k_fallback = k; L.k = kbulk; L.nbulk = nbulk; L.grid = grid_bulk; }
        p->launches.push_back(L);
      }
      // the compensation buffers follow the row copy; keep every buffer start
      // 256-byte aligned (the kernels' vector loads need 16-byte alignment)
      span = (span + 255) & ~int64_t(255);
      p->stream_span = span;
      // ping-pong copy of the rows, plus (FP32) two compensation buffers of one
      // byte per node (span / 4 elements each)
      p->scratch_elems = dtype == 0 ? span + span / 2 : span;
    } else {
      // FP32 lagged BTCS, Crank-Nicolson, Picard and Newton rows that fit a
      // cluster stay resident in its shared memory (k_btcs_cluster_x2):
      // 128-thread CTAs of 4096 nodes in clusters of up to 16 where the
      // device schedules them (8 in portable mode), else 256-thread CTAs of
      // 8192 nodes in clusters of up to 8; longer rows go through the
      // multi-level solver, as do rows whose cluster the device cannot
      // schedule for the variant's kernel (the iterating variants also stage
      // the iterate's e).
      std::vector<int64_t> mlrows;
      struct CGrp {
        int nt, c, cs;
        std::vector<std::pair<double, int64_t>> rows;
      };
      std::vector<CGrp> cgroups;
      const bool cl = (scheme == BURGERS_BTCS || scheme == BURGERS_CN ||
                       scheme == BURGERS_PICARD || scheme == BURGERS_NEWTON) &&
                      ctx->cluster && ctx->resident_max == 0 && !ctx->resident_override;
      const int ckind = scheme == BURGERS_CN       ? K_CN_CLUSTER
                        : scheme == BURGERS_PICARD ? K_PICARD_CLUSTER
                        : scheme == BURGERS_NEWTON ? K_NEWTON_CLUSTER
                                                   : K_BTCS_CLUSTER;
      for (int64_t b : longs) {
        const burgers_instance& in = batch->inst[b];
        int nt = 0, c = 0;
        if (cl && dtype == 0) {
          const int64_t cs128 = ctx->cluster == 2 ? 8 : ctx->cluster_cs128;
          if (in.n <= cs128 * 4096) { nt = 128; c = 32; }
          else if (in.n <= 8 * 8192) { nt = 256; c = 32; }
        }
        const int64_t W = int64_t(nt) * c;
        const int cs = nt ? int((in.n + W - 1) / W) : 0;
        const KernelEntry* ck = nt && cs >= 2 ? find_kernel(ckind, dtype, nt, c, cs) : nullptr;
        // (the context's cluster limit was taken on the BTCS kernel; the
        // variants' own kernels are checked with the occupancy API)
        if (!ck || (ckind != K_BTCS_CLUSTER && !cluster_fits(*ck))) {
          mlrows.push_back(b);
          continue;
        }
        CGrp* g = nullptr;
        for (CGrp& x : cgroups)
          if (x.nt == nt && x.c == c && x.cs == cs) g = &x;
        if (!g) {
          cgroups.push_back(CGrp{nt, c, cs, {}});
          g = &cgroups.back();
        }
        g->rows.emplace_back(double(in.n) * double(in.nsteps), b);
      }
      for (CGrp& g : cgroups) {
        std::stable_sort(g.rows.begin(), g.rows.end(),
                         [](const auto& a, const auto& b) { return a.first > b.first; });
        const KernelEntry* k = find_kernel(ckind, dtype, g.nt, g.c, g.cs);
        int begin = int(p->rows.size());
        for (auto& pr : g.rows) {
          p->rows.push_back(make_row(batch->inst[pr.second], iters));
          p->row_inst.push_back(int32_t(pr.second));
        }
        const int cnt = int(g.rows.size());
        // one cluster per row: grid = rows x cluster size
        for (int i0 = 0; i0 < cnt; i0 += ctx->plain ? 1 : cnt) {
          Launch L;
          L.k = k;
          L.type = LAUNCH_RESIDENT;
          L.row_begin = begin + i0;
          L.row_count = ctx->plain ? 1 : cnt;
          L.grid = L.row_count * g.cs;
          L.counter = p->ncounters++;
          p->launches.push_back(L);
        }
      }
      if (!mlrows.empty()) {
        const int var = scheme == BURGERS_CN       ? 1
                        : scheme == BURGERS_PICARD ? 2
                        : scheme == BURGERS_NEWTON ? 3
                        : scheme == SCHEME_BTCS_T  ? 4
                                                   : 0;
        burgers_status st = plan_multilevel(ctx, batch, mlrows, p, var, iters);
        if (st != BURGERS_OK) return st;
      }
    }
  }
  // per-thread Thomas workspaces follow whatever the long rows use of the scratch
  for (Launch& L : p->launches)
    if (L.type == LAUNCH_THOMAS) {
      L.ws_off = (p->scratch_elems + 63) & ~int64_t(63);
      p->scratch_elems = L.ws_off + L.ws_elems;
    }
  // device image: rows | items | counters (+ multilevel descriptors)
  size_t off = 0;
  auto align = [](size_t x) { return (x + 255) & ~size_t(255); };
  p->rows_off = off;
  off = align(off + p->rows.size() * sizeof(RowDesc));
  p->items_off = off;
  off = align(off + p->items.size() * sizeof(TileItem));
  p->counters_off = off;
  off = align(off + size_t(p->ncounters) * sizeof(int));
  p->ml_off = off;
  off = align(off + p->ml_bytes.size());
  p->dev_bytes = off;
  if (off > 0) {
    unsigned char* img = nullptr;
    std::vector<unsigned char> tmp;
    if (ext) {  // reusable buffers of the caller (serving): no allocation per plan
      cudaError_t e = ext->dev.ensure(off);
      if (e == cudaSuccess) e = ext->host.ensure_host(off);
      if (e != cudaSuccess) return set_error(BURGERS_ENOMEM, "plan descriptors: out of memory");
      img = static_cast<unsigned char*>(ext->host.hptr);
      memset(img, 0, off);
      p->dev = ext->dev.ptr;
      p->dev_external = true;
    } else {
      cudaError_t e = cudaMalloc(&p->dev, off);
      if (e != cudaSuccess) return set_error(BURGERS_ENOMEM, "plan descriptors: out of device memory");
      tmp.assign(off, 0);
      img = tmp.data();
    }
    if (!p->rows.empty()) memcpy(img + p->rows_off, p->rows.data(), p->rows.size() * sizeof(RowDesc));
    if (!p->items.empty())
      memcpy(img + p->items_off, p->items.data(), p->items.size() * sizeof(TileItem));
    if (!p->ml_bytes.empty()) memcpy(img + p->ml_off, p->ml_bytes.data(), p->ml_bytes.size());
    cudaError_t e = ext ? cudaMemcpyAsync(p->dev, img, off, cudaMemcpyHostToDevice, ext_stream)
                        : cudaMemcpy(p->dev, img, off, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_error(e, "plan upload");
  }
  for (const Launch& L : p->launches)
    if (L.k) ++p->kernel_launches;
  return BURGERS_OK;
}

Plan::~Plan() {
  if (gexec) cudaGraphExecDestroy(gexec);
  if (dev && !dev_external) cudaFree(dev);
  if (dtdev) cudaFree(dtdev);
}

static cudaError_t enqueue_plan(burgers_ctx* ctx, Plan* p, void* u, cudaStream_t st) {
  char* base = static_cast<char*>(p->dev);
  RowDesc* rows = reinterpret_cast<RowDesc*>(base + p->rows_off);
  TileItem* items = reinterpret_cast<TileItem*>(base + p->items_off);
  int* counters = reinterpret_cast<int*>(base + p->counters_off);
  const size_t esz = p->dtype == 0 ? 4 : 8;
  if (p->ncounters > 0) {
    cudaError_t e = cudaMemsetAsync(counters, 0, sizeof(int) * size_t(p->ncounters), st);
    if (e != cudaSuccess) return e;
  }
  void* scratch = ctx->scratch.ptr;
  void* lo_a = nullptr;
  void* lo_b = nullptr;
  if (p->stream_span > 0 && p->dtype == 0) {  // one compensation byte per node
    lo_a = static_cast<char*>(scratch) + size_t(p->stream_span) * esz;
    lo_b = static_cast<char*>(lo_a) + size_t(p->stream_span);
    cudaError_t e = cudaMemsetAsync(lo_a, 0, size_t(p->stream_span), st);
    if (e != cudaSuccess) return e;
  }
  if (p->ml_span > 0 && p->dtype == 0) {  // multi-level Kahan terms (a byte a node) start at zero
    cudaError_t e = cudaMemsetAsync(static_cast<char*>(scratch) + size_t(p->ml_span) * esz, 0,
                                    size_t(p->ml_span), st);
    if (e != cudaSuccess) return e;
  }
  // Resident launches are independent of each other and of the long-row
  // sequence: spread them over the side streams (forked from and joined back
  // into st) so that one group's tail overlaps the next group's work. The
  // long-row launches keep their order on st.
  int nres = 0;
  for (const Launch& L : p->launches) nres += L.type == LAUNCH_RESIDENT ? 1 : 0;
  const bool fan = nres > 1 && !ctx->plain;
  bool used[burgers_ctx::kSide] = {};
  if (fan) {
    cudaError_t e = cudaEventRecord(ctx->fork_ev, st);
    if (e != cudaSuccess) return e;
  }
  int ri = 0;
  for (const Launch& L : p->launches) {
    cudaError_t e = cudaSuccess;
    if (L.type == LAUNCH_RESIDENT) {
      RowDesc* r = rows + L.row_begin;
      int cnt = L.row_count;
      int* ctr = counters + L.counter;
      void* args[] = {&u, &r, &cnt, &ctr};
      cudaStream_t ls = st;
      const int lane = fan ? ri % (burgers_ctx::kSide + 1) : 0;
      ++ri;
      if (lane > 0) {
        ls = ctx->side[lane - 1];
        if (!used[lane - 1]) {
          e = cudaStreamWaitEvent(ls, ctx->fork_ev, 0);
          if (e != cudaSuccess) return e;
          used[lane - 1] = true;
        }
      }
      e = cudaLaunchKernel(L.k->fn, dim3(L.grid), dim3(L.k->nt), args, L.k->dyn_smem, ls);
    } else if (L.type == LAUNCH_THOMAS) {
      RowDesc* r = rows + L.row_begin;
      int cnt = L.row_count;
      void* ws = static_cast<char*>(scratch) + size_t(L.ws_off) * esz;
      void* args[] = {&u, &r, &cnt, &ws};
      e = cudaLaunchKernel(L.k->fn, dim3(L.grid), dim3(L.k->nt), args, L.k->dyn_smem, st);
    } else if (L.type == LAUNCH_STREAM) {
      const void* src = L.to_scratch ? u : scratch;
      void* dst = L.to_scratch ? scratch : u;
      const void* lsrc = L.to_scratch ? lo_a : lo_b;
      void* ldst = L.to_scratch ? lo_b : lo_a;
      RowDesc* r = rows + L.row_begin;
      TileItem* it = items + L.item_begin;
      int ni = L.item_count, K = L.K;
      int64_t sb = L.step_base;
      const bool bulk_ok = L.nbulk >= 0 && (reinterpret_cast<uintptr_t>(u) & 15) == 0 &&
                           (reinterpret_cast<uintptr_t>(scratch) & 15) == 0;
      if (bulk_ok) {
        int nb = L.nbulk;
        int* err = static_cast<int*>(ctx->errbuf.ptr);
        void* args[] = {&src, &dst, &lsrc, &ldst, &r, &it, &nb, &ni, &sb, &err};
        e = cudaLaunchKernel(L.k->fn, dim3(L.grid), dim3(L.k->nt), args, L.k->dyn_smem, st);
      } else {
        // the per-tile kernel handles any tile (a bulk launch's fallback when the
        // caller's buffer does not start 16-byte aligned)
        const KernelEntry* k1 = L.nbulk >= 0 ? L.k_fallback : L.k;
        const int g1 = L.nbulk >= 0 ? std::min(ni, 1 << 20) : L.grid;
        void* args[] = {&src, &dst, &lsrc, &ldst, &r, &it, &ni, &K, &sb};
        e = cudaLaunchKernel(k1->fn, dim3(g1), dim3(k1->nt), args, k1->dyn_smem, st);
      }
    } else {
      e = enqueue_multilevel_launch(ctx, p, L, u, st);
    }
    if (e != cudaSuccess) return e;
  }
  for (int i = 0; i < burgers_ctx::kSide; ++i) {
    if (!used[i]) continue;
    cudaError_t e = cudaEventRecord(ctx->join_ev[i], ctx->side[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ctx->join_ev[i], 0);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static burgers_status run_plan(burgers_ctx* ctx, Plan* p, void* u, cudaStream_t st,
                               bool allow_graph = true) {
  if (p->scratch_elems > 0) {
    cudaError_t e = ctx->scratch.ensure(size_t(p->scratch_elems) * (p->dtype == 0 ? 4 : 8));
    if (e != cudaSuccess) return set_error(BURGERS_ENOMEM, "streaming scratch: out of device memory");
  }
  if (p->ml_ws_elems > 0) {
    cudaError_t e = ctx->mlws.ensure(size_t(p->ml_ws_elems) * (p->dtype == 0 ? 4 : 8));
    if (e != cudaSuccess) return set_error(BURGERS_ENOMEM, "multi-level workspace: out of device memory");
  }
  const bool use_graph = allow_graph && ctx->graphs && !ctx->plain && p->launches.size() > 1 &&
                         p->launches.size() <= 20000;
  if (use_graph) {
    const bool valid = p->gexec && p->g_u == u && p->g_scratch_gen == ctx->scratch.generation &&
                       p->g_ml_gen == ctx->mlws.generation;
    if (!valid) {
      if (p->gexec) {
        cudaGraphExecDestroy(p->gexec);
        p->gexec = nullptr;
      }
      cudaError_t e = cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_error(e, "begin capture");
      cudaError_t e1 = enqueue_plan(ctx, p, u, ctx->capture_stream);
      cudaGraph_t g = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(ctx->capture_stream, &g);
      if (e1 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_error(e1, "capture enqueue");
      }
      if (e2 != cudaSuccess) return cuda_error(e2, "end capture");
      e = cudaGraphInstantiate(&p->gexec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        p->gexec = nullptr;
        return cuda_error(e, "graph instantiate");
      }
      p->g_u = u;
      p->g_scratch_gen = ctx->scratch.generation;
      p->g_ml_gen = ctx->mlws.generation;
    }
    cudaError_t e = cudaGraphLaunch(p->gexec, st);
    if (e != cudaSuccess) return cuda_error(e, "graph launch");
  } else {
    cudaError_t e = enqueue_plan(ctx, p, u, st);
    if (e != cudaSuccess) return cuda_error(e, "kernel launch");
  }
  ctx->launches += p->kernel_launches;
  return BURGERS_OK;
}

static uint64_t plan_key(const burgers_ctx* ctx, int scheme, const burgers_batch* b, int iters,
                         bool dtdev) {
  uint64_t h = fnv1a(b->inst, sizeof(burgers_instance) * size_t(b->count));
  const int32_t flags = (ctx->plain ? 1 : 0) | (ctx->cluster ? 2 : 0) | (dtdev ? 4 : 0) |
                        (ctx->cluster == 2 ? 8 : 0);
  int32_t hdr[8] = {scheme, b->dtype, flags, ctx->stream_k,
                    int32_t(ctx->resident_max), int32_t(ctx->tune_version), ctx->resident_override,
                    iters};
  return fnv1a(hdr, sizeof hdr, h);
}

Plan* get_plan(burgers_ctx* ctx, int scheme, const burgers_batch* batch, burgers_status* st,
               int iters, bool dtdev) {
  const uint64_t key = plan_key(ctx, scheme, batch, iters, dtdev);
  for (auto it = ctx->plans.begin(); it != ctx->plans.end(); ++it) {
    if ((*it)->key == key && (*it)->count == batch->count) {
      ctx->plans.splice(ctx->plans.begin(), ctx->plans, it);  // most recent first
      *st = BURGERS_OK;
      return ctx->plans.front().get();
    }
  }
  auto p = std::make_unique<Plan>();
  p->key = key;
  p->count = batch->count;
  *st = build_plan(ctx, scheme, batch, p.get(), nullptr, nullptr, iters);
  if (*st != BURGERS_OK) return nullptr;
  ctx->plans.push_front(std::move(p));
  while (ctx->plans.size() > 64) {
    cudaDeviceSynchronize();
    ctx->plans.pop_back();
  }
  return ctx->plans.front().get();
}

burgers_status advance(burgers_ctx* ctx, int scheme, const burgers_batch* batch, void* u_dev,
                       cudaStream_t stream, int iters) {
  if (!ctx) return set_error(BURGERS_EINVAL, "ctx is NULL");
  if (!valid_scheme(scheme)) return set_error(BURGERS_EINVAL, "bad scheme");
  if (iters < 1 || iters > 64) return set_error(BURGERS_EINVAL, "iterations outside [1, 64]");
  burgers_status st = validate_batch(batch, false);
  if (st != BURGERS_OK) return st;
  if (batch->count == 0) return BURGERS_OK;
  if (!u_dev) return set_error(BURGERS_EINVAL, "u_dev is NULL");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_error(e, "cudaSetDevice");
  Plan* p = get_plan(ctx, scheme, batch, &st, iters, false);
  if (!p) return st;
  return run_plan(ctx, p, u_dev, stream);
}

burgers_status transposed_btcs_solve(burgers_ctx* ctx, const burgers_batch* batch, const void* u,
                                     const void* lam, void* nu, cudaStream_t st) {
  burgers_status s = BURGERS_OK;
  Plan* p = get_plan(ctx, SCHEME_BTCS_T, batch, &s, 1, false);
  if (!p) return s;
  const size_t esz = p->dtype == 0 ? 4 : 8;
  cudaError_t e = ctx->scratch.ensure(size_t(p->scratch_elems) * esz);
  if (e != cudaSuccess) return set_error(BURGERS_ENOMEM, "adjoint scratch: out of device memory");
  int64_t cover = 0;  // elements of the caller's buffers the rows cover
  for (int64_t b = 0; b < batch->count; ++b)
    cover = std::max<int64_t>(cover, batch->inst[b].offset + batch->inst[b].n);
  char* ea = static_cast<char*>(ctx->scratch.ptr) + size_t(p->ml_e_off) * esz;
  char* eb = ea + size_t(p->ml_span) * esz;
  e = cudaMemcpyAsync(ea, lam, size_t(cover) * esz, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_error(e, "adjoint lambda copy");
  // the state pointer changes from call to call: direct launches, no graph
  s = run_plan(ctx, p, const_cast<void*>(u), st, false);
  if (s != BURGERS_OK) return s;
  e = cudaMemcpyAsync(nu, eb, size_t(cover) * esz, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_error(e, "adjoint nu copy");
  return BURGERS_OK;
}

// One-off plan through caller-owned descriptor buffers (no cache, no graph):
// the serving loop, whose batch changes every slice. The caller must not
// reuse `ps` before the work enqueued here has consumed the upload.
// Two uncached calls on disjoint rows of the same buffer (the serving loop's
// explicit and BTCS slices). When at most one of the plans needs the
// context's scratch buffers they run concurrently, the second on stream_b
// forked from and joined back into stream_a; otherwise one after the other.
burgers_status advance_uncached_pair(burgers_ctx* ctx, int scheme_a, const burgers_batch* a,
                                     PlanScratch* ps_a, int scheme_b, const burgers_batch* b,
                                     PlanScratch* ps_b, void* u_dev, cudaStream_t stream_a,
                                     cudaStream_t stream_b, cudaEvent_t fork, cudaEvent_t join) {
  const bool has_a = a->count > 0, has_b = b->count > 0;
  burgers_status st = BURGERS_OK;
  if (has_a && (st = validate_batch(a, false)) != BURGERS_OK) return st;
  if (has_b && (st = validate_batch(b, false)) != BURGERS_OK) return st;
  Plan pa, pb;
  if (has_a && (st = build_plan(ctx, scheme_a, a, &pa, ps_a, stream_a)) != BURGERS_OK) return st;
  if (has_b && (st = build_plan(ctx, scheme_b, b, &pb, ps_b, stream_a)) != BURGERS_OK) return st;
  const bool scratch_a = pa.scratch_elems > 0 || pa.ml_ws_elems > 0;
  const bool scratch_b = pb.scratch_elems > 0 || pb.ml_ws_elems > 0;
  if (!has_a || !has_b || (scratch_a && scratch_b)) {
    if (has_a && (st = run_plan(ctx, &pa, u_dev, stream_a, false)) != BURGERS_OK) return st;
    if (has_b) st = run_plan(ctx, &pb, u_dev, stream_a, false);
    return st;
  }
  cudaError_t e = cudaEventRecord(fork, stream_a);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(stream_b, fork, 0);
  if (e != cudaSuccess) return cuda_error(e, "fork");
  if ((st = run_plan(ctx, &pb, u_dev, stream_b, false)) != BURGERS_OK) return st;
  if ((st = run_plan(ctx, &pa, u_dev, stream_a, false)) != BURGERS_OK) return st;
  e = cudaEventRecord(join, stream_b);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(stream_a, join, 0);
  if (e != cudaSuccess) return cuda_error(e, "join");
  return BURGERS_OK;
}

burgers_status advance_uncached(burgers_ctx* ctx, int scheme, const burgers_batch* batch,
                                void* u_dev, cudaStream_t stream, PlanScratch* ps) {
  burgers_status st = validate_batch(batch, false);
  if (st != BURGERS_OK) return st;
  if (batch->count == 0) return BURGERS_OK;
  Plan p;
  st = build_plan(ctx, scheme, batch, &p, ps, stream);
  if (st != BURGERS_OK) return st;
  return run_plan(ctx, &p, u_dev, stream, false);
}

}  // namespace burgers

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

burgers_status burgers_ctx_create(int device, burgers_ctx** out) {
  if (!out) return set_error(BURGERS_EINVAL, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDeviceCount");
  if (device < 0 || device >= ndev) return set_error(BURGERS_EINVAL, "bad device index");
  e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_error(e, "cudaSetDevice");
  auto ctx = std::make_unique<burgers_ctx>();
  ctx->device = device;
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, device);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDeviceProperties");
  ctx->sm_count = prop.multiProcessorCount;
  ctx->smem_optin = prop.sharedMemPerBlockOptin;
  e = prepare_kernels();
  if (e != cudaSuccess) return cuda_error(e, "kernel attributes");
  for (int cs = 9; cs <= 16; ++cs) {  // wide clusters: every size up to the largest that fits
    const KernelEntry* k = find_kernel(K_BTCS_CLUSTER, 0, 128, 32, cs);
    if (!k || !cluster_fits(*k)) break;
    ctx->cluster_cs128 = cs;
  }
  e = cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamCreate");
  for (int i = 0; i < burgers_ctx::kSide && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&ctx->side[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->join_ev[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = ctx->errbuf.ensure(256);
  if (e == cudaSuccess) e = cudaMemset(ctx->errbuf.ptr, 0, 256);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->io_h2d, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->io_d2h, cudaStreamNonBlocking);
  for (int i = 0; i < burgers_ctx::kIoChunks && e == cudaSuccess; ++i) {
    e = cudaEventCreateWithFlags(&ctx->io_in[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->io_out[i], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamCreate");
  *out = ctx.release();
  return BURGERS_OK;
}

void burgers_ctx_destroy(burgers_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  ctx->plans.clear();
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  for (int i = 0; i < burgers_ctx::kSide; ++i) {
    if (ctx->side[i]) cudaStreamDestroy(ctx->side[i]);
    if (ctx->join_ev[i]) cudaEventDestroy(ctx->join_ev[i]);
  }
  if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
  for (int i = 0; i < burgers_ctx::kIoChunks; ++i) {
    if (ctx->io_in[i]) cudaEventDestroy(ctx->io_in[i]);
    if (ctx->io_out[i]) cudaEventDestroy(ctx->io_out[i]);
  }
  if (ctx->io_h2d) cudaStreamDestroy(ctx->io_h2d);
  if (ctx->io_d2h) cudaStreamDestroy(ctx->io_d2h);
  if (ctx->adj_event) cudaEventDestroy(ctx->adj_event);
  if (ctx->adjl_event) cudaEventDestroy(ctx->adjl_event);
  delete ctx;
}

const char* burgers_last_error(void) { return g_last_error.c_str(); }

burgers_status burgers_ctx_set(burgers_ctx* ctx, int32_t option, int64_t value) {
  if (!ctx) return set_error(BURGERS_EINVAL, "ctx is NULL");
  switch (option) {
    case BURGERS_OPT_GRAPHS: ctx->graphs = value != 0; return BURGERS_OK;
    case BURGERS_OPT_PLAIN: ctx->plain = value != 0; return BURGERS_OK;
    case BURGERS_OPT_STREAM_K:
      if (value < 0 || value > 64) return set_error(BURGERS_EINVAL, "stream K out of range");
      ctx->stream_k = int(value);
      return BURGERS_OK;
    case BURGERS_OPT_RESIDENT_MAX:
      if (value < 0 || value > (int64_t(1) << 30)) return set_error(BURGERS_EINVAL, "bad resident max");
      ctx->resident_max = value;
      return BURGERS_OK;
    case BURGERS_OPT_AUTOTUNE: ctx->autotune = value != 0; return BURGERS_OK;
    case BURGERS_OPT_LAUNCH_COUNT: ctx->launches = 0; return BURGERS_OK;
    case BURGERS_OPT_CLUSTER:
      if (value < 0 || value > 2) return set_error(BURGERS_EINVAL, "cluster mode is 0, 1 or 2");
      ctx->cluster = int(value);
      return BURGERS_OK;
    default: return set_error(BURGERS_EINVAL, "unknown option");
  }
}

burgers_status burgers_ctx_get(const burgers_ctx* ctx, int32_t key, int64_t* value) {
  if (!ctx || !value) return set_error(BURGERS_EINVAL, "NULL pointer");
  int64_t v = 0;
  switch (key) {
    case BURGERS_OPT_GRAPHS: v = ctx->graphs ? 1 : 0; break;
    case BURGERS_OPT_PLAIN: v = ctx->plain ? 1 : 0; break;
    case BURGERS_OPT_STREAM_K: v = ctx->stream_k; break;
    case BURGERS_OPT_RESIDENT_MAX: v = ctx->resident_max; break;
    case BURGERS_OPT_AUTOTUNE: v = ctx->autotune ? 1 : 0; break;
    case BURGERS_OPT_CLUSTER: v = ctx->cluster; break;
    case BURGERS_INFO_SM_COUNT: v = ctx->sm_count; break;
    case BURGERS_INFO_CLUSTER_CTAS_MAX: v = ctx->cluster_cs128; break;
    default: return set_error(BURGERS_EINVAL, "unknown key");
  }
  *value = v;
  return BURGERS_OK;
}

int64_t burgers_launch_count(const burgers_ctx* ctx) { return ctx ? ctx->launches.load() : 0; }

burgers_status burgers_device_error(burgers_ctx* ctx, int32_t* bits, int32_t clear) {
  if (!ctx || !bits) return set_error(BURGERS_EINVAL, "NULL pointer");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int32_t v = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&v, ctx->errbuf.ptr, sizeof v, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && clear) e = cudaMemset(ctx->errbuf.ptr, 0, sizeof v);
  if (e != cudaSuccess) return cuda_error(e, "device error word");
  *bits = v;
  return BURGERS_OK;
}

burgers_status burgers_explicit_advance(burgers_ctx* ctx, const burgers_batch* batch, void* u_dev,
                                        burgers_stream stream) {
  return advance(ctx, BURGERS_EXPLICIT, batch, u_dev, reinterpret_cast<cudaStream_t>(stream));
}

burgers_status burgers_btcs_advance(burgers_ctx* ctx, const burgers_batch* batch, void* u_dev,
                                    burgers_stream stream) {
  return advance(ctx, BURGERS_BTCS, batch, u_dev, reinterpret_cast<cudaStream_t>(stream));
}

burgers_status burgers_rk4_advance(burgers_ctx* ctx, const burgers_batch* batch, void* u_dev,
                                   burgers_stream stream) {
  return advance(ctx, BURGERS_RK4, batch, u_dev, reinterpret_cast<cudaStream_t>(stream));
}

burgers_status burgers_cn_advance(burgers_ctx* ctx, const burgers_batch* batch, void* u_dev,
                                  burgers_stream stream) {
  return advance(ctx, BURGERS_CN, batch, u_dev, reinterpret_cast<cudaStream_t>(stream));
}

burgers_status burgers_picard_advance(burgers_ctx* ctx, const burgers_batch* batch, void* u_dev,
                                      int32_t iters, burgers_stream stream) {
  return advance(ctx, BURGERS_PICARD, batch, u_dev, reinterpret_cast<cudaStream_t>(stream), iters);
}

burgers_status burgers_newton_advance(burgers_ctx* ctx, const burgers_batch* batch, void* u_dev,
                                      int32_t iters, burgers_stream stream) {
  return advance(ctx, BURGERS_NEWTON, batch, u_dev, reinterpret_cast<cudaStream_t>(stream), iters);
}

burgers_status burgers_adjoint(burgers_ctx* ctx, int32_t scheme, const burgers_batch* batch,
                               const void* u0_dev, const void* gT_dev, void* gu0_dev,
                               double* gnu_dev, int64_t ckpt_stride, burgers_stream stream) {
  if (!ctx) return set_error(BURGERS_EINVAL, "ctx is NULL");
  if (scheme != BURGERS_EXPLICIT && scheme != BURGERS_BTCS) return set_error(BURGERS_EINVAL, "bad scheme");
  if (ckpt_stride < 0) return set_error(BURGERS_EINVAL, "negative checkpoint stride");
  burgers_status st = validate_batch(batch, false);
  if (st != BURGERS_OK) return st;
  if (batch->count == 0) return BURGERS_OK;
  if (!u0_dev || !gT_dev || !gu0_dev || !gnu_dev) return set_error(BURGERS_EINVAL, "NULL pointer");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_error(e, "cudaSetDevice");
  return adjoint_run(ctx, scheme, batch, u0_dev, gT_dev, gu0_dev, gnu_dev, ckpt_stride,
                     reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"

namespace burgers {

// Reduction plan: one item per (row, chunk of NORM_CHUNK nodes).
static burgers_status reduction_setup(burgers_ctx* ctx, const burgers_batch* batch,
                                      std::vector<RowDesc>* rows, std::vector<TileItem>* items,
                                      std::vector<int32_t>* first) {
  rows->clear();
  items->clear();
  first->assign(size_t(batch->count) + 1, 0);
  for (int64_t b = 0; b < batch->count; ++b) {
    rows->push_back(make_row(batch->inst[b]));
    (*first)[size_t(b)] = int32_t(items->size());
    int64_t chunks = (batch->inst[b].n + NORM_CHUNK - 1) / NORM_CHUNK;
    for (int64_t c = 0; c < chunks; ++c) items->push_back(TileItem{int32_t(b), int32_t(c)});
  }
  (*first)[size_t(batch->count)] = int32_t(items->size());
  (void)ctx;
  return BURGERS_OK;
}

// Uploads a reduction plan into the context's reduction workspace.
static burgers_status reduction_upload(burgers_ctx* ctx, const std::vector<RowDesc>& rows,
                                       const std::vector<TileItem>& items,
                                       const std::vector<int32_t>& first, size_t extra_bytes,
                                       const void* extra, cudaStream_t st, char** base_out) {
  auto align = [](size_t x) { return (x + 255) & ~size_t(255); };
  size_t o_rows = 0;
  size_t o_items = align(rows.size() * sizeof(RowDesc));
  size_t o_first = align(o_items + items.size() * sizeof(TileItem));
  size_t o_extra = align(o_first + first.size() * sizeof(int32_t));
  size_t o_partial = align(o_extra + extra_bytes);
  size_t o_out = align(o_partial + items.size() * sizeof(double2));
  size_t total = align(o_out + 2 * rows.size() * sizeof(double));
  cudaError_t e = ctx->redws.ensure(total);
  if (e != cudaSuccess) return set_error(BURGERS_ENOMEM, "reduction workspace");
  e = ctx->redhost.ensure_host(o_partial);
  if (e != cudaSuccess) return set_error(BURGERS_ENOMEM, "pinned staging");
  char* h = static_cast<char*>(ctx->redhost.hptr);
  memcpy(h + o_rows, rows.data(), rows.size() * sizeof(RowDesc));
  memcpy(h + o_items, items.data(), items.size() * sizeof(TileItem));
  memcpy(h + o_first, first.data(), first.size() * sizeof(int32_t));
  if (extra_bytes) memcpy(h + o_extra, extra, extra_bytes);
  e = cudaMemcpyAsync(ctx->redws.ptr, h, o_partial, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_error(e, "reduction upload");
  *base_out = static_cast<char*>(ctx->redws.ptr);
  ctx->red_offsets[0] = o_rows;
  ctx->red_offsets[1] = o_items;
  ctx->red_offsets[2] = o_first;
  ctx->red_offsets[3] = o_extra;
  ctx->red_offsets[4] = o_partial;
  ctx->red_offsets[5] = o_out;
  return BURGERS_OK;
}

cudaError_t HostBuf::ensure_host(size_t need) {
  if (need <= bytes) return cudaSuccess;
  if (hptr) cudaFreeHost(hptr);
  hptr = nullptr;
  bytes = 0;
  size_t want = std::max(need, size_t(1) << 16);
  cudaError_t e = cudaMallocHost(&hptr, want);
  if (e != cudaSuccess) {
    hptr = nullptr;
    return e;
  }
  bytes = want;
  return cudaSuccess;
}

HostBuf::~HostBuf() {
  if (hptr) cudaFreeHost(hptr);
}

}  // namespace burgers

// Row coefficients of a device-dt plan from the per-instance dt on the device:
// the same FP64 operations as make_row on dt = factor * dt_dev[b], so a
// device-dt advance gives bitwise the result of a host advance with that dt.
// An instance without a finite CFL limit (dt_dev < 0: u == 0 and nu == 0)
// gets dt = 0, which leaves its row as it is.
__global__ void k_rows_from_dt(RowDesc* __restrict__ rows, const int32_t* __restrict__ row_inst,
                               const double2* __restrict__ dxnu, const double* __restrict__ dt_dev,
                               double factor, int nrows) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrows) return;
  const int b = row_inst[i];
  const double d0 = dt_dev[b];
  const double dt = d0 > 0.0 ? d0 * factor : 0.0;
  const double dx = dxnu[b].x, nu = dxnu[b].y;
  rows[i].r = dt / dx;
  rows[i].s = nu * dt / (dx * dx);
  rows[i].ds_dnu = dt / (dx * dx);
  set_fp32_coefs(rows[i]);
}

// The batch with dt and nsteps replaced by placeholders (the device-dt
// entry points ignore the rows' dt; the CFL reduction also their nsteps).
static std::vector<burgers_instance> placeholder_dt(const burgers_batch* batch, bool keep_steps) {
  std::vector<burgers_instance> tmp(batch->inst, batch->inst + batch->count);
  for (auto& in : tmp) {
    in.dt = 1.0;
    if (!keep_steps) in.nsteps = 0;
  }
  return tmp;
}

extern "C" {

burgers_status burgers_rel_l2(burgers_ctx* ctx, const burgers_batch* batch, const void* u_dev,
                              const void* ref_dev, int32_t ref_dtype, double* out_host,
                              double* rms_host, burgers_stream stream) {
  if (!ctx) return set_error(BURGERS_EINVAL, "ctx is NULL");
  burgers_status st = validate_batch(batch, false);
  if (st != BURGERS_OK) return st;
  if (batch->count == 0) return BURGERS_OK;
  if (!u_dev || !ref_dev || !out_host) return set_error(BURGERS_EINVAL, "NULL pointer");
  if (ref_dtype != BURGERS_F32 && ref_dtype != BURGERS_F64) return set_error(BURGERS_EINVAL, "bad ref dtype");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_error(e, "cudaSetDevice");
  std::vector<RowDesc> rows;
  std::vector<TileItem> items;
  std::vector<int32_t> first;
  reduction_setup(ctx, batch, &rows, &items, &first);
  char* base = nullptr;
  st = reduction_upload(ctx, rows, items, first, 0, nullptr, s, &base);
  if (st != BURGERS_OK) return st;
  auto* o = ctx->red_offsets;
  double* rel_d = reinterpret_cast<double*>(base + o[5]);
  double* rms_d = rel_d + rows.size();
  e = launch_rel_l2(batch->dtype, ref_dtype, u_dev, ref_dev,
                    reinterpret_cast<RowDesc*>(base + o[0]), reinterpret_cast<TileItem*>(base + o[1]),
                    int(items.size()), reinterpret_cast<int32_t*>(base + o[2]), int(rows.size()),
                    NORM_CHUNK, reinterpret_cast<double2*>(base + o[4]), rel_d, rms_d, s);
  if (e != cudaSuccess) return cuda_error(e, "rel_l2 launch");
  ctx->launches += 2;
  std::vector<double> tmp(2 * rows.size());
  e = cudaMemcpyAsync(tmp.data(), rel_d, 2 * rows.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_error(e, "rel_l2");
  memcpy(out_host, tmp.data(), rows.size() * sizeof(double));
  if (rms_host) memcpy(rms_host, tmp.data() + rows.size(), rows.size() * sizeof(double));
  return BURGERS_OK;
}

burgers_status burgers_cfl_dt(burgers_ctx* ctx, const burgers_batch* batch, const void* u_dev,
                              double cfl, double* dt_host, burgers_stream stream) {
  if (!ctx) return set_error(BURGERS_EINVAL, "ctx is NULL");
  if (!batch || batch->count < 0 || (batch->count > 0 && !batch->inst))
    return set_error(BURGERS_EINVAL, "bad batch");
  if (batch->count == 0) return BURGERS_OK;
  if (!u_dev || !dt_host) return set_error(BURGERS_EINVAL, "NULL pointer");
  if (!(cfl > 0.0)) return set_error(BURGERS_EINVAL, "cfl must be > 0");
  // dt and nsteps of the rows are ignored: check the rest with placeholders
  std::vector<burgers_instance> tmp(batch->inst, batch->inst + batch->count);
  for (auto& in : tmp) {
    in.dt = 1.0;
    in.nsteps = 0;
  }
  burgers_batch b2 = *batch;
  b2.inst = tmp.data();
  burgers_status st = validate_batch(&b2, false);
  if (st != BURGERS_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_error(e, "cudaSetDevice");
  std::vector<RowDesc> rows;
  std::vector<TileItem> items;
  std::vector<int32_t> first;
  reduction_setup(ctx, &b2, &rows, &items, &first);
  std::vector<double2> dxnu(size_t(batch->count));
  for (int64_t b = 0; b < batch->count; ++b) dxnu[size_t(b)] = make_double2(tmp[b].dx, tmp[b].nu);
  char* base = nullptr;
  st = reduction_upload(ctx, rows, items, first, dxnu.size() * sizeof(double2), dxnu.data(), s, &base);
  if (st != BURGERS_OK) return st;
  auto* o = ctx->red_offsets;
  double* dt_d = reinterpret_cast<double*>(base + o[5]);
  e = launch_cfl(batch->dtype, u_dev, reinterpret_cast<RowDesc*>(base + o[0]),
                 reinterpret_cast<TileItem*>(base + o[1]), int(items.size()),
                 reinterpret_cast<int32_t*>(base + o[2]), reinterpret_cast<double2*>(base + o[3]),
                 int(rows.size()), NORM_CHUNK, cfl, reinterpret_cast<double*>(base + o[4]), dt_d, s);
  if (e != cudaSuccess) return cuda_error(e, "cfl launch");
  ctx->launches += 2;
  e = cudaMemcpyAsync(dt_host, dt_d, rows.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_error(e, "cfl_dt");
  for (size_t b = 0; b < rows.size(); ++b)
    if (dt_host[b] < 0) return set_error(BURGERS_EINVAL, "a row has no finite CFL limit");
  return BURGERS_OK;
}

burgers_status burgers_solve_host(burgers_ctx* ctx, int32_t scheme, const burgers_batch* batch,
                                  void* u_host, burgers_stream stream) {
  if (!ctx) return set_error(BURGERS_EINVAL, "ctx is NULL");
  if (!valid_scheme(scheme)) return set_error(BURGERS_EINVAL, "bad scheme");
  burgers_status st = validate_batch(batch, false);
  if (st != BURGERS_OK) return st;
  if (batch->count == 0) return BURGERS_OK;
  if (!u_host) return set_error(BURGERS_EINVAL, "u_host is NULL");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_error(e, "cudaSetDevice");
  const size_t esz = batch->dtype == BURGERS_F32 ? 4 : 8;
  // rows in offset order, cut into up to kIoChunks chunks of whole rows: the
  // copy of chunk c+1 in overlaps the solve of chunk c, and the copy of chunk
  // c out overlaps the solve of chunk c+1 (copy streams, event-ordered)
  std::vector<int64_t> order(static_cast<size_t>(batch->count));
  for (int64_t b = 0; b < batch->count; ++b) order[size_t(b)] = b;
  std::sort(order.begin(), order.end(), [&](int64_t x, int64_t y) {
    return batch->inst[x].offset < batch->inst[y].offset;
  });
  int64_t lo = INT64_MAX, hi = 0;
  for (int64_t b = 0; b < batch->count; ++b) {
    lo = std::min<int64_t>(lo, batch->inst[b].offset);
    hi = std::max<int64_t>(hi, batch->inst[b].offset + batch->inst[b].n);
  }
  e = ctx->iobuf.ensure(size_t(hi - lo) * esz);
  if (e != cudaSuccess) return set_error(BURGERS_ENOMEM, "host-solve buffer: out of device memory");
  const int nch = int(std::min<int64_t>(batch->count >= 64 ? burgers_ctx::kIoChunks : 1,
                                        batch->count));
  char* dbase = static_cast<char*>(ctx->iobuf.ptr);
  char* hbase = static_cast<char*>(u_host);
  // per chunk: its rows (offsets relative to lo) and merged contiguous host spans
  std::vector<std::vector<burgers_instance>> cinst(static_cast<size_t>(nch));
  std::vector<std::vector<std::pair<int64_t, int64_t>>> cruns(static_cast<size_t>(nch));
  for (int c = 0; c < nch; ++c) {
    const int64_t r0 = batch->count * c / nch, r1 = batch->count * (c + 1) / nch;
    for (int64_t i = r0; i < r1; ++i) {
      burgers_instance in = batch->inst[order[size_t(i)]];
      const int64_t a = in.offset, z = in.offset + in.n;
      auto& rn = cruns[size_t(c)];
      if (!rn.empty() && rn.back().second == a) rn.back().second = z;
      else rn.emplace_back(a, z);
      in.offset -= lo;
      cinst[size_t(c)].push_back(in);
    }
  }
  const bool pipe = nch > 1;
  cudaStream_t sin = pipe ? ctx->io_h2d : s, sout = pipe ? ctx->io_d2h : s;
  if (pipe) {  // the copies start after whatever the caller queued on s
    e = cudaEventRecord(ctx->io_out[0], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sin, ctx->io_out[0], 0);
    if (e != cudaSuccess) return cuda_error(e, "solve_host order");
  }
  for (int c = 0; c < nch; ++c) {
    for (auto& rn : cruns[size_t(c)]) {
      e = cudaMemcpyAsync(dbase + (rn.first - lo) * esz, hbase + rn.first * esz,
                          size_t(rn.second - rn.first) * esz, cudaMemcpyHostToDevice, sin);
      if (e != cudaSuccess) return cuda_error(e, "solve_host H2D");
    }
    if (pipe) {
      e = cudaEventRecord(ctx->io_in[c], sin);
      if (e != cudaSuccess) return cuda_error(e, "solve_host record");
    }
  }
  // consecutive chunks alternate between two compute streams so that the tail
  // of one chunk's persistent launch overlaps the start of the next
  for (int c = 0; c < nch; ++c) {
    cudaStream_t sc = (pipe && (c & 1)) ? ctx->side[burgers_ctx::kSide - 1] : s;
    if (pipe) {
      e = cudaStreamWaitEvent(sc, ctx->io_in[c], 0);
      if (e != cudaSuccess) return cuda_error(e, "solve_host wait");
    }
    burgers_batch bc = *batch;
    bc.count = int64_t(cinst[size_t(c)].size());
    bc.inst = cinst[size_t(c)].data();
    st = advance(ctx, scheme, &bc, dbase, sc);
    if (st != BURGERS_OK) return st;
    if (pipe) {
      e = cudaEventRecord(ctx->io_out[c], sc);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(sout, ctx->io_out[c], 0);
      if (e != cudaSuccess) return cuda_error(e, "solve_host order");
    }
    for (auto& rn : cruns[size_t(c)]) {
      e = cudaMemcpyAsync(hbase + rn.first * esz, dbase + (rn.first - lo) * esz,
                          size_t(rn.second - rn.first) * esz, cudaMemcpyDeviceToHost, sout);
      if (e != cudaSuccess) return cuda_error(e, "solve_host D2H");
    }
  }
  e = cudaStreamSynchronize(sout);
  if (e == cudaSuccess && pipe) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && pipe) e = cudaStreamSynchronize(ctx->side[burgers_ctx::kSide - 1]);
  if (e != cudaSuccess) return cuda_error(e, "solve_host sync");
  return BURGERS_OK;
}

burgers_status burgers_cfl_dt_device(burgers_ctx* ctx, const burgers_batch* batch,
                                     const void* u_dev, double cfl, double* dt_dev,
                                     burgers_stream stream) {
  if (!ctx) return set_error(BURGERS_EINVAL, "ctx is NULL");
  if (!batch || batch->count < 0 || (batch->count > 0 && !batch->inst))
    return set_error(BURGERS_EINVAL, "bad batch");
  if (batch->count == 0) return BURGERS_OK;
  if (!u_dev || !dt_dev) return set_error(BURGERS_EINVAL, "NULL pointer");
  if (!(cfl > 0.0)) return set_error(BURGERS_EINVAL, "cfl must be > 0");
  std::vector<burgers_instance> tmp = placeholder_dt(batch, false);
  burgers_batch b2 = *batch;
  b2.inst = tmp.data();
  burgers_status st = validate_batch(&b2, false);
  if (st != BURGERS_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_error(e, "cudaSetDevice");
  // the reduction's descriptors depend on the batch layout only: built and
  // uploaded once per layout, then reused by every call (no host staging)
  int32_t hdr[2] = {batch->dtype, 0};
  const uint64_t key = fnv1a(hdr, sizeof hdr, fnv1a(tmp.data(), tmp.size() * sizeof(burgers_instance)));
  auto it = ctx->redcache.find(key);
  if (it == ctx->redcache.end()) {
    if (ctx->redcache.size() >= 16) {  // bounded: drop the cached layouts
      e = cudaDeviceSynchronize();
      if (e != cudaSuccess) return cuda_error(e, "cfl cache");
      for (auto& kv : ctx->redcache) cudaFree(kv.second.dev);
      ctx->redcache.clear();
    }
    std::vector<RowDesc> rows;
    std::vector<TileItem> items;
    std::vector<int32_t> first;
    reduction_setup(ctx, &b2, &rows, &items, &first);
    std::vector<double2> dxnu(size_t(batch->count));
    for (int64_t b = 0; b < batch->count; ++b) dxnu[size_t(b)] = make_double2(tmp[b].dx, tmp[b].nu);
    auto align = [](size_t x) { return (x + 255) & ~size_t(255); };
    RedCache rc;
    rc.off[0] = 0;
    rc.off[1] = align(rows.size() * sizeof(RowDesc));
    rc.off[2] = align(rc.off[1] + items.size() * sizeof(TileItem));
    rc.off[3] = align(rc.off[2] + first.size() * sizeof(int32_t));
    rc.off[4] = align(rc.off[3] + dxnu.size() * sizeof(double2));
    const size_t total = align(rc.off[4] + items.size() * sizeof(double));
    rc.nrows = int(rows.size());
    rc.nitems = int(items.size());
    std::vector<unsigned char> img(rc.off[4], 0);
    memcpy(img.data() + rc.off[0], rows.data(), rows.size() * sizeof(RowDesc));
    memcpy(img.data() + rc.off[1], items.data(), items.size() * sizeof(TileItem));
    memcpy(img.data() + rc.off[2], first.data(), first.size() * sizeof(int32_t));
    memcpy(img.data() + rc.off[3], dxnu.data(), dxnu.size() * sizeof(double2));
    e = cudaMalloc(&rc.dev, total);
    if (e != cudaSuccess) return set_error(BURGERS_ENOMEM, "cfl descriptors: out of device memory");
    e = cudaMemcpy(rc.dev, img.data(), img.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(rc.dev);
      return cuda_error(e, "cfl descriptors");
    }
    it = ctx->redcache.emplace(key, rc).first;
  }
  const RedCache& rc = it->second;
  char* base = static_cast<char*>(rc.dev);
  e = launch_cfl(batch->dtype, u_dev, reinterpret_cast<RowDesc*>(base + rc.off[0]),
                 reinterpret_cast<TileItem*>(base + rc.off[1]), rc.nitems,
                 reinterpret_cast<int32_t*>(base + rc.off[2]), reinterpret_cast<double2*>(base + rc.off[3]),
                 rc.nrows, NORM_CHUNK, cfl, reinterpret_cast<double*>(base + rc.off[4]), dt_dev, s);
  if (e != cudaSuccess) return cuda_error(e, "cfl launch");
  ctx->launches += 2;
  return BURGERS_OK;
}

burgers_status burgers_advance_dt_device(burgers_ctx* ctx, int32_t scheme,
                                         const burgers_batch* batch, void* u_dev,
                                         const double* dt_dev, double dt_factor, int32_t iters,
                                         burgers_stream stream) {
  if (!ctx) return set_error(BURGERS_EINVAL, "ctx is NULL");
  if (!valid_scheme(scheme)) return set_error(BURGERS_EINVAL, "bad scheme");
  if (iters < 1 || iters > 64) return set_error(BURGERS_EINVAL, "iterations outside [1, 64]");
  if (!batch || batch->count < 0 || (batch->count > 0 && !batch->inst))
    return set_error(BURGERS_EINVAL, "bad batch");
  if (batch->count == 0) return BURGERS_OK;
  if (!u_dev || !dt_dev) return set_error(BURGERS_EINVAL, "NULL pointer");
  if (!(dt_factor > 0.0)) return set_error(BURGERS_EINVAL, "dt_factor must be > 0");
  std::vector<burgers_instance> tmp = placeholder_dt(batch, true);
  burgers_batch b2 = *batch;
  b2.inst = tmp.data();
  burgers_status st = validate_batch(&b2, false);
  if (st != BURGERS_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_error(e, "cudaSetDevice");
  const int it_used = (scheme == BURGERS_PICARD || scheme == BURGERS_NEWTON) ? iters : 1;
  Plan* p = get_plan(ctx, scheme, &b2, &st, it_used, true);
  if (!p) return st;
  if (p->ml_rows > 0)
    return set_error(BURGERS_EINVAL,
                     "device dt: rows that take the multi-level solver are not supported");
  if (!p->rows.empty()) {
    if (!p->dtdev) {  // the plan's map from rows to instances and their (dx, nu), once
      const size_t o_dx = (p->row_inst.size() * sizeof(int32_t) + 255) & ~size_t(255);
      std::vector<unsigned char> img(o_dx + size_t(batch->count) * sizeof(double2), 0);
      memcpy(img.data(), p->row_inst.data(), p->row_inst.size() * sizeof(int32_t));
      double2* dxnu = reinterpret_cast<double2*>(img.data() + o_dx);
      for (int64_t b = 0; b < batch->count; ++b) dxnu[b] = make_double2(tmp[b].dx, tmp[b].nu);
      e = cudaMalloc(&p->dtdev, img.size());
      if (e != cudaSuccess) {
        p->dtdev = nullptr;
        return set_error(BURGERS_ENOMEM, "device-dt descriptors: out of device memory");
      }
      e = cudaMemcpy(p->dtdev, img.data(), img.size(), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return cuda_error(e, "device-dt descriptors");
    }
    const size_t o_dx = (p->row_inst.size() * sizeof(int32_t) + 255) & ~size_t(255);
    const int nrows = int(p->rows.size());
    RowDesc* rows = reinterpret_cast<RowDesc*>(static_cast<char*>(p->dev) + p->rows_off);
    k_rows_from_dt<<<(nrows + 255) / 256, 256, 0, s>>>(
        rows, static_cast<const int32_t*>(p->dtdev),
        reinterpret_cast<const double2*>(static_cast<char*>(p->dtdev) + o_dx), dt_dev, dt_factor, nrows);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "device-dt rows");
    ctx->launches += 1;
  }
  return run_plan(ctx, p, u_dev, s);
}

}  // extern "C"
