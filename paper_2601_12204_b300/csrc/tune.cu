// tune.cu -- launch-shape autotuner and its persistent table.
//
// For every capacity class present in a batch (resident kernels: all
// registered (threads, nodes-per-thread) shapes of that capacity; streaming
// explicit kernel: window shapes x steps-per-pass K) the tuner copies up to
// TUNE_ROWS of the caller's rows into a private buffer, runs each candidate
// for a bounded number of steps, times it with CUDA events on the caller's
// stream and records the fastest in the context's table. Plans built after
// tuning use the table (the plan cache key includes its version).
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "../../include/burgers.h"
#include "api_internal.h"
#include "kernels.h"

namespace burgers {

constexpr int TUNE_ROWS = 512;
constexpr int THOMAS_TUNE_ROWS = 65536;

struct Cand {
  int nt, c, k;
};

// Times `reps` runs of one shape over a packed copy of `rows` (row data in buf).
static burgers_status time_resident(burgers_ctx* ctx, const KernelEntry* k,
                                    const std::vector<RowDesc>& rows, void* buf, const void* orig,
                                    const std::vector<int64_t>& orig_off, size_t esz,
                                    cudaStream_t st, float* ms) {
  DevBuf& d = ctx->tunews;
  const size_t need = rows.size() * sizeof(RowDesc) + 256;
  cudaError_t e = d.ensure(need);
  if (e != cudaSuccess) return set_error(BURGERS_ENOMEM, "tune descriptors");
  char* base = static_cast<char*>(d.ptr);
  RowDesc* rd = reinterpret_cast<RowDesc*>(base + 256);
  int* ctr = reinterpret_cast<int*>(base);
  e = cudaMemcpyAsync(rd, rows.data(), rows.size() * sizeof(RowDesc), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_error(e, "tune upload");
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k->fn, k->nt, k->dyn_smem) != cudaSuccess ||
      occ < 1)
    occ = 1;
  int cnt = int(rows.size());
  int grid = std::min(cnt, ctx->sm_count * occ);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    for (size_t i = 0; i < rows.size(); ++i) {  // fresh copy of the rows
      e = cudaMemcpyAsync(static_cast<char*>(buf) + size_t(rows[i].offset) * esz,
                          static_cast<const char*>(orig) + size_t(orig_off[i]) * esz,
                          size_t(rows[i].n) * esz, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) break;
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(ctr, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    void* args[] = {&buf, &rd, &cnt, &ctr};
    if (e == cudaSuccess) e = cudaLaunchKernel(k->fn, dim3(grid), dim3(k->nt), args, k->dyn_smem, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) break;
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    if (rep > 0) best = std::min(best, t);  // first run warms up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_error(e, "tune run");
  ctx->launches += 3;
  *ms = best;
  return BURGERS_OK;
}

// Times the per-thread Thomas kernel k over the same rows (one CTA per k->nt
// rows, its workspace in the context's scratch buffer).
static burgers_status time_thomas(burgers_ctx* ctx, const KernelEntry* k,
                                  const std::vector<RowDesc>& rows, void* buf, const void* orig,
                                  const std::vector<int64_t>& orig_off, size_t esz, int dtype,
                                  cudaStream_t st, float* ms) {
  DevBuf& d = ctx->tunews;
  const size_t need = rows.size() * sizeof(RowDesc) + 256;
  cudaError_t e = d.ensure(need);
  if (e != cudaSuccess) return set_error(BURGERS_ENOMEM, "tune descriptors");
  RowDesc* rd = reinterpret_cast<RowDesc*>(static_cast<char*>(d.ptr) + 256);
  e = cudaMemcpyAsync(rd, rows.data(), rows.size() * sizeof(RowDesc), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_error(e, "tune upload");
  int cnt = int(rows.size());
  const int grid = (cnt + k->nt - 1) / k->nt;
  e = ctx->scratch.ensure(std::max<size_t>(1, size_t(grid) * thomas_ws_values(dtype, k->nt, k->c, k->exact) * esz));
  if (e != cudaSuccess) return set_error(BURGERS_ENOMEM, "tune workspace");
  void* ws = ctx->scratch.ptr;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    for (size_t i = 0; i < rows.size(); ++i) {  // fresh copy of the rows
      e = cudaMemcpyAsync(static_cast<char*>(buf) + size_t(rows[i].offset) * esz,
                          static_cast<const char*>(orig) + size_t(orig_off[i]) * esz,
                          size_t(rows[i].n) * esz, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) break;
    }
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    void* args[] = {&buf, &rd, &cnt, &ws};
    if (e == cudaSuccess) e = cudaLaunchKernel(k->fn, dim3(grid), dim3(k->nt), args, k->dyn_smem, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) break;
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    if (rep > 0) best = std::min(best, t);  // first run warms up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_error(e, "tune run");
  ctx->launches += 3;
  *ms = best;
  return BURGERS_OK;
}

burgers_status autotune(burgers_ctx* ctx, int scheme, const burgers_batch* batch,
                        const void* u_dev, int64_t probe_steps, cudaStream_t st,
                        int* tuned_out) {
  const int dtype = batch->dtype;
  const size_t esz = dtype == 0 ? 4 : 8;
  const int kind = resident_kind(scheme);
  const int64_t rlim = resident_capacity(ctx, kind, dtype);
  // capacity classes of the resident rows
  std::map<std::pair<int64_t, int>, std::vector<int64_t>> classes;
  std::vector<int64_t> longs;
  for (int64_t b = 0; b < batch->count; ++b) {
    const burgers_instance& in = batch->inst[b];
    if (in.nsteps == 0) continue;
    if (in.n > rlim) {
      longs.push_back(b);
      continue;
    }
    int64_t cap = resident_class(kind, dtype, in.n);
    if (cap > 0) classes[{cap, cap == in.n ? 1 : 0}].push_back(b);
  }
  int ntuned = 0;
  for (auto& kv : classes) {
    const int64_t cap = kv.first.first;
    const int exact = kv.first.second;
    std::vector<Cand> cands;
    for (const auto& sh : resident_shape_list(kind, dtype))
      if (int64_t(sh.first) * sh.second == cap && find_kernel(kind, dtype, sh.first, sh.second, exact))
        cands.push_back(Cand{sh.first, sh.second, 0});
    // BTCS: the per-thread Thomas kernels of this capacity (k = 1 + planes in
    // the workspace)
    if (scheme == BURGERS_BTCS && !ctx->plain)
      for (const KernelEntry& e : kernel_registry())
        if (e.kind == K_BTCS_THOMAS && e.dtype == dtype && e.c == cap)
          cands.push_back(Cand{e.nt, e.c, 1 + e.exact});
    if (cands.size() < 2) continue;
    std::vector<int64_t>& ids = kv.second;
    // the per-thread Thomas kernel's speed depends on how many rows fill the
    // GPU: classes where it competes are probed with up to THOMAS_TUNE_ROWS
    const bool thomas = std::any_of(cands.begin(), cands.end(), [](const Cand& c) { return c.k >= 1; });
    const size_t probe_rows = thomas ? size_t(THOMAS_TUNE_ROWS) : size_t(TUNE_ROWS);
    if (ids.size() > probe_rows) ids.resize(probe_rows);
    std::vector<RowDesc> rows;
    std::vector<int64_t> orig_off;
    int64_t off = 0;
    for (int64_t b : ids) {
      const burgers_instance& in = batch->inst[b];
      RowDesc d;
      d.offset = off;
      d.nsteps = std::min<int64_t>(in.nsteps, probe_steps);
      d.r = in.dt / in.dx;
      d.s = in.nu * in.dt / (in.dx * in.dx);
      d.ds_dnu = in.dt / (in.dx * in.dx);
      d.n = in.n;
      d.bc = in.bc;
      set_fp32_coefs(d);
      rows.push_back(d);
      orig_off.push_back(in.offset);
      off += in.n;
    }
    cudaError_t e = ctx->tunebuf.ensure(size_t(off) * esz);
    if (e != cudaSuccess) return set_error(BURGERS_ENOMEM, "tune buffer");
    float best = 1e30f;
    Cand pick = cands[0];
    for (const Cand& c : cands) {
      float ms = 0.f;
      burgers_status s2;
      if (c.k >= 1) {
        const KernelEntry* k = find_kernel(K_BTCS_THOMAS, dtype, c.nt, c.c, c.k - 1);
        s2 = time_thomas(ctx, k, rows, ctx->tunebuf.ptr, u_dev, orig_off, esz, dtype, st, &ms);
      } else {
        const KernelEntry* k = find_kernel(kind, dtype, c.nt, c.c, exact);
        s2 = time_resident(ctx, k, rows, ctx->tunebuf.ptr, u_dev, orig_off, esz, st, &ms);
      }
      if (s2 != BURGERS_OK) return s2;
      if (ms < best) {
        best = ms;
        pick = c;
      }
    }
    TuneVal tv;
    tv.nt = pick.nt;
    tv.c = pick.c;
    tv.k = pick.k;
    ctx->tuned[tune_key(kind, dtype, cap, exact)] = tv;
    ++ntuned;
  }
  if (scheme == BURGERS_EXPLICIT && !longs.empty()) {
    // streaming: try window shapes x K on the first long rows through the
    // normal advance path (plans are rebuilt per candidate)
    std::vector<burgers_instance> probe;
    int64_t nmin = INT64_MAX;
    for (int64_t b : longs) nmin = std::min<int64_t>(nmin, batch->inst[b].n);
    for (size_t i = 0; i < longs.size() && i < 4; ++i) probe.push_back(batch->inst[longs[i]]);
    int64_t off = 0, lo = INT64_MAX;
    for (auto& in : probe) lo = std::min<int64_t>(lo, in.offset);
    std::vector<int64_t> orig_off;
    for (auto& in : probe) {
      orig_off.push_back(in.offset);
      in.offset = off;
      off += in.n;
    }
    cudaError_t e = ctx->tunebuf.ensure(size_t(off) * esz);
    if (e != cudaSuccess) return set_error(BURGERS_ENOMEM, "tune buffer");
    const int shapes32[][2] = {{128, 16}, {256, 16}, {512, 16}, {256, 32}};
    const int shapes64[][2] = {{128, 8}, {256, 8}, {256, 16}};
    const int ns = dtype == 0 ? 4 : 3;
    const int Ks[] = {8, 16, 32, 48, 64, 96, 128};
    float best = 1e30f;
    TuneVal pick;
    const int saved_k = ctx->stream_k;
    const bool saved_graphs = ctx->graphs;
    ctx->graphs = false;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int si = 0; si < ns; ++si) {
      const int nt = dtype == 0 ? shapes32[si][0] : shapes64[si][0];
      const int c = dtype == 0 ? shapes32[si][1] : shapes64[si][1];
      if (int64_t(nt) * c > nmin) continue;
      for (int K : Ks) {
        if (4 * K > nt * c) continue;
        TuneVal tv;
        tv.nt = nt;
        tv.c = c;
        tv.k = K;
        ctx->tuned[tune_key(K_EXPLICIT_STREAM, dtype, 0, 0)] = tv;
        ctx->tune_version++;
        ctx->stream_k = 0;
        for (auto& in : probe) in.nsteps = std::max<int64_t>(4 * K, std::min<int64_t>(probe_steps, 256));
        burgers_batch pb = *batch;
        pb.count = int64_t(probe.size());
        pb.inst = probe.data();
        float t = 0.f;
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
          for (size_t i = 0; i < probe.size() && e == cudaSuccess; ++i)
            e = cudaMemcpyAsync(static_cast<char*>(ctx->tunebuf.ptr) + size_t(probe[i].offset) * esz,
                                static_cast<const char*>(u_dev) + size_t(orig_off[i]) * esz,
                                size_t(probe[i].n) * esz, cudaMemcpyDeviceToDevice, st);
          if (e != cudaSuccess) break;
          cudaEventRecord(e0, st);
          ctx->resident_override = 1;  // force the long rows through streaming
          burgers_status s2 = advance(ctx, BURGERS_EXPLICIT, &pb, ctx->tunebuf.ptr, st);
          ctx->resident_override = 0;
          if (s2 != BURGERS_OK) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            ctx->graphs = saved_graphs;
            ctx->stream_k = saved_k;
            return s2;
          }
          cudaEventRecord(e1, st);
          e = cudaEventSynchronize(e1);
          cudaEventElapsedTime(&t, e0, e1);
        }
        if (e != cudaSuccess) break;
        double cells = 0;
        for (auto& in : probe) cells += double(in.n) * double(in.nsteps);
        const float per = float(t / cells);
        if (per < best) {
          best = per;
          pick = tv;
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->graphs = saved_graphs;
    ctx->stream_k = saved_k;
    if (e != cudaSuccess) return cuda_error(e, "stream tune");
    if (pick.nt > 0) {
      ctx->tuned[tune_key(K_EXPLICIT_STREAM, dtype, 0, 0)] = pick;
      ++ntuned;
    } else {
      ctx->tuned.erase(tune_key(K_EXPLICIT_STREAM, dtype, 0, 0));
    }
    (void)lo;
  }
  ctx->tune_version++;
  if (tuned_out) *tuned_out = ntuned;
  return BURGERS_OK;
}

}  // namespace burgers

extern "C" {

burgers_status burgers_autotune(burgers_ctx* ctx, int32_t scheme, const burgers_batch* batch,
                                const void* u_dev, int64_t probe_steps, int32_t* tuned,
                                burgers_stream stream) {
  using namespace burgers;
  if (!ctx) return set_error(BURGERS_EINVAL, "ctx is NULL");
  if (!valid_scheme(scheme)) return set_error(BURGERS_EINVAL, "bad scheme");
  if (probe_steps < 1) return set_error(BURGERS_EINVAL, "probe_steps must be >= 1");
  burgers_status st = validate_batch(batch, false);
  if (st != BURGERS_OK) return st;
  if (batch->count == 0) return BURGERS_OK;
  if (!u_dev) return set_error(BURGERS_EINVAL, "u_dev is NULL");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_error(e, "cudaSetDevice");
  int n = 0;
  st = autotune(ctx, scheme, batch, u_dev, probe_steps, reinterpret_cast<cudaStream_t>(stream), &n);
  if (tuned) *tuned = n;
  return st;
}

burgers_status burgers_tune_save(const burgers_ctx* ctx, const char* path) {
  using namespace burgers;
  if (!ctx || !path) return set_error(BURGERS_EINVAL, "NULL argument");
  FILE* f = fopen(path, "w");
  if (!f) return set_error(BURGERS_EINVAL, std::string("cannot write ") + path);
  fprintf(f, "# libburgers tuning table: key nt c k\n");
  for (const auto& kv : ctx->tuned)
    fprintf(f, "%llu %d %d %d\n", (unsigned long long)kv.first, kv.second.nt, kv.second.c, kv.second.k);
  fclose(f);
  return BURGERS_OK;
}

burgers_status burgers_tune_load(burgers_ctx* ctx, const char* path) {
  using namespace burgers;
  if (!ctx || !path) return set_error(BURGERS_EINVAL, "NULL argument");
  FILE* f = fopen(path, "r");
  if (!f) return set_error(BURGERS_EINVAL, std::string("cannot read ") + path);
  char line[256];
  std::map<uint64_t, TuneVal> tab;
  while (fgets(line, sizeof line, f)) {
    if (line[0] == '#') continue;
    unsigned long long key = 0;
    TuneVal v;
    if (sscanf(line, "%llu %d %d %d", &key, &v.nt, &v.c, &v.k) != 4) {
      fclose(f);
      return set_error(BURGERS_EINVAL, "malformed tuning table");
    }
    const int kind = int(key >> 56), dtype = int((key >> 52) & 0xf), exact = int((key >> 48) & 0xf);
    const int exact_lookup = kind == K_EXPLICIT_STREAM ? 0 : exact;
    // a BTCS class entry with k >= 1 names a per-thread Thomas kernel
    const bool thomas = kind == K_BTCS_RESIDENT && v.k >= 1;
    const bool known = thomas ? find_kernel(K_BTCS_THOMAS, dtype, v.nt, v.c, v.k - 1) != nullptr
                              : find_kernel(kind, dtype, v.nt, v.c, exact_lookup) != nullptr;
    // k: steps per pass of a streaming entry (up to 128), else a kernel index
    const int kmax = (kind == K_EXPLICIT_STREAM || kind == K_RK4_STREAM) ? 128 : 64;
    if (!known || v.k < 0 || v.k > kmax) {
      fclose(f);
      return set_error(BURGERS_EINVAL, "tuning table names a kernel shape that does not exist");
    }
    tab[key] = v;
  }
  fclose(f);
  for (auto& kv : tab) ctx->tuned[kv.first] = kv.second;
  ctx->tune_version++;
  return BURGERS_OK;
}

}  // extern "C"
