// api_internal.h -- host-side state of libburgers shared by its translation
// units (context, plans, workspaces).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <list>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/burgers.h"
#include "kernels.h"

namespace burgers {

burgers_status set_error(burgers_status st, const std::string& msg);
burgers_status cuda_error(cudaError_t e, const char* where);
burgers_status validate_batch(const burgers_batch* batch, bool allow_empty);

// Growable device allocation; `generation` changes whenever the pointer does.
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  uint64_t generation = 0;
  cudaError_t ensure(size_t need);
  ~DevBuf();
};

// Growable pinned host allocation.
struct HostBuf {
  void* hptr = nullptr;
  size_t bytes = 0;
  cudaError_t ensure_host(size_t need);
  ~HostBuf();
};

enum LaunchType : int { LAUNCH_RESIDENT = 0, LAUNCH_STREAM = 1, LAUNCH_ML = 2, LAUNCH_THOMAS = 3 };

struct Launch {
  const KernelEntry* k = nullptr;
  int type = LAUNCH_RESIDENT;
  int grid = 1;
  int row_begin = 0, row_count = 0;
  int counter = -1;
  int item_begin = 0, item_count = 0;
  int K = 0;
  int nbulk = -1;  // bulk-copy single-step launch: items [0, nbulk) are whole aligned tiles
  int64_t ws_off = 0, ws_elems = 0;  // per-thread Thomas launch: its workspace in the scratch
  const KernelEntry* k_fallback = nullptr;  // its per-tile kernel (unaligned buffers)
  int64_t step_base = 0;
  bool to_scratch = false;
  int level = 0;   // multi-level: level of a reduce/recover launch
  int ml_phase = 0;
  int iter = 0;    // multi-level: iteration of the step (Picard, Newton)
};

struct Plan {
  uint64_t key = 0;
  int64_t count = 0;
  int dtype = 0, scheme = 0;
  std::vector<RowDesc> rows;
  std::vector<int32_t> row_inst;        // batch instance of each entry of rows
  std::vector<TileItem> items;
  std::vector<unsigned char> ml_bytes;  // multi-level row descriptors
  int ml_rows = 0;
  std::vector<Launch> launches;
  int ncounters = 0;
  int64_t kernel_launches = 0;
  int64_t scratch_elems = 0;  // streaming ping-pong (+ compensation) buffers, elements
  int64_t stream_span = 0;    // elements covered by the streaming rows
  int64_t ml_span = 0;        // elements covered by the multi-level rows
  int64_t ml_ws_elems = 0;    // multi-level workspace, elements
  int64_t ml_e_off = 0;       // multi-level: scratch offset of the two e planes, elements
  void* dev = nullptr;
  bool dev_external = false;
  size_t rows_off = 0, items_off = 0, counters_off = 0, ml_off = 0, dev_bytes = 0;
  void* dtdev = nullptr;  // device-dt plans: row_inst and (dx, nu) per instance
  cudaGraphExec_t gexec = nullptr;
  void* g_u = nullptr;
  uint64_t g_scratch_gen = 0, g_ml_gen = 0;
  ~Plan();
};

// Device-resident descriptors of the CFL reduction of one batch layout
// (burgers_cfl_dt_device).
struct RedCache {
  void* dev = nullptr;
  size_t off[6] = {0, 0, 0, 0, 0, 0};
  int nrows = 0, nitems = 0;
};

// Descriptor buffers owned by a caller of advance_uncached().
struct PlanScratch {
  DevBuf dev;
  HostBuf host;
};

struct TuneVal {
  int nt = 0, c = 0, k = 0;
};

inline uint64_t tune_key(int kind, int dtype, int64_t cap, int exact) {
  return (uint64_t(kind) << 56) ^ (uint64_t(dtype) << 52) ^ (uint64_t(exact) << 48) ^ uint64_t(cap);
}

}  // namespace burgers

struct burgers_ctx {
  int device = 0;
  int sm_count = 1;
  size_t smem_optin = 0;
  bool graphs = true;
  bool plain = false;
  int cluster = 1;      // cluster-resident BTCS: 0 off, 1 any size the device fits, 2 portable (<= 8)
  int cluster_cs128 = 8;  // largest schedulable cluster of 128-thread BTCS CTAs (8..16)
  bool autotune = false;
  int stream_k = 0;
  int64_t resident_max = 0;
  int tune_version = 0;
  std::atomic<int64_t> launches{0};
  cudaStream_t capture_stream = nullptr;
  // independent resident launches of one plan overlap on these side streams
  static constexpr int kSide = 3;
  cudaStream_t side[kSide] = {};
  cudaEvent_t fork_ev = nullptr, join_ev[kSide] = {};
  // host-memory solves: copy streams and per-chunk events of the pipeline
  static constexpr int kIoChunks = 8;
  cudaStream_t io_h2d = nullptr, io_d2h = nullptr;
  cudaEvent_t io_in[kIoChunks] = {}, io_out[kIoChunks] = {};
  std::list<std::unique_ptr<burgers::Plan>> plans;
  std::map<uint64_t, burgers::TuneVal> tuned;
  burgers::DevBuf scratch;  // streaming ping-pong
  burgers::DevBuf mlws;     // multi-level reduced systems
  burgers::DevBuf redws;    // reductions
  burgers::DevBuf iobuf;    // burgers_solve_host
  burgers::DevBuf tunews;   // autotuner descriptors
  burgers::DevBuf tunebuf;  // autotuner row copies
  int resident_override = 0;  // autotuner: send every long-enough row to the long-row path
  burgers::HostBuf redhost;
  burgers::DevBuf errbuf;   // device error word of the bounded waits (bit 0: a bulk-copy wait gave up)
  burgers::DevBuf adjws;    // adjoint checkpoints and segment states
  burgers::DevBuf adjdesc;  // adjoint descriptors
  burgers::HostBuf adjhost;
  cudaEvent_t adj_event = nullptr;
  burgers::DevBuf adjlong;   // long-row explicit adjoint: states, checkpoints, lambda
  burgers::DevBuf adjldesc;  // its descriptors
  burgers::HostBuf adjlhost;
  cudaEvent_t adjl_event = nullptr;
  size_t red_offsets[6] = {0, 0, 0, 0, 0, 0};
  std::map<uint64_t, burgers::RedCache> redcache;  // burgers_cfl_dt_device
  burgers_ctx();
  ~burgers_ctx();
};

namespace burgers {
// nu = A(u)^{-T} (lam - A(u)^T lam) for every row of `batch` (its nsteps must
// be 1), u the state in the batch layout, lam and nu device buffers of the
// same layout covering the rows; through the multi-level solver.
burgers_status transposed_btcs_solve(burgers_ctx* ctx, const burgers_batch* batch, const void* u,
                                     const void* lam, void* nu, cudaStream_t st);
// Long-row adjoint (adjoint_long.cu): the rows `longs` of the batch.
burgers_status adjoint_long_run(burgers_ctx* ctx, int scheme, const burgers_batch* batch,
                                const std::vector<int64_t>& longs, const void* u0, const void* gT,
                                void* gu0, double* gnu, int64_t stride, cudaStream_t st);
// var: 0 lagged BTCS, 1 Crank-Nicolson, 2 Picard, 3 Newton; iters: iterations
// per step of the last two.
burgers_status plan_multilevel(burgers_ctx* ctx, const burgers_batch* batch,
                               const std::vector<int64_t>& longs, Plan* p, int var, int iters);
cudaError_t enqueue_multilevel_launch(burgers_ctx* ctx, Plan* p, const Launch& L, void* u,
                                      cudaStream_t st);
// Resident kernel kind of a scheme (burgers_scheme).
inline int resident_kind(int scheme) {
  switch (scheme) {
    case BURGERS_EXPLICIT: return K_EXPLICIT_RESIDENT;
    case BURGERS_RK4: return K_RK4_RESIDENT;
    case BURGERS_CN: return K_CN_RESIDENT;
    case BURGERS_PICARD: return K_PICARD_RESIDENT;
    case BURGERS_NEWTON: return K_NEWTON_RESIDENT;
    default: return K_BTCS_RESIDENT;
  }
}
inline bool valid_scheme(int scheme) { return scheme >= BURGERS_EXPLICIT && scheme <= BURGERS_NEWTON; }
// Internal scheme of the long-row BTCS adjoint: one solve with A(u)^T per row
// through the multi-level solver (never valid on the public entry points).
constexpr int SCHEME_BTCS_T = 100;
// Every scheme has a path for long rows: streaming windows (explicit Euler,
// RK4) or the multi-level solver (BTCS and the implicit variants).
inline bool has_long_path(int scheme) { return valid_scheme(scheme) || scheme == SCHEME_BTCS_T; }

burgers_status advance(burgers_ctx* ctx, int scheme, const burgers_batch* batch, void* u_dev,
                       cudaStream_t stream, int iters = 1);
burgers_status advance_uncached(burgers_ctx* ctx, int scheme, const burgers_batch* batch,
                                void* u_dev, cudaStream_t stream, PlanScratch* ps);
burgers_status advance_uncached_pair(burgers_ctx* ctx, int scheme_a, const burgers_batch* a,
                                     PlanScratch* ps_a, int scheme_b, const burgers_batch* b,
                                     PlanScratch* ps_b, void* u_dev, cudaStream_t stream_a,
                                     cudaStream_t stream_b, cudaEvent_t fork, cudaEvent_t join);
int64_t adjoint_max_n(int dtype);
// Workspace values of one CTA of the per-thread Thomas kernel (btcs_thomas.cu).
size_t thomas_ws_values(int dtype, int nt, int nmax, int mode);
// The per-thread Thomas kernel a BTCS row of n nodes takes, or nullptr for the
// partitioned resident kernel (tuning table first, then the default classes;
// class_rows: rows of the row's capacity class in the call).
const KernelEntry* pick_thomas(const burgers_ctx* ctx, int dtype, int64_t n, int64_t class_rows);
int64_t resident_capacity(const burgers_ctx* ctx, int kind, int dtype);
int64_t resident_class(int kind, int dtype, int64_t n);
std::vector<std::pair<int, int>> resident_shape_list(int kind, int dtype);
burgers_status autotune(burgers_ctx* ctx, int scheme, const burgers_batch* batch,
                        const void* u_dev, int64_t probe_steps, cudaStream_t st, int* tuned_out);
burgers_status adjoint_run(burgers_ctx* ctx, int scheme, const burgers_batch* batch,
                           const void* u0, const void* gT, void* gu0, double* gnu,
                           int64_t stride, cudaStream_t st);
}  // namespace burgers
