// serve.cu -- continuous-batching server for mixed Burgers requests.
//
// Requests (scheme, BC, n, dx, nu, dt, nsteps, u0) arrive from any thread and
// wait in a FIFO. A worker thread owns one CUDA stream and a device memory
// pool sized by the HBM budget; it repeats:
//   1. admission: pending requests whose state fits the pool (a first-fit free
//      list; long rows use their own region so the long-row scratch buffers
//      stay bounded) become active, and their u0 is copied into their slot;
//   2. slice: every active request advances min(S, remaining) steps, the
//      explicit ones in one batched call and the BTCS ones in another, all
//      through the same kernels as burgers_*_advance (the pool is the packed
//      buffer, slot offsets are the row offsets);
//   3. completion: finished requests are copied back to host memory and their
//      slots return to the free list, which is what lets the next arrivals in.
// Which requests a slice finishes follows from the step counts, so the worker
// plans and enqueues the next slice (with its admission and result copies)
// while the current one runs: two slices in flight at most, and the GPU is not
// idle during a slice boundary's host work. Requests that arrive while a slice
// runs join at the next slice boundary.
// Slices start at fixed multiples of S steps of each request, so a request's
// result does not depend on what else is in the mix (same kernel shape, same
// slice boundaries): the result alone and in the mix is bitwise the same.
//
// Every wait is bounded: the worker polls its event with a deadline and
// records BURGERS_ETIMEOUT on the affected requests instead of hanging, and
// burgers_serve_wait takes a timeout.
#include <string.h>
#include <time.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/burgers.h"
#include "api_internal.h"

namespace burgers {

// Slices whose device-time stamps are kept at once (two in flight plus the
// previous end of each).
constexpr int kSliceRing = 4;

static double now_s() {
  struct timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return double(ts.tv_sec) + 1e-9 * double(ts.tv_nsec);
}

// First-fit allocator over [base, base + size) with coalescing.
class Region {
 public:
  void init(int64_t base, int64_t size) {
    free_.clear();
    if (size > 0) free_[base] = size;
    total_ = size;
    used_ = 0;
  }
  bool alloc(int64_t bytes, int64_t* off) {
    bytes = (bytes + 255) & ~int64_t(255);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const int64_t rest = it->second - bytes;
        const int64_t start = it->first + bytes;
        free_.erase(it);
        if (rest > 0) free_[start] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(int64_t off, int64_t bytes) {
    bytes = (bytes + 255) & ~int64_t(255);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  int64_t total() const { return total_; }
  int64_t used() const { return used_; }

 private:
  std::map<int64_t, int64_t> free_;
  int64_t total_ = 0, used_ = 0;
};

// Page-locked host buffers for request states, carved out of 64 MiB slabs
// (grown on demand up to a cap): u0 is copied into one at submit, the device
// copies read and write it asynchronously at full DMA rate, and the result
// lands in the same buffer. Past the cap requests fall back to pageable
// vectors. Not thread-safe: the server's mutex guards every call.
class PinnedArena {
 public:
  static constexpr int64_t kSlab = int64_t(64) << 20;
  static constexpr int64_t kCap = int64_t(8) << 30;
  unsigned char* alloc(int64_t bytes) {
    // first fit, starting at the slab that served the last request (requests
    // come and go roughly in order, so the slabs before it are mostly full)
    const size_t ns = slabs_.size();
    for (size_t k = 0; k < ns; ++k) {
      const size_t i = (hint_ + k) % ns;
      int64_t off;
      if (slabs_[i].rg.alloc(bytes, &off)) {
        hint_ = i;
        return slabs_[i].base + off;
      }
    }
    const int64_t size = std::max<int64_t>(kSlab, (bytes + 255) & ~int64_t(255));
    if (total_ + size > kCap) return nullptr;
    void* p = nullptr;
    if (cudaHostAlloc(&p, size_t(size), cudaHostAllocMapped) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    // the copy kernels reach the slab through its device alias; without one
    // its requests fall back to cudaMemcpyAsync
    void* dp = nullptr;
    if (cudaHostGetDevicePointer(&dp, p, 0) != cudaSuccess) {
      cudaGetLastError();
      dp = nullptr;
    }
    total_ += size;
    slabs_.push_back(Slab{static_cast<unsigned char*>(p), static_cast<unsigned char*>(dp), size,
                          Region()});
    Slab& sl = slabs_.back();
    sl.rg.init(0, size);
    int64_t off = 0;
    sl.rg.alloc(bytes, &off);
    hint_ = slabs_.size() - 1;
    return sl.base + off;
  }
  void reserve(int slabs) {
    std::vector<unsigned char*> held;
    for (int i = 0; i < slabs; ++i) {
      unsigned char* p = alloc(kSlab);
      if (!p) break;
      held.push_back(p);
    }
    for (unsigned char* p : held) release(p, kSlab);
  }
  void release(unsigned char* p, int64_t bytes) {
    for (Slab& sl : slabs_)
      if (p >= sl.base && p < sl.base + sl.size) {
        sl.rg.release(p - sl.base, bytes);
        return;
      }
  }
  // Device alias of the page-locked bytes [p, p + bytes), or nullptr.
  void* device_alias(unsigned char* p, int64_t bytes) const {
    for (const Slab& sl : slabs_)
      if (p >= sl.base && p + bytes <= sl.base + sl.size)
        return sl.dev ? static_cast<void*>(sl.dev + (p - sl.base)) : nullptr;
    return nullptr;
  }
  ~PinnedArena() {
    for (Slab& sl : slabs_) cudaFreeHost(sl.base);
  }

 private:
  struct Slab {
    unsigned char* base;
    unsigned char* dev;  // device alias of the mapped slab
    int64_t size;
    Region rg;
  };
  std::vector<Slab> slabs_;
  size_t hint_ = 0;
  int64_t total_ = 0;
};

// One request's transfer between its page-locked buffer (through the device
// alias) and its slot in the pool. Both ends 16-byte aligned, bytes a
// multiple of 4 (FP32 / FP64 rows).
struct CopyDesc {
  const void* src;
  void* dst;
  int64_t bytes;
};

// All admission (or all result) transfers of a slice in one launch instead
// of one cudaMemcpyAsync per request, whose host-side cost dominated the
// worker's slice boundary: CTA i moves requests i, i + grid, ... with
// 16-byte accesses (the tail in 4-byte words).
__global__ void __launch_bounds__(256) k_serve_copy(const CopyDesc* __restrict__ d, int count) {
  for (int i = blockIdx.x; i < count; i += gridDim.x) {
    const CopyDesc c = d[i];
    const int64_t nv = c.bytes >> 4;
    const uint4* src = static_cast<const uint4*>(c.src);
    uint4* dst = static_cast<uint4*>(c.dst);
    for (int64_t k = threadIdx.x; k < nv; k += blockDim.x) dst[k] = src[k];
    const int tail = int((c.bytes - (nv << 4)) >> 2);
    if (int(threadIdx.x) < tail) {
      const uint32_t* s4 = reinterpret_cast<const uint32_t*>(static_cast<const char*>(c.src) + (nv << 4));
      uint32_t* d4 = reinterpret_cast<uint32_t*>(static_cast<char*>(c.dst) + (nv << 4));
      d4[threadIdx.x] = s4[threadIdx.x];
    }
  }
}

// Page-locked, mapped descriptor list of one direction of one slice (the
// kernel reads it through its device alias). Rewritten only after the slice
// that last read it has retired.
class CopyStage {
 public:
  bool push(const void* src, void* dst, int64_t bytes) {
    if (n_ == cap_ && !grow()) return false;
    host_[n_++] = CopyDesc{src, dst, bytes};
    return true;
  }
  void clear() { n_ = 0; }
  int size() const { return n_; }
  const CopyDesc* device() const { return dev_; }
  ~CopyStage() {
    if (host_) cudaFreeHost(host_);
  }

 private:
  bool grow() {
    const int cap = cap_ ? 2 * cap_ : 1024;
    void* p = nullptr;
    if (cudaHostAlloc(&p, sizeof(CopyDesc) * size_t(cap), cudaHostAllocMapped) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    void* dp = nullptr;
    if (cudaHostGetDevicePointer(&dp, p, 0) != cudaSuccess) {
      cudaGetLastError();
      cudaFreeHost(p);
      return false;
    }
    if (n_) memcpy(p, host_, sizeof(CopyDesc) * size_t(n_));
    // the old list is not in use: this stage's previous slice has retired
    if (host_) cudaFreeHost(host_);
    host_ = static_cast<CopyDesc*>(p);
    dev_ = static_cast<CopyDesc*>(dp);
    cap_ = cap;
    return true;
  }
  CopyDesc* host_ = nullptr;
  CopyDesc* dev_ = nullptr;
  int n_ = 0, cap_ = 0;
};

enum ReqState : int { RQ_PENDING = 0, RQ_ACTIVE = 1, RQ_DONE = 2, RQ_CANCELED = 3, RQ_FAILED = 4 };

struct Req {
  uint64_t ticket = 0;
  burgers_request r{};
  std::vector<unsigned char> u0;   // pageable fallback of pin
  std::vector<unsigned char> out;  // pageable fallback of pin
  unsigned char* pin = nullptr;    // page-locked state: u0, later the result
  void* pin_dev = nullptr;         // its device alias (nullptr: copied by cudaMemcpyAsync)
  int state = RQ_PENDING;
  burgers_status status = BURGERS_OK;
  bool long_row = false;
  bool cancel = false;
  int64_t off = 0, bytes = 0, done_steps = 0, slices = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
};

}  // namespace burgers

struct burgers_server {
  burgers_ctx* ctx = nullptr;
  burgers_serve_cfg cfg{};
  size_t esz = 4;
  void* pool = nullptr;
  int64_t pool_bytes = 0;
  burgers::Region short_region, long_region;
  cudaStream_t stream = nullptr, stream_b = nullptr;  // BTCS slices run on stream_b
  cudaEvent_t ev[2] = {nullptr, nullptr};  // end of the slices in flight (by parity)
  // device-time stamps of the start and end of each slice, a ring of four
  // slices (two in flight, and the previous end of each kept for the gap)
  cudaEvent_t tev[2 * burgers::kSliceRing] = {};
  int64_t slices_enqueued = 0;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<burgers::Req*> pending;
  std::vector<burgers::Req*> active;
  std::unordered_map<uint64_t, std::unique_ptr<burgers::Req>> reqs;
  std::deque<uint64_t> done_q;  // finished tickets not yet reported by wait_any
  uint64_t next_ticket = 1;
  bool stop = false;
  burgers_status fault = BURGERS_OK;
  std::string fault_msg;
  burgers::PlanScratch ps_explicit[2], ps_btcs[2];  // descriptors of the slices in flight
  burgers::CopyStage stage_in[2], stage_out[2];     // their admission / result transfers
  std::mutex pin_mu;  // guards `pinned` (taken alone, or after mu)
  burgers::PinnedArena pinned;
  burgers_serve_stats stats{};
  double t0 = 0;
};

namespace burgers {

static int64_t long_limit(burgers_server* sv, int scheme) {
  const int kind = scheme == BURGERS_EXPLICIT ? K_EXPLICIT_RESIDENT : K_BTCS_RESIDENT;
  return resident_capacity(sv->ctx, kind, sv->cfg.dtype);
}

// Admits pending requests in arrival order while their state fits the pool
// (a request that does not fit blocks the ones behind it: no overtaking).
static void admit(burgers_server* sv, std::vector<Req*>* admitted) {
  while (!sv->pending.empty()) {
    Req* q = sv->pending.front();
    if (q->cancel) {
      sv->pending.pop_front();
      q->state = RQ_CANCELED;
      q->status = BURGERS_ECANCELED;
      q->t_done = now_s() - sv->t0;
      sv->done_q.push_back(q->ticket);
      sv->cv_done.notify_all();
      continue;
    }
    if (sv->cfg.max_active > 0 && int64_t(sv->active.size()) >= sv->cfg.max_active) break;
    Region& rg = q->long_row ? sv->long_region : sv->short_region;
    int64_t off = 0;
    if (!rg.alloc(q->bytes, &off)) break;
    q->off = off;
    q->state = RQ_ACTIVE;
    q->t_admit = now_s() - sv->t0;
    sv->pending.pop_front();
    sv->active.push_back(q);
    admitted->push_back(q);
  }
}

static void fail_all(burgers_server* sv, burgers_status st, const std::string& msg) {
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->fault = st;
  sv->fault_msg = msg;
  for (Req* q : sv->active) {
    q->state = RQ_FAILED;
    q->status = st;
    sv->done_q.push_back(q->ticket);
  }
  for (Req* q : sv->pending) {
    q->state = RQ_FAILED;
    q->status = st;
    sv->done_q.push_back(q->ticket);
  }
  sv->active.clear();
  sv->pending.clear();
  sv->cv_done.notify_all();
}

// Waits for one of the worker's events with a deadline (never spins unbounded).
static burgers_status wait_event(burgers_server* sv, cudaEvent_t ev, double timeout_s) {
  const double end = now_s() + timeout_s;
  for (;;) {
    cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return BURGERS_OK;
    if (e != cudaErrorNotReady) return cuda_error(e, "serve slice");
    if (now_s() > end) return set_error(BURGERS_ETIMEOUT, "serve slice exceeded its deadline");
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

// A slice in flight: its event (recorded after the slice and the result
// copies of the requests it finishes) and those requests.
struct InFlight {
  bool on = false;
  int64_t no = 0;  // slice number (its timing events: slot no % kSliceRing)
  std::vector<Req*> finished;
};

// Device time of slice f (its first to its last stamp on the worker's stream)
// and the idle time before it (from the previous slice's last stamp), added
// to the statistics; both stamps have completed once the slice has.
static void account_slice(burgers_server* sv, const InFlight& f) {
  const int i = int(f.no % kSliceRing);
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, sv->tev[2 * i], sv->tev[2 * i + 1]) == cudaSuccess)
    sv->stats.t_gpu_s += 1e-3 * ms;
  else
    (void)cudaGetLastError();
  if (f.no > 0) {
    const int j = int((f.no - 1) % kSliceRing);
    if (cudaEventElapsedTime(&ms, sv->tev[2 * j + 1], sv->tev[2 * i]) == cudaSuccess)
      sv->stats.t_gpu_gap_s += 1e-3 * std::max(0.f, ms);
    else
      (void)cudaGetLastError();
  }
}

// Waits for a slice in flight and reports the requests it finished.
static burgers_status retire(burgers_server* sv, InFlight& f, int idx) {
  const double tw = now_s();
  burgers_status st = wait_event(sv, sv->ev[idx], sv->cfg.slice_timeout_s);
  if (st != BURGERS_OK) return st;
  std::lock_guard<std::mutex> lk(sv->mu);
  const double t = now_s() - sv->t0;
  sv->stats.t_slice_s += now_s() - tw;
  account_slice(sv, f);
  for (Req* q : f.finished) {
    q->state = RQ_DONE;
    q->t_done = t;
    sv->done_q.push_back(q->ticket);
    sv->stats.completed += 1;
    sv->stats.cell_updates += double(q->r.n) * double(q->r.nsteps);
    std::vector<unsigned char>().swap(q->u0);
  }
  if (!f.finished.empty()) sv->cv_done.notify_all();
  f.finished.clear();
  f.on = false;
  return BURGERS_OK;
}

// Fails every request, including those of the slices in flight.
static void fail_worker(burgers_server* sv, InFlight* fl, burgers_status st, const std::string& msg) {
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    for (int k = 0; k < 2; ++k) {
      for (Req* q : fl[k].finished) {
        q->state = RQ_FAILED;
        q->status = st;
        sv->done_q.push_back(q->ticket);
      }
      fl[k].finished.clear();
      fl[k].on = false;
    }
  }
  fail_all(sv, st, msg);
}

static bool aligned16(const void* a, const void* b) {
  return ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15) == 0;
}

// Moves the transfers listed in `st` on the worker's stream.
static cudaError_t launch_copies(burgers_server* sv, const CopyStage& st) {
  if (st.size() == 0) return cudaSuccess;
  const int grid = std::min(st.size(), 4 * sv->ctx->sm_count);
  k_serve_copy<<<grid, 256, 0, sv->stream>>>(st.device(), st.size());
  sv->ctx->launches += 1;
  return cudaGetLastError();
}

// The worker. Which requests a slice finishes follows from the step counts,
// so the next slice is planned, its admission copies queued and it is
// enqueued while the current one runs (two slices in flight at most, each
// with its own descriptor buffers and event): the GPU is not left idle while
// the host does a slice boundary's bookkeeping. Everything of a slice is
// ordered on the worker's stream (the BTCS half forks to stream_b and joins
// back), so a slot released by a finished request can take an admitted one
// at once: its upload is queued after the result copy that frees it.
static void worker_loop(burgers_server* sv) {
  cudaSetDevice(sv->ctx->device);
  const int64_t S = sv->cfg.slice_steps;
  std::vector<burgers_instance> ie, ib;
  std::vector<Req*> admitted, finished;
  InFlight fl[2];
  int par = 0;  // parity of the next slice
  for (;;) {
    admitted.clear();
    bool work = false;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      for (;;) {
        if (sv->stop) return;
        // drop cancelled active requests at the slice boundary
        for (size_t i = 0; i < sv->active.size();) {
          Req* q = sv->active[i];
          if (q->cancel) {
            (q->long_row ? sv->long_region : sv->short_region).release(q->off, q->bytes);
            q->state = RQ_CANCELED;
            q->status = BURGERS_ECANCELED;
            q->t_done = now_s() - sv->t0;
            sv->done_q.push_back(q->ticket);
            sv->active[i] = sv->active.back();
            sv->active.pop_back();
            sv->cv_done.notify_all();
          } else {
            ++i;
          }
        }
        admit(sv, &admitted);
        if (!sv->active.empty()) {
          work = true;
          break;
        }
        if (fl[0].on || fl[1].on) break;  // nothing new: finish what is in flight
        sv->cv_work.wait_for(lk, std::chrono::milliseconds(2));
      }
    }
    if (!work) {  // retire the slices in flight, oldest first
      for (int k = 0; k < 2; ++k) {
        const int idx = (par + k) & 1;
        if (!fl[idx].on) continue;
        burgers_status st = retire(sv, fl[idx], idx);
        if (st != BURGERS_OK) {
          fail_worker(sv, fl, st, burgers_last_error());
          return;
        }
      }
      continue;
    }
    // ---- copy the new requests' u0 into their slots (one kernel for those
    // in mapped page-locked buffers, a copy each for the rest)
    double tw0 = now_s();
    const int64_t sno = sv->slices_enqueued;
    const int ring = int(sno % kSliceRing);
    cudaError_t e = cudaEventRecord(sv->tev[2 * ring], sv->stream);
    CopyStage& sin = sv->stage_in[par];
    sin.clear();
    for (Req* q : admitted) {
      char* slot = static_cast<char*>(sv->pool) + q->off;
      const void* src = q->pin_dev;
      if (src && aligned16(src, slot) && sin.push(src, slot, q->bytes)) continue;
      e = cudaMemcpyAsync(slot, q->pin ? static_cast<const void*>(q->pin) : q->u0.data(),
                          size_t(q->bytes), cudaMemcpyHostToDevice, sv->stream);
      if (e != cudaSuccess) break;
    }
    if (e == cudaSuccess) e = launch_copies(sv, sin);
    if (e != cudaSuccess) {
      fail_worker(sv, fl, cuda_error(e, "serve admission copy"), burgers_last_error());
      return;
    }
    double tw1 = now_s();
    // ---- one slice over every active request
    ie.clear(); ib.clear(); finished.clear();
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      for (Req* q : sv->active) {
        burgers_instance in;
        in.offset = q->off / int64_t(sv->esz);
        in.n = q->r.n;
        in.bc = q->r.bc;
        in.dx = q->r.dx;
        in.nu = q->r.nu;
        in.dt = q->r.dt;
        in.nsteps = std::min<int64_t>(S, q->r.nsteps - q->done_steps);
        if (q->r.scheme == BURGERS_EXPLICIT) ie.push_back(in);
        else ib.push_back(in);
      }
    }
    burgers_batch be{sv->cfg.dtype, 0, int64_t(ie.size()), ie.data()};
    burgers_batch bb{sv->cfg.dtype, 0, int64_t(ib.size()), ib.data()};
    burgers_status st =
        advance_uncached_pair(sv->ctx, BURGERS_EXPLICIT, &be, &sv->ps_explicit[par], BURGERS_BTCS,
                              &bb, &sv->ps_btcs[par], sv->pool, sv->stream, sv->stream_b,
                              sv->ev_fork, sv->ev_join);
    double tw2 = now_s();
    if (st != BURGERS_OK) {
      fail_worker(sv, fl, st, burgers_last_error());
      return;
    }
    // ---- the requests this slice finishes: result copies queued after it
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      for (Req* q : sv->active) {
        q->done_steps += std::min<int64_t>(S, q->r.nsteps - q->done_steps);
        q->slices += 1;
        if (q->done_steps >= q->r.nsteps) finished.push_back(q);
      }
    }
    CopyStage& sout = sv->stage_out[par];
    sout.clear();
    for (Req* q : finished) {
      const char* slot = static_cast<const char*>(sv->pool) + q->off;
      void* alias = q->pin_dev;
      if (alias && aligned16(alias, slot) && sout.push(slot, alias, q->bytes)) continue;
      void* dst = q->pin;
      if (!dst) {
        q->out.resize(size_t(q->bytes));
        dst = q->out.data();
      }
      e = cudaMemcpyAsync(dst, slot, size_t(q->bytes), cudaMemcpyDeviceToHost, sv->stream);
      if (e != cudaSuccess) break;
    }
    if (e == cudaSuccess) e = launch_copies(sv, sout);
    if (e == cudaSuccess) e = cudaEventRecord(sv->tev[2 * ring + 1], sv->stream);
    if (e == cudaSuccess) e = cudaEventRecord(sv->ev[par], sv->stream);
    if (e != cudaSuccess) {
      fail_worker(sv, fl, cuda_error(e, "serve result copy"), burgers_last_error());
      return;
    }
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      for (Req* q : finished)
        (q->long_row ? sv->long_region : sv->short_region).release(q->off, q->bytes);
      if (!finished.empty()) {
        auto& act = sv->active;
        act.erase(std::remove_if(act.begin(), act.end(),
                                 [](Req* q) { return q->done_steps >= q->r.nsteps; }),
                  act.end());
      }
      sv->stats.slices += 1;
      sv->stats.t_copy_s += (tw1 - tw0) + (now_s() - tw2);
      sv->stats.t_enqueue_s += tw2 - tw1;
      sv->stats.active_max = std::max<int64_t>(sv->stats.active_max,
                                               int64_t(sv->active.size() + finished.size()));
      sv->stats.pool_used_max = std::max<int64_t>(
          sv->stats.pool_used_max, sv->short_region.used() + sv->long_region.used());
    }
    fl[par].on = true;
    fl[par].no = sno;
    sv->slices_enqueued = sno + 1;
    fl[par].finished.swap(finished);
    // keep at most two slices in flight: wait for the previous one
    if (fl[par ^ 1].on) {
      st = retire(sv, fl[par ^ 1], par ^ 1);
      if (st != BURGERS_OK) {
        fail_worker(sv, fl, st, burgers_last_error());
        return;
      }
    }
    par ^= 1;
  }
}

}  // namespace burgers

using namespace burgers;

extern "C" {

burgers_status burgers_serve_create(burgers_ctx* ctx, const burgers_serve_cfg* cfg,
                                    burgers_server** out) {
  if (!ctx || !out) return set_error(BURGERS_EINVAL, "NULL argument");
  *out = nullptr;
  burgers_serve_cfg c{};
  if (cfg) c = *cfg;
  if (c.dtype != BURGERS_F32 && c.dtype != BURGERS_F64) return set_error(BURGERS_EINVAL, "bad dtype");
  if (c.slice_steps <= 0) c.slice_steps = 256;
  if (c.slice_timeout_s <= 0) c.slice_timeout_s = 60.0;
  if (c.max_active < 0 || c.hbm_budget < 0) return set_error(BURGERS_EINVAL, "negative limit");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_error(e, "cudaSetDevice");
  if (c.hbm_budget == 0) {
    size_t fr = 0, tot = 0;
    e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemGetInfo");
    c.hbm_budget = int64_t(fr / 2);
  }
  auto sv = std::make_unique<burgers_server>();
  sv->ctx = ctx;
  sv->cfg = c;
  sv->esz = c.dtype == BURGERS_F32 ? 4 : 8;
  // budget: pool (short + long regions) plus the long-row scratch and
  // multi-level workspace the kernels need for the long region
  const int64_t pool = (c.hbm_budget / 2) & ~int64_t(255);
  const int64_t long_bytes = (pool / 4) & ~int64_t(255);
  if (pool < (int64_t(1) << 20)) return set_error(BURGERS_EINVAL, "HBM budget too small (< 2 MiB)");
  e = cudaMalloc(&sv->pool, size_t(pool));
  if (e != cudaSuccess) return set_error(BURGERS_ENOMEM, "serve pool: out of device memory");
  sv->pool_bytes = pool;
  sv->long_region.init(0, long_bytes);
  sv->short_region.init(long_bytes, pool - long_bytes);
  e = ctx->scratch.ensure(size_t(3 * long_bytes));
  if (e == cudaSuccess) e = ctx->mlws.ensure(size_t(long_bytes));
  if (e != cudaSuccess) {
    cudaFree(sv->pool);
    return set_error(BURGERS_ENOMEM, "serve scratch: out of device memory");
  }
  sv->pinned.reserve(16);  // 1 GiB of page-locked request buffers up front
  e = cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->stream_b, cudaStreamNonBlocking);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k)
    e = cudaEventCreateWithFlags(&sv->ev[k], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sv->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sv->ev_join, cudaEventDisableTiming);
  for (int k = 0; k < 2 * kSliceRing && e == cudaSuccess; ++k)
    e = cudaEventCreate(&sv->tev[k]);
  if (e != cudaSuccess) {
    cudaFree(sv->pool);
    return cuda_error(e, "serve stream");
  }
  sv->t0 = now_s();
  burgers_server* raw = sv.release();
  raw->worker = std::thread(worker_loop, raw);
  *out = raw;
  return BURGERS_OK;
}

burgers_status burgers_serve_submit(burgers_server* sv, const burgers_request* rq, uint64_t* ticket) {
  if (!sv || !rq || !ticket) return set_error(BURGERS_EINVAL, "NULL argument");
  if (rq->scheme != BURGERS_EXPLICIT && rq->scheme != BURGERS_BTCS) return set_error(BURGERS_EINVAL, "bad scheme");
  if (!rq->u0_host) return set_error(BURGERS_EINVAL, "u0_host is NULL");
  burgers_instance in{0, rq->n, rq->bc, rq->dx, rq->nu, rq->dt, rq->nsteps};
  burgers_batch b{sv->cfg.dtype, 0, 1, &in};
  burgers_status st = validate_batch(&b, false);
  if (st != BURGERS_OK) return st;
  auto q = std::make_unique<Req>();
  q->r = *rq;
  q->r.u0_host = nullptr;
  q->bytes = int64_t(rq->n) * int64_t(sv->esz);
  q->long_row = rq->n > long_limit(sv, rq->scheme);
  const Region& rg = q->long_row ? sv->long_region : sv->short_region;
  if (q->bytes > rg.total()) return set_error(BURGERS_ENOMEM, "request larger than the pool region");
  // the page-locked copy of u0 is made outside the server lock (the arena has
  // its own), so neither the worker nor other submitters wait on it
  {
    std::lock_guard<std::mutex> pk(sv->pin_mu);
    q->pin = sv->pinned.alloc(q->bytes);
    if (q->pin) q->pin_dev = sv->pinned.device_alias(q->pin, q->bytes);
  }
  if (q->pin) {
    memcpy(q->pin, rq->u0_host, size_t(q->bytes));
  } else {
    q->u0.assign(static_cast<const unsigned char*>(rq->u0_host),
                 static_cast<const unsigned char*>(rq->u0_host) + q->bytes);
  }
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->fault != BURGERS_OK) {
    if (q->pin) {
      std::lock_guard<std::mutex> pk(sv->pin_mu);
      sv->pinned.release(q->pin, q->bytes);
    }
    return set_error(sv->fault, "server failed: " + sv->fault_msg);
  }
  q->t_submit = now_s() - sv->t0;
  q->ticket = sv->next_ticket++;
  *ticket = q->ticket;
  sv->pending.push_back(q.get());
  sv->reqs[q->ticket] = std::move(q);
  sv->stats.submitted += 1;
  sv->cv_work.notify_one();
  return BURGERS_OK;
}

static burgers_status take_result(burgers_server* sv, Req* q, void* out_host,
                                  burgers_req_stats* rs) {
  if (rs) {
    rs->t_submit = q->t_submit;
    rs->t_admit = q->t_admit;
    rs->t_done = q->t_done;
    rs->slices = q->slices;
    rs->status = q->status;
  }
  burgers_status st = q->status;
  if (q->state == RQ_DONE && out_host)
    memcpy(out_host, q->pin ? q->pin : q->out.data(), size_t(q->bytes));
  if (q->pin) {
    std::lock_guard<std::mutex> pk(sv->pin_mu);  // lock order: mu, then pin_mu
    sv->pinned.release(q->pin, q->bytes);
  }
  sv->reqs.erase(q->ticket);
  if (st != BURGERS_OK) return set_error(st, "request did not complete");
  return BURGERS_OK;
}

burgers_status burgers_serve_submit_timed(burgers_server* sv, const burgers_request* rqs,
                                          const double* t_arrive, int64_t count,
                                          uint64_t* tickets, double* late_s) {
  if (!sv || count < 0 || (count > 0 && (!rqs || !t_arrive || !tickets || !late_s)))
    return set_error(BURGERS_EINVAL, "NULL argument or negative count");
  for (int64_t i = 0; i < count; ++i) {
    tickets[i] = 0;
    late_s[i] = 0.0;
  }
  using clk = std::chrono::steady_clock;
  const clk::time_point t0 = clk::now();
  for (int64_t i = 0; i < count; ++i) {
    const clk::time_point due =
        t0 + std::chrono::duration_cast<clk::duration>(std::chrono::duration<double>(t_arrive[i]));
    if (clk::now() < due) std::this_thread::sleep_until(due);
    const burgers_status st = burgers_serve_submit(sv, &rqs[i], &tickets[i]);
    if (st != BURGERS_OK) {
      tickets[i] = 0;
      return st;
    }
    // how late the request reached the server against its arrival time
    late_s[i] = std::max(0.0, std::chrono::duration<double>(clk::now() - due).count());
  }
  return BURGERS_OK;
}

burgers_status burgers_serve_poll(burgers_server* sv, uint64_t ticket, void* out_host,
                                  burgers_req_stats* rs) {
  if (!sv) return set_error(BURGERS_EINVAL, "NULL server");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return set_error(BURGERS_ENOTFOUND, "unknown ticket");
  Req* q = it->second.get();
  if (q->state == RQ_PENDING || q->state == RQ_ACTIVE) return BURGERS_EAGAIN;
  return take_result(sv, q, out_host, rs);
}

burgers_status burgers_serve_wait(burgers_server* sv, uint64_t ticket, double timeout_s,
                                  void* out_host, burgers_req_stats* rs) {
  if (!sv) return set_error(BURGERS_EINVAL, "NULL server");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return set_error(BURGERS_ENOTFOUND, "unknown ticket");
  Req* q = it->second.get();
  const auto deadline = std::chrono::steady_clock::now() +
                        std::chrono::microseconds(int64_t(std::max(0.0, timeout_s) * 1e6));
  while (q->state == RQ_PENDING || q->state == RQ_ACTIVE) {
    if (sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout &&
        (q->state == RQ_PENDING || q->state == RQ_ACTIVE))
      return set_error(BURGERS_ETIMEOUT, "request not finished before the timeout");
  }
  return take_result(sv, q, out_host, rs);
}

burgers_status burgers_serve_wait_any(burgers_server* sv, double timeout_s, uint64_t* ticket) {
  if (!sv || !ticket) return set_error(BURGERS_EINVAL, "NULL argument");
  std::unique_lock<std::mutex> lk(sv->mu);
  const auto deadline = std::chrono::steady_clock::now() +
                        std::chrono::microseconds(int64_t(std::max(0.0, timeout_s) * 1e6));
  for (;;) {
    while (!sv->done_q.empty()) {
      const uint64_t t = sv->done_q.front();
      sv->done_q.pop_front();
      if (sv->reqs.count(t)) {  // skip tickets already taken by poll / wait
        *ticket = t;
        return BURGERS_OK;
      }
    }
    if (sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && sv->done_q.empty())
      return set_error(BURGERS_ETIMEOUT, "no request finished before the timeout");
  }
}

burgers_status burgers_serve_cancel(burgers_server* sv, uint64_t ticket) {
  if (!sv) return set_error(BURGERS_EINVAL, "NULL server");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return set_error(BURGERS_ENOTFOUND, "unknown ticket");
  it->second->cancel = true;
  sv->cv_work.notify_one();
  return BURGERS_OK;
}

burgers_status burgers_serve_get_stats(burgers_server* sv, burgers_serve_stats* out) {
  if (!sv || !out) return set_error(BURGERS_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  *out = sv->stats;
  out->pending = int64_t(sv->pending.size());
  out->active = int64_t(sv->active.size());
  out->pool_bytes = sv->pool_bytes;
  out->pool_used = sv->short_region.used() + sv->long_region.used();
  out->now_s = now_s() - sv->t0;
  return BURGERS_OK;
}

burgers_status burgers_serve_destroy(burgers_server* sv) {
  if (!sv) return set_error(BURGERS_EINVAL, "NULL server");
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  cudaSetDevice(sv->ctx->device);
  if (sv->stream) cudaStreamSynchronize(sv->stream);
  if (sv->stream_b) cudaStreamSynchronize(sv->stream_b);
  for (int k = 0; k < 2; ++k)
    if (sv->ev[k]) cudaEventDestroy(sv->ev[k]);
  if (sv->ev_fork) cudaEventDestroy(sv->ev_fork);
  if (sv->ev_join) cudaEventDestroy(sv->ev_join);
  for (int k = 0; k < 2 * kSliceRing; ++k)
    if (sv->tev[k]) cudaEventDestroy(sv->tev[k]);
  if (sv->stream_b) cudaStreamDestroy(sv->stream_b);
  if (sv->stream) cudaStreamDestroy(sv->stream);
  if (sv->pool) cudaFree(sv->pool);
  burgers_status st = sv->fault;
  delete sv;
  return st == BURGERS_OK ? BURGERS_OK : st;
}

}  // extern "C"
