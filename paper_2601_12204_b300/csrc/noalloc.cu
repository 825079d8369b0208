// noalloc.cu -- explicit solve of one long row without any device allocation.
//
// Some callers cannot allocate device memory while they run: an application
// whose memory arena already owns the whole GPU, a service that must keep a
// fixed footprint after start-up, or code called while another allocator
// holds its lock. burgers_explicit_advance_noalloc serves them. It runs the
// same streaming window kernel as burgers_explicit_advance, but the kernel's
// working copies (the ping-pong copy of the row, the two FP32 compensation
// buffers) and its launch descriptors live in one file-scope device array of
// fixed size that every GPU loading this library holds until the process
// exits. The caller still passes the row itself.
//
// The array is shared by every call on a device and keeps the last call's
// contents; what must start at zero (the compensation buffer) is cleared by
// each call. Calls whose work overlaps on the GPU (two streams, or two host
// threads) race on the array and must be serialised by the caller.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "../../include/burgers.h"
#include "api_internal.h"
#include "kernels.h"

namespace burgers {

constexpr int64_t NOALLOC_MAX_NODES = int64_t(1) << 20;
constexpr size_t NOALLOC_BYTES = size_t(16) << 20;
constexpr size_t NA_DESC = 0;           // one RowDesc
constexpr size_t NA_ITEMS = 256;        // up to NA_MAX_ITEMS tile items
constexpr int NA_MAX_ITEMS = int((8192 - 256) / sizeof(TileItem));
constexpr size_t NA_DATA = 8192;        // row copy, then the two compensation buffers

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// Writes the row descriptor and the tile list of one row into the array.
__global__ void k_noalloc_setup(RowDesc rd, RowDesc* desc, TileItem* items, int ntiles) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *desc = rd;
  for (int t = i; t < ntiles; t += gridDim.x * blockDim.x) items[t] = TileItem{0, t};
}

// Device address of the static array on the current device. Looked up on
// every call (a table lookup once the module is loaded, and no allocation), so
// a context recreated after cudaDeviceReset, whose module and array may sit
// elsewhere, is never handed a stale address. The first call on a device
// loads the library's module there, which is why it must not happen inside a
// stream capture.
static burgers_status noalloc_base(char** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(no-alloc scratch)");
  *out = static_cast<char*>(p);
  return BURGERS_OK;
}

}  // namespace burgers

using namespace burgers;

extern "C" burgers_status burgers_explicit_advance_noalloc(const burgers_instance* inst,
                                                           int32_t dtype, void* u_dev,
                                                           burgers_stream stream) {
  if (!inst || !u_dev) return set_error(BURGERS_EINVAL, "NULL argument");
  if (dtype != BURGERS_F32 && dtype != BURGERS_F64) return set_error(BURGERS_EINVAL, "bad dtype");
  const burgers_instance& in = *inst;
  if (in.bc != BURGERS_PERIODIC && in.bc != BURGERS_DIRICHLET) return set_error(BURGERS_EINVAL, "bad bc");
  if (!(in.dx > 0.0) || !(in.nu >= 0.0) || !(in.dt > 0.0) || in.nsteps < 0 || in.offset < 0)
    return set_error(BURGERS_EINVAL, "need dx > 0, nu >= 0, dt > 0, nsteps >= 0, offset >= 0");
  if (in.n < 128)
    return set_error(BURGERS_EINVAL, "no-alloc solve needs n >= 128 (use burgers_explicit_advance)");
  if (in.n > NOALLOC_MAX_NODES)
    return set_error(BURGERS_EINVAL,
                     "row longer than the 1048576-node limit of the no-alloc scratch array");
  if (in.nsteps == 0) return BURGERS_OK;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  char* base = nullptr;
  burgers_status st = noalloc_base(&base);
  if (st != BURGERS_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // window shape: 256 threads of 16 (FP32) or 8 (FP64) nodes for rows of 4096
  // nodes or more, 32 threads of 4 nodes below; K steps per pass (32 FP32, 16
  // FP64, at most a quarter of the window). The streaming path of
  // burgers_explicit_advance picks its shape from its tuning table instead, and
  // sends rows that fit one CTA to the resident kernel; results agree within
  // the FP32 / FP64 parity bars, not bitwise.
  const int nt = in.n >= 4096 ? 256 : 32;
  const int c = in.n >= 4096 ? (dtype == BURGERS_F32 ? 16 : 8) : 4;
  const int W = nt * c;
  const int K = std::min(dtype == BURGERS_F32 ? 32 : 16, W / 4);
  const int O = W - 2 * K;
  const int ntiles = int((in.n + O - 1) / O);
  if (ntiles > NA_MAX_ITEMS) return set_error(BURGERS_EINVAL, "row needs too many windows");
  const KernelEntry* k = find_kernel(K_EXPLICIT_STREAM, dtype, nt, c, 0);
  if (!k) return set_error(BURGERS_EINVAL, "streaming kernel shape missing");
  const size_t esz = dtype == BURGERS_F32 ? 4 : 8;
  // the array holds the row at offset 0: shift the caller's pointer instead
  char* u_row = static_cast<char*>(u_dev) + size_t(in.offset) * esz;
  RowDesc rd;
  rd.offset = 0;
  rd.nsteps = in.nsteps;
  rd.r = in.dt / in.dx;
  rd.s = in.nu * in.dt / (in.dx * in.dx);
  rd.ds_dnu = in.dt / (in.dx * in.dx);
  rd.n = in.n;
  rd.bc = in.bc;
  set_fp32_coefs(rd);
  RowDesc* desc = reinterpret_cast<RowDesc*>(base + NA_DESC);
  TileItem* items = reinterpret_cast<TileItem*>(base + NA_ITEMS);
  // the row copy, then (FP32) two compensation buffers of one byte per node,
  // each start 256-byte aligned
  const size_t span = (size_t(in.n) * esz + 255) & ~size_t(255);
  const size_t lo_span = (size_t(in.n) + 255) & ~size_t(255);
  void* copy = base + NA_DATA;
  void* lo_a = dtype == BURGERS_F32 ? base + NA_DATA + span : nullptr;
  void* lo_b = dtype == BURGERS_F32 ? base + NA_DATA + span + lo_span : nullptr;
  k_noalloc_setup<<<(ntiles + 255) / 256, 256, 0, s>>>(rd, desc, items, ntiles);
  e = cudaGetLastError();
  if (e == cudaSuccess && lo_a) e = cudaMemsetAsync(lo_a, 0, size_t(in.n), s);
  if (e != cudaSuccess) return cuda_error(e, "no-alloc set-up");
  if (k->dyn_smem > 0) {  // no context may have prepared the kernel on this device
    e = cudaFuncSetAttribute(k->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(k->dyn_smem));
    if (e != cudaSuccess) return cuda_error(e, "no-alloc kernel attribute");
  }
  int sms = 1, occ = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k->fn, k->nt, k->dyn_smem) != cudaSuccess ||
      occ < 1)
    occ = 1;
  const int grid = std::min(ntiles, sms * occ);
  const int64_t passes = (in.nsteps + K - 1) / K;
  int nitems = ntiles, kk = K;
  for (int64_t p = 0; p <= passes; ++p) {
    if (p == passes && passes % 2 == 0) break;  // result already back in the caller's row
    const bool to_copy = (p % 2) == 0;
    const void* src = to_copy ? static_cast<const void*>(u_row) : copy;
    void* dst = to_copy ? copy : static_cast<void*>(u_row);
    const void* lsrc = to_copy ? lo_a : lo_b;
    void* ldst = to_copy ? lo_b : lo_a;
    const RowDesc* rp = desc;
    const TileItem* ip = items;
    int64_t sb = p < passes ? p * K : in.nsteps;  // the extra pass only copies back
    void* args[] = {&src, &dst, &lsrc, &ldst, &rp, &ip, &nitems, &kk, &sb};
    e = cudaLaunchKernel(k->fn, dim3(grid), dim3(k->nt), args, k->dyn_smem, s);
    if (e != cudaSuccess) return cuda_error(e, "no-alloc streaming launch");
  }
  return BURGERS_OK;
}
