// multilevel.cu -- multi-level partitioned BTCS solver for rows too long to
// stay resident in one CTA (filled in below).
#include "api_internal.h"
#include "kernels.h"

namespace burgers {

void register_multilevel(std::vector<KernelEntry>& reg) { (void)reg; }

burgers_status plan_multilevel(burgers_ctx* ctx, const burgers_batch* batch,
                               const std::vector<int64_t>& longs, Plan* p) {
  (void)ctx; (void)batch; (void)longs; (void)p;
  return set_error(BURGERS_EINVAL, "BTCS rows longer than the resident limit are not supported yet");
}

cudaError_t enqueue_multilevel_launch(burgers_ctx* ctx, Plan* p, const Launch& L, void* u,
                                      cudaStream_t st) {
  (void)ctx; (void)p; (void)L; (void)u; (void)st;
  return cudaErrorNotSupported;
}

}  // namespace burgers
