// adjoint.h -- per-row descriptor of the adjoint kernels (adjoint.cu).
#pragma once

#include <stdint.h>

namespace burgers {

struct AdjRow {
  int64_t ckpt;       // workspace offset of the checkpoints (nckpt states of n values)
  int64_t seg;        // workspace offset of the segment states (stride + 1 of n values)
  int64_t stride;     // steps between checkpoints
  int64_t nckpt;      // number of checkpoints
  int32_t out_index;  // index of the row in the caller's batch (dJ/dnu slot)
  int32_t pad;
};

}  // namespace burgers
