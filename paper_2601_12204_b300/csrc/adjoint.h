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

// Per-row record of the long-row explicit adjoint (adjoint_long.cu).
struct AdjLongRow {
  int32_t tile_begin, tile_end;  // the row's tiles in the item list
  int32_t out_index;             // index of the row in the caller's batch
  int32_t pad;
  double ds_dnu;                 // dt / dx^2
};

}  // namespace burgers
