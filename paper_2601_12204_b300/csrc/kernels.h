// kernels.h -- host-side registry of the libburgers CUDA kernels.
//
// Every kernel template instantiation is registered with its kind, dtype and
// launch shape, so the dispatcher and the autotuner can query occupancy and
// launch any of them through cudaLaunchKernel without a switch per shape.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"

namespace burgers {

enum KernelKind : int32_t {
  K_EXPLICIT_RESIDENT = 0,  // whole row in registers, all steps in one launch
  K_EXPLICIT_STREAM = 1,    // window of a long row, K steps per HBM pass
  K_BTCS_RESIDENT = 2,      // whole row in registers, partitioned solve per step
  K_BTCS_REDUCE = 3,        // multi-level BTCS: chunk elimination of one level
  K_BTCS_RECOVER = 4,       // multi-level BTCS: back-substitution of one level
  K_BTCS_TOP = 5,           // multi-level BTCS: resident solve of the top level
  K_ADJ_EXPLICIT = 6,       // adjoint of the explicit solve (resident rows)
  K_ADJ_BTCS = 7,           // adjoint of the BTCS solve (resident rows)
  K_EXPLICIT_STEP1 = 8,     // one explicit step per HBM pass over tiles of long rows
  K_RK4_RESIDENT = 9,       // RK4 (Eq. 22), whole row in registers
  K_RK4_STREAM = 10,        // RK4 window of a long row, K steps per HBM pass
  K_CN_RESIDENT = 11,       // Crank-Nicolson (lagged upwind), whole row per CTA
  K_PICARD_RESIDENT = 12,   // Picard-iterated implicit upwind, whole row per CTA
  K_NEWTON_RESIDENT = 13,   // Newton on the Eq. 11 residual, whole row per CTA
  K_BTCS_CLUSTER = 14,      // lagged BTCS, row resident in a cluster of `exact` CTAs
  K_EXPLICIT_STEP1_BULK = 15,  // K_EXPLICIT_STEP1 over tiles moved by bulk copies, `exact` stages
  K_BTCS_THOMAS = 16,       // lagged BTCS, one thread per row (Thomas), c = longest row
  K_CN_CLUSTER = 17,        // Crank-Nicolson, row resident in a cluster of `exact` CTAs
  K_PICARD_CLUSTER = 18,    // Picard-iterated implicit upwind, row resident in a cluster
  K_NEWTON_CLUSTER = 19,    // Newton on the Eq. 11 residual, row resident in a cluster
  K_KIND_COUNT
};

// Work item of the tiled kernels: tile `tile` of row `row`.
struct TileItem {
  int32_t row;
  int32_t tile;
};

struct KernelEntry {
  int32_t kind;
  int32_t dtype;  // 0 FP32, 1 FP64
  int32_t nt;     // threads per CTA
  int32_t c;      // nodes (or rows) per thread
  int32_t exact;  // resident kernels: row length == nt * c
  const void* fn;
  size_t dyn_smem;  // dynamic shared memory per CTA
};

// All registered kernels (built on first use).
const std::vector<KernelEntry>& kernel_registry();

// Looks up a kernel; nullptr if that shape is not instantiated.
const KernelEntry* find_kernel(int kind, int dtype, int nt, int c, int exact);

// Sets the dynamic shared memory attribute of every registered kernel.
cudaError_t prepare_kernels();

// Whether at least one cluster of a K_BTCS_CLUSTER entry (exact = cluster
// size) can be resident on the current device.
bool cluster_fits(const KernelEntry& e);

}  // namespace burgers
