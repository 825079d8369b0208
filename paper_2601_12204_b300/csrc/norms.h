// norms.h -- launchers of the FP64 row reductions (norms.cu).
#pragma once

#include <cuda_runtime.h>

#include "kernels.h"

namespace burgers {

constexpr int NORM_CHUNK = 16384;  // nodes per reduction item

cudaError_t launch_rel_l2(int dtype_u, int dtype_ref, const void* u, const void* ref,
                          const RowDesc* rows, const TileItem* items, int nitems,
                          const int32_t* first_item, int count, int chunk, double2* partial,
                          double* rel, double* rms, cudaStream_t st);

cudaError_t launch_cfl(int dtype, const void* u, const RowDesc* rows, const TileItem* items,
                       int nitems, const int32_t* first_item, const double2* dxnu, int count,
                       int chunk, double cfl, double* partial, double* dt, cudaStream_t st);

}  // namespace burgers
