// registry.cu -- collects the kernel template instantiations of every
// translation unit into one searchable table.
#include <mutex>

#include "kernels.h"

namespace burgers {

void register_explicit(std::vector<KernelEntry>& reg);
void register_btcs(std::vector<KernelEntry>& reg);
void register_cn(std::vector<KernelEntry>& reg);
void register_picard(std::vector<KernelEntry>& reg);
void register_newton(std::vector<KernelEntry>& reg);
void register_btcs_cluster(std::vector<KernelEntry>& reg);
void register_multilevel(std::vector<KernelEntry>& reg);
void register_adjoint(std::vector<KernelEntry>& reg);
void register_step1_bulk(std::vector<KernelEntry>& reg);
void register_btcs_thomas(std::vector<KernelEntry>& reg);
void register_adjoint_long(std::vector<KernelEntry>& reg);

const std::vector<KernelEntry>& kernel_registry() {
  static std::vector<KernelEntry> reg;
  static std::once_flag once;
  std::call_once(once, [] {
    register_explicit(reg);
    register_btcs(reg);
    register_cn(reg);
    register_picard(reg);
    register_newton(reg);
    register_btcs_cluster(reg);
    register_multilevel(reg);
    register_adjoint(reg);
    register_step1_bulk(reg);
    register_btcs_thomas(reg);
    register_adjoint_long(reg);
  });
  return reg;
}

const KernelEntry* find_kernel(int kind, int dtype, int nt, int c, int exact) {
  for (const KernelEntry& e : kernel_registry())
    if (e.kind == kind && e.dtype == dtype && e.nt == nt && e.c == c && e.exact == exact)
      return &e;
  return nullptr;
}

cudaError_t prepare_kernels() {
  for (const KernelEntry& e : kernel_registry()) {
    if (e.dyn_smem > 0) {
      cudaError_t err = cudaFuncSetAttribute(e.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(e.dyn_smem));
      if (err != cudaSuccess) return err;
    }
    if ((e.kind == K_BTCS_CLUSTER || e.kind == K_CN_CLUSTER || e.kind == K_PICARD_CLUSTER ||
         e.kind == K_NEWTON_CLUSTER) &&
        e.exact > 8) {
      // a refusal only leaves the wide clusters unused (cluster_fits says so)
      if (cudaFuncSetAttribute(e.fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
          cudaSuccess)
        (void)cudaGetLastError();
    }
  }
  return cudaSuccess;
}

bool cluster_fits(const KernelEntry& e) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(e.exact));
  cfg.blockDim = dim3(unsigned(e.nt));
  cfg.dynamicSmemBytes = e.dyn_smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = unsigned(e.exact);
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, e.fn, &cfg) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return n > 0;
}

}  // namespace burgers
