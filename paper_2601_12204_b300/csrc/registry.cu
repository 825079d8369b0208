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
  }
  return cudaSuccess;
}

}  // namespace burgers
