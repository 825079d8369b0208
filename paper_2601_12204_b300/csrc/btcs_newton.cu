// btcs_newton.cu -- instantiations of the resident implicit kernel for
// Newton-Raphson on the residual of Eq. 11 (Eq. 10-15).
#include "btcs_x2.cuh"

namespace burgers {

#define REG_VAR(KIND, VAR, T, DT, NT, C)                                                    \
  reg.push_back({KIND, DT, NT, C, 1,                                                        \
                 reinterpret_cast<const void*>(&k_btcs_resident<T, NT, C, true, VAR>),     \
                 btcs_dsm<T, NT, C, VAR>()});                                              \
  reg.push_back({KIND, DT, NT, C, 0,                                                        \
                 reinterpret_cast<const void*>(&k_btcs_resident<T, NT, C, false, VAR>),    \
                 btcs_dsm<T, NT, C, VAR>()});
// FP32 rows with C even: the packed-pair kernel (exact rows; ragged rows where C >= 4)
#define REG_VAR_X2(KIND, VAR, NT, C)                                                         \
  reg.push_back({KIND, 0, NT, C, 1,                                                         \
                 reinterpret_cast<const void*>(&k_btcs_resident_x2<NT, C, VAR>),           \
                 btcs_x2_dsm<NT, C, VAR>()});                                              \
  reg.push_back(ragged_fp32_entry<NT, C, VAR>(KIND));
#define REG_SHAPES(KIND, VAR)                                                                \
  REG_VAR(KIND, VAR, float, 0, 32, 1) REG_VAR_X2(KIND, VAR, 32, 2)                         \
  REG_VAR_X2(KIND, VAR, 32, 4) REG_VAR_X2(KIND, VAR, 32, 8)                                \
  REG_VAR_X2(KIND, VAR, 64, 8) REG_VAR_X2(KIND, VAR, 128, 8)                               \
  REG_VAR_X2(KIND, VAR, 64, 32)                                                            \
  REG_VAR_X2(KIND, VAR, 256, 8) REG_VAR_X2(KIND, VAR, 128, 16)                             \
  REG_VAR_X2(KIND, VAR, 256, 16) REG_VAR_X2(KIND, VAR, 128, 32)                            \
  REG_VAR_X2(KIND, VAR, 256, 32)                                                           \
  REG_VAR(KIND, VAR, double, 1, 32, 1) REG_VAR(KIND, VAR, double, 1, 32, 2)                \
  REG_VAR(KIND, VAR, double, 1, 32, 4) REG_VAR(KIND, VAR, double, 1, 32, 8)                \
  REG_VAR(KIND, VAR, double, 1, 64, 8) REG_VAR(KIND, VAR, double, 1, 128, 8)               \
  REG_VAR(KIND, VAR, double, 1, 256, 8) REG_VAR(KIND, VAR, double, 1, 128, 16)             \
  REG_VAR(KIND, VAR, double, 1, 512, 8)

void register_newton(std::vector<KernelEntry>& reg) { REG_SHAPES(K_NEWTON_RESIDENT, VAR_NEWTON) }

}  // namespace burgers
