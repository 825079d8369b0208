// btcs.cu -- implicit BTCS step with lagged upwind coefficients (Sec. 2.4,
// Eq. 23): A(u^n) u^{n+1} = u^n with, for node i and a = u^n_i,
//   l_i = -r a+ - s,   d_i = 1 + r|a| + 2s,   c_i = r a- - s,
// periodic rows cyclic (Eq. 18), Dirichlet end nodes held (Eq. 16-17, written
// here as identity rows). The coefficients are formed from u^n in registers and
// never stored.
//
// Partitioned elimination. Thread t owns a chunk of C consecutive rows with
// end row e. A forward sweep normalises each row to
//     x_i + ch_i x_{i+1} + ah_i L = dh_i          (L = x of the previous chunk's end)
// and a backward sweep turns the rows before e into
//     x_i = delta_i - alpha_i L - gamma_i X_t      (X_t = x_e).
// Substituting the next chunk's first-row relation into row e gives one
// tridiagonal row per chunk in the unknowns X_{t-1}, X_t, X_{t+1}: a reduced
// system of NT rows (cyclic for periodic rows). Warp 0 solves it: the
// cyclic corners are split off by Sherman-Morrison (gamma = -B_0, correction
// factor (v.y)/(1 + v.z) with its denominator in extended precision), each lane eliminates Q = NT/32
// reduced rows the same way, and the remaining 32-row system is solved by
// parallel cyclic reduction over warp shuffles. Back-substitution then
// recovers every node from delta, alpha, gamma and the chunk-end values.
//
// All pivots are >= 1 because every matrix involved is diagonally dominant by
// a margin of one (an M-matrix and its Schur complements), so no pivoting is
// needed.
#include "btcs_x2.cuh"

namespace burgers {

// FP32 rows with C even run the packed-pair kernel (btcs_x2.cuh): rows of
// exactly NT*C nodes, and ragged rows where C >= 4.
#define REG_BTCS_X2(NT, C)                                                                      \
  reg.push_back({K_BTCS_RESIDENT, 0, NT, C, 1,                                                  \
                 reinterpret_cast<const void*>(&k_btcs_resident_x2<NT, C, VAR_BTCS>),          \
                 btcs_x2_dsm<NT, C, VAR_BTCS>()});                                              \
  reg.push_back(ragged_fp32_entry<NT, C, VAR_BTCS>(K_BTCS_RESIDENT));

#define REG_BTCS(T, DT, NT, C)                                                                  \
  reg.push_back({K_BTCS_RESIDENT, DT, NT, C, 1,                                                 \
                 reinterpret_cast<const void*>(&k_btcs_resident<T, NT, C, true, VAR_BTCS>),    \
                 btcs_dsm<T, NT, C, VAR_BTCS>()});                                              \
  reg.push_back({K_BTCS_RESIDENT, DT, NT, C, 0,                                                 \
                 reinterpret_cast<const void*>(&k_btcs_resident<T, NT, C, false, VAR_BTCS>),   \
                 btcs_dsm<T, NT, C, VAR_BTCS>()});

void register_btcs(std::vector<KernelEntry>& reg) {
  REG_BTCS(float, 0, 32, 1) REG_BTCS_X2(32, 2) REG_BTCS_X2(32, 4)
  REG_BTCS_X2(32, 8) REG_BTCS_X2(64, 8) REG_BTCS_X2(128, 8)
  REG_BTCS_X2(256, 8) REG_BTCS_X2(128, 16) REG_BTCS_X2(256, 16)
  REG_BTCS_X2(512, 8) REG_BTCS_X2(512, 16) REG_BTCS_X2(1024, 8)
  REG_BTCS_X2(64, 32) REG_BTCS_X2(128, 32) REG_BTCS_X2(256, 32)
  REG_BTCS(double, 1, 32, 1) REG_BTCS(double, 1, 32, 2) REG_BTCS(double, 1, 32, 4)
  REG_BTCS(double, 1, 32, 8) REG_BTCS(double, 1, 64, 8) REG_BTCS(double, 1, 128, 8)
  REG_BTCS(double, 1, 256, 8) REG_BTCS(double, 1, 512, 8) REG_BTCS(double, 1, 256, 16)
  REG_BTCS(double, 1, 128, 16)
}

}  // namespace burgers
