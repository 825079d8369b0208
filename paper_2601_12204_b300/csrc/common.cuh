// common.cuh -- device-side types and helpers shared by the libburgers kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace burgers {

constexpr unsigned FULL_MASK = 0xffffffffu;

// Per-row launch record, packed on the host from burgers_instance.
// r = dt/dx and s = nu dt/dx^2 are formed in FP64 on the host.
struct RowDesc {
  int64_t offset;  // first element of the row
  int64_t nsteps;  // steps to advance
  double r;        // dt / dx
  double s;        // nu dt / dx^2
  double ds_dnu;   // dt / dx^2 (derivative of s with respect to nu)
  int32_t n;       // nodes
  int32_t bc;      // 0 periodic, 1 Dirichlet
  int32_t iters = 1;  // iterations per step (Picard / Newton variants)
  int32_t pad = 0;
  float rf = 0.f, hf = 0.f, sf = 0.f;  // r, r/2, s rounded once to FP32 (set_fp32_coefs)
  int32_t pad2 = 0;
};

// Fills the FP32 copies of a row's coefficients from its FP64 r and s, so the
// FP32 kernels that read a descriptor per tile convert nothing: bitwise the
// values float(r), float(r / 2) (= float(r) / 2) and float(s).
__host__ __device__ inline void set_fp32_coefs(RowDesc& d) {
  d.rf = static_cast<float>(d.r);
  d.hf = static_cast<float>(0.5 * d.r);
  d.sf = static_cast<float>(d.s);
}

// r, r/2 and s of a row in the kernel's type.
template <typename T>
struct RowCoefs {
  T r, h, s;
};
__device__ __forceinline__ RowCoefs<float> row_coefs(const RowDesc& d, float) {
  return {d.rf, d.hf, d.sf};
}
__device__ __forceinline__ RowCoefs<double> row_coefs(const RowDesc& d, double) {
  return {d.r, 0.5 * d.r, d.s};
}

enum : int32_t { BC_PERIODIC = 0, BC_DIRICHLET = 1 };

__device__ __forceinline__ float tfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double tfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float tabs(float x) { return fabsf(x); }
__device__ __forceinline__ double tabs(double x) { return fabs(x); }
__device__ __forceinline__ float tmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double tmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float tmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double tmin(double a, double b) { return fmin(a, b); }

// Reciprocal used in the tridiagonal eliminations. Every pivot there is >= 1
// (the BTCS matrices are diagonally dominant by a margin of one, and so are
// their Schur complements), so the FP32 hardware approximation (relative error
// about 2^-23 on normal inputs) is safe; FP64 uses the IEEE division.
__device__ __forceinline__ float recip(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// Shared-memory store executed only where pred holds: a predicated store
// instruction, so the edge lanes publishing their values cost no branch.
__device__ __forceinline__ void st_shared_if(float* p, float v, bool pred) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t@q st.shared.f32 [%0], %1;\n\t}"
      :: "r"(static_cast<unsigned>(__cvta_generic_to_shared(p))), "f"(v), "r"(int(pred))
      : "memory");
}
__device__ __forceinline__ void st_shared_if(double* p, double v, bool pred) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t@q st.shared.f64 [%0], %1;\n\t}"
      :: "r"(static_cast<unsigned>(__cvta_generic_to_shared(p))), "d"(v), "r"(int(pred))
      : "memory");
}

template <typename T>
__device__ __forceinline__ T shfl(T v, int src) {
  return __shfl_sync(FULL_MASK, v, src);
}
template <typename T>
__device__ __forceinline__ T shfl_up(T v, int d) {
  return __shfl_up_sync(FULL_MASK, v, d);
}
template <typename T>
__device__ __forceinline__ T shfl_down(T v, int d) {
  return __shfl_down_sync(FULL_MASK, v, d);
}

// Explicit forward-Euler upwind/central increment of node value u with left
// and right neighbours ul, ur (Eq. 21 with the upwind side of Sec. 2.2):
//   u' - u = -r (u+ (u - ul) + u- (ur - u)) + s (ur - 2u + ul)
//          = p (ur - u) - q (u - ul),
//   p = s - r u- = s + h (|u| - u),   q = s + r u+ = p + r u,   h = r/2,
// returned plus `add`. FP64: one difference (u - ul is the previous node's
// ur - u) and five FP64 operations, no min/max. FP32 forms q as s + r u+
// (one rounding, from max(u, 0)), bitwise what the packed-pair steps of the
// resident and windowed kernels compute, so every FP32 kernel (forward,
// windowed, single-step, adjoint recompute) follows the same trajectory.
template <typename T>
__device__ __forceinline__ T explicit_increment(T u, T ul, T ur, T r, T h, T s, T add) {
  const T dr = ur - u;
  const T dl = u - ul;
  const T p = tfma(h, tabs(u) - u, s);
  if constexpr (sizeof(T) == 4) {
    const T q = tfma(r, tmax(u, T(0)), s);
    return tfma(p, dr, tfma(-q, dl, add));
  } else {
    const T q = tfma(r, u, p);
    return tfma(p, dr, tfma(-q, dl, add));
  }
}

// Packed FP32 arithmetic (the f32x2 forms of add, sub and fma): one
// instruction applies the operation to two independent float lanes, each
// rounded as its scalar form would be. The FMA pipe executes the same number
// of lane operations either way; the packed forms halve the instructions the
// schedulers must issue, which is what limits the register-resident stencil.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

// u' = u + increment. FP64 adds directly (one rounding per step is far below
// the FP64 parity bar). FP32 carries the rounding error of every addition in
// a per-node compensation term lo (Kahan summation over the time steps): the
// stencil reads u only, the increment is formed minus lo and the new rounding
// error goes back into lo. This keeps the FP32 state within ~1e-7 relative of
// the FP64 trajectory over thousands of steps, where plain FP32 accumulation
// drifts coherently on smooth, diffusion-limited rows.
template <typename T>
struct Kahan {
  static constexpr bool on = false;
};
template <>
struct Kahan<float> {
  static constexpr bool on = true;
};

// Steps between folds of the FP32 split state (value at the last fold plus
// the increments summed since) of the explicit kernels.
constexpr int SPLIT_FOLD = 32;

// The 16-byte vector type of T (four floats or two doubles).
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
};
template <>
struct Vec16<double> {
  using type = double2;
};

template <typename T>
__device__ __forceinline__ T explicit_update(T u, T ul, T ur, T r, T h, T s, T& lo) {
  if constexpr (Kahan<T>::on) {
    const T y = explicit_increment(u, ul, ur, r, h, s, -lo);
    const T t = u + y;
    lo = (t - u) - y;
    return t;
  } else {
    (void)lo;
    return explicit_increment(u, ul, ur, r, h, s, u);
  }
}

// The FP32 compensation term of a streamed state, stored in 8 bits. After a
// compensated update the term lo of the value v satisfies |lo| <= ulp(v) / 2,
// so lo / (ulp(v) / 256) lies in [-128, 128]: it is stored as that integer
// (rounded to nearest, saturated to [-128, 127]) and read back as
// q ulp(v) / 256. The quantum, 1/256 ulp(v), is far below what the
// compensation has to carry across HBM passes (a 2^24-node diffusion-limited
// run keeps the full Kahan accuracy with it). Both directions scale by powers
// of two built from v's exponent bits with integer arithmetic (no branch):
// 256 / ulp(v) = 2^(158 - e) and ulp(v) / 256 = 2^(e - 158) for the biased
// exponent e of v. Values with e <= 31 (|v| < 2^-95) read back 0 whatever
// was stored.
__device__ __forceinline__ signed char lo8_encode(float v, float lo) {
  const unsigned ebits = __float_as_uint(v) & 0x7f800000u;
  const float inv = __uint_as_float(0x8e800000u - ebits);  // 2^(158 - e), exact for e >= 31
  int q;
  asm("cvt.rni.sat.s8.f32 %0, %1;" : "=r"(q) : "f"(lo * inv));
  return static_cast<signed char>(q);
}
__device__ __forceinline__ float lo8_decode(float v, signed char q) {
  const int ebits = int(__float_as_uint(v) & 0x7f800000u) - (31 << 23);
  return static_cast<float>(q) * __int_as_float(ebits > 0 ? ebits : 0);  // 2^(e - 158), or 0
}

// u + d with the same compensation (BTCS increments).
template <typename T>
__device__ __forceinline__ T comp_add(T u, T d, T& lo) {
  if constexpr (Kahan<T>::on) {
    const T y = d - lo;
    const T t = u + y;
    lo = (t - u) - y;
    return t;
  } else {
    (void)lo;
    return u + d;
  }
}

}  // namespace burgers
