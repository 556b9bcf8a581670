// Pieces shared by the FP64 integrators (one thread per trajectory in
// integrate.cu, a group of lanes per trajectory in integrate_grp.cu): the FP32
// magnitudes the step-size controller works with, the controller's MUFU
// arithmetic, and the float-float copy of the Runge-Kutta-Nystrom
// coefficients (Dormand-Prince 5(4), Sec. 3.2).
#pragma once

#include <cuda_runtime.h>

#include "dp5_tableau.cuh"
#include "ff.cuh"

namespace qcams {
namespace {

// |x| as a float, truncated to 20 mantissa bits, using only integer
// instructions on the high word of x; values below 2^-126 become 0 and
// values above FLT_MAX saturate.  Sets `bad` for inf / NaN.
__device__ __forceinline__ float mag_f(double x, unsigned& bad) {
  const unsigned hi = (unsigned)__double2hiint(x) & 0x7fffffffu;
  bad |= (hi >= 0x7ff00000u) ? 1u : 0u;
  const int e = (int)(hi >> 20) - 896;
  unsigned bits = ((unsigned)e << 23) | ((hi & 0x000fffffu) << 3);
  bits = (e <= 0) ? 0u : bits;
  bits = (e >= 255) ? 0x7f7fffffu : bits;
  return __uint_as_float(bits);
}
__device__ __forceinline__ float signed_f(double x) {
  unsigned bad = 0;
  const float m = mag_f(x, bad);
  return (__double2hiint(x) < 0) ? -m : m;
}
// |x| of an FP32 error estimate; sets `bad` for inf / NaN.
__device__ __forceinline__ float err_mag(float x, unsigned& bad) {
  bad |= ((__float_as_uint(x) & 0x7f800000u) == 0x7f800000u) ? 1u : 0u;
  return fabsf(x);
}
// Approximate reciprocal (one MUFU instruction, about 1 ulp): the error
// norm's scales are positive and far from the FP32 range limits (atol > 0).
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// x^(-1/10) for the step-size factor, as 2^(-log2(x) / 10) (two MUFU
// instructions and a multiply).  x = 0 or subnormal gives +inf, which the
// controller caps at the maximum growth factor as it does for a zero norm.
__device__ __forceinline__ float pow_m01(float x) {
  float l, r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(x));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(-0.1f * l));
  return r;
}
// Order of non-negative doubles equals the order of their bit patterns.
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }

// The coefficients of the float-float sums as float pairs.
struct RknTabFF {
  FFc a2[8][8];
  FFc e[8];
  FFc ea[8];
};
__host__ __device__ constexpr RknTabFF make_rkn_tab_ff() {
  RknTabFF f{};
  const RknTab t = make_rkn_tab();
  for (int s = 1; s <= 7; ++s) {
    f.e[s] = make_ffc(t.e[s]);
    f.ea[s] = make_ffc(t.ea[s]);
    for (int q = 1; q <= 7; ++q) f.a2[s][q] = make_ffc(t.a2[s][q]);
  }
  return f;
}

}  // namespace
}  // namespace qcams
