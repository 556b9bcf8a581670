// FP64 elementary functions of the integrator's pair forces, arranged so that
// most of their work runs on the FP32 and integer pipes.  The FP64 pipe is the
// integrator's bottleneck (a GB300 SM retires 2 FP64 lanes per cycle against
// 128 FP32 lanes), so each routine takes an FP32 estimate and finishes it
// with as few FP64 instructions as its accuracy needs:
//   rsqrt_seeded   1/sqrt(s) in 3 FP64 instructions (plus an FP32 sqrt(s)),
//   texp_hint      e^x in 3, given an FP32 approximation of x.
#pragma once

#include <cuda_runtime.h>

#include "ff.cuh"
#include "texp.cuh"

namespace qcams {
namespace {

// 1/sqrt(s) for a double s in the FP32 normal range [2^-126, 2^128); other
// inputs (0, subnormal, huge, inf, NaN, negative) give NaN.  On return rf
// holds an FP32 approximation of sqrt(s) (relative error below 2^-21).
//
// The seed y0 is the FP32 hardware reciprocal square root of s truncated to
// 24 bits (relative error below 2^-21).  With e = 1 - s y0^2 the series
// 1/sqrt(s) = y0 (1 - e)^(-1/2) = y0 (1 + e/2 + 3e^2/8 + 5e^3/16 + ...)
// truncated after e^2 leaves 5|e|^3/16 < 2^-60.  Because y0 carries 24
// significant bits, y0^2 is exact in a double: it is formed by an integer
// multiply of the significands, so e costs one FMA.  y0/2 and 3y0/8 are
// built on the integer / FP32 pipes (3y0/8 only multiplies e, so its FP32
// rounding does not matter).  FP64 work: e, then two FMAs of the series.
__device__ __forceinline__ double rsqrt_seeded(double s, float& rf) {
  const unsigned hi = (unsigned)__double2hiint(s), lo = (unsigned)__double2loint(s);
  // biased exponent in [897, 1150] <=> FP32 normal (sign bit set: out of range)
  const bool in_range = (hi >> 20) - 897u < 254u;
  // FP32 copy of s: exponent rebiased by 1023 - 127 = 896, significand truncated
  const float sf = __uint_as_float(__funnelshift_l(lo, hi - (896u << 20), 3));
  float yf;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(sf));
  rf = sf * yf;
  const unsigned yb = __float_as_uint(yf);
  const unsigned yhi = (yb >> 3) + (896u << 20), ylo = yb << 29;   // yf as a double
  const double y0 = __hiloint2double(in_range ? (int)yhi : 0x7ff80000, (int)ylo);
  const double y0h = __hiloint2double((int)(yhi - (1u << 20)), (int)ylo);
  const unsigned y38b = __float_as_uint(0.375f * yf);
  const double y38 = __hiloint2double((int)((y38b >> 3) + (896u << 20)), (int)(y38b << 29));
  // y0^2: the 24-bit significand M squared is a 47- or 48-bit integer
  const unsigned long long M = (yb & 0x7fffffu) | 0x800000u;
  const unsigned long long P = M * M;
  const unsigned top = (unsigned)(P >> 47);
  const long long ey = (long long)(yb >> 23) - 127;
  // P << (6 - top) puts the leading bit at bit 52, where it adds one to the
  // exponent field: hence the bias 1022 instead of 1023
  const double Y = __longlong_as_double((long long)(P << (6 - top)) + ((2 * ey + top + 1022) << 52));
  const double e = fma(-s, Y, 1.0);
  const double c = fma(e, y38, y0h);
  return fma(e, c, y0);
}

constexpr float kExpInvLf = (float)kExpInvL;

// e^x by the table method of texp, for x < 700; below -700 the result is
// 2^-1010 as in texp.  xa is an FP32 approximation of x (|xa - x| below about
// 1e-5 + 2^-20 |x|), from which k = round(x N / ln 2) is formed on the FP32
// pipe (the 1.5 * 2^23 shift rounds to an integer) and converted to a double
// on the integer pipe.  For |x| up to about 100, k is at most one away from
// the nearest integer, which only widens |r| from ln2/(2N) to about
// 0.62 ln2/N, where the cubic's truncation stays below 1e-16 relative; near
// x = -700 it grows to about 2e-14 relative, on values below 1e-304.  The
// reduction uses ln2/N rounded to a double, without the tail constant: that
// adds an error of |x| 2^-54.7 to the argument, below the |x| 2^-53 that the
// rounding of x itself already carries.
// With |r| <= 2.1e-4, e^r - 1 = r + w, w = r^2/2 + r^3/6 <= 2.2e-8: w is
// needed to ~1e-18 absolute (the result's relative error is that of 1 + r +
// w), so r^2/2 is formed in float-float (r split into a float pair on the
// integer pipe, r_h^2 split exactly by an FMA) and r^3/6 <= 1.5e-12 in
// FP32, then w is rebuilt as a double on the integer pipe.  FP64 work: the
// reduction, r + w, and the table product.
__device__ __forceinline__ double texp_hint(double x, float xa, const double* __restrict__ T) {
  const float kf = fmaf(xa, kExpInvLf, 12582912.0f);   // 1.5 * 2^23 + k
  const int k = __float_as_int(kf) - 0x4B400000;
  const unsigned kb = __float_as_uint(kf - 12582912.0f);   // k as an FP32 value, exact
  const unsigned khi = (kb & 0x80000000u) | (((kb & 0x7fffffffu) >> 3) + (896u << 20));
  const double kd = __hiloint2double(kb ? (int)khi : 0, (int)(kb << 29));
  const double r = fma(-kd, kExpL1, x);
  float rh, rl;
  split_ff(r, rh, rl);
  const float P = __fmul_rn(rh, rh);
  const float Pl = fmaf(2.0f * rh, rl, fmaf(rh, rh, -P));   // r^2 = P + Pl to 2^-46
  const float cub = (P * rh) * (1.0f / 6.0f);
  const double p = r + ff_to_double(0.5f * P, fmaf(0.5f, Pl, cub));
  const double Tj = T[k & (kExpTableSize - 1)];
  const double y = fma(Tj, p, Tj);
  const double ex = __hiloint2double(__double2hiint(y) + ((k >> 11) << 20), __double2loint(y));
  return ((unsigned)__double2hiint(x) > 0xC085E000u) ? 0x1.0p-1010 : ex;
}

}  // namespace
}  // namespace qcams
