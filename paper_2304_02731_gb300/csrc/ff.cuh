// Float-float ("double-float") arithmetic on the FP32 and integer pipes, for
// the integrator's linear combinations that do not need a full FP64 result:
// the stage positions' acceleration corrections and the embedded error
// estimate.  A value is an unevaluated sum hi + lo of two floats.  GB300
// runs FP32 64 times faster than FP64, so a compensated dot product of ~11
// FP32 instructions per term is cheaper than one DFMA on the FP64 pipe.
#pragma once

#include <cuda_runtime.h>

namespace qcams {
namespace {

// a = hi + lo, |a - hi - lo| <= 2^-46 |a|, on the integer pipe: hi is a
// truncated to 24 significant bits, lo the next 23 bits.  |a| < 2^-80
// (and 0) gives (0, 0); inf / NaN give (NaN, 0); |a| >= 2^80 saturates to
// (+-2^80, 0), so that sums of a few such terms with weights below 2^40
// stay finite: an integrator stage that met a huge (finite) force then
// yields a huge error estimate and a rejected step, as in FP64, instead of
// a NaN.
__device__ __forceinline__ void split_ff(double a, float& hi, float& lo) {
  const unsigned h = (unsigned)__double2hiint(a), l = (unsigned)__double2loint(a);
  const unsigned sgn = h & 0x80000000u, ha = h & 0x7fffffffu;
  const bool ok = ha >= (943u << 20);     // exponent of 2^-80 and above
  const bool big = ha >= (1103u << 20);   // 2^80 and above (inf / NaN too)
  const unsigned hb = __funnelshift_l(l, ha - (896u << 20), 3) | sgn;
  // remaining 29 significand bits m, value m 2^(E-52); m >> 6 is an exact
  // FP32 integer below 2^23 (the 2^23 shift trick), scaled by 2^(E-46)
  const float mf = __uint_as_float(0x4B000000u | ((l & 0x1fffffffu) >> 6)) - 8388608.0f;
  const float sc = __uint_as_float(((ha >> 20) - 942u) << 23);
  const unsigned lb = __float_as_uint(mf * sc) | sgn;
  const unsigned hsel = big ? ((ha >= 0x7ff00000u) ? 0x7fc00000u : (0x67800000u | sgn)) : hb;
  hi = __uint_as_float(ok ? hsel : 0u);
  lo = __uint_as_float((ok && !big) ? lb : 0u);
}

// One term of a compensated dot product (Ogita, Rump & Oishi, SIAM J. Sci.
// Comput. 26 (2005), "Dot2"): (s, c) += (wh + wl)(ah + al).  The leading
// product is split exactly by an FMA and added to s by an error-free
// two-sum; the rounding errors and the cross terms wh al + wl ah go to c.
// The error-free steps use the _rn intrinsics, which the compiler never
// contracts into FMAs (a contracted s + wh ah would break the two-sum).
__device__ __forceinline__ void ff_dot_acc(float& s, float& c, float wh, float wl, float ah,
                                           float al) {
  const float p = __fmul_rn(wh, ah);
  const float pe = fmaf(wh, ah, -p);
  const float t = __fadd_rn(s, p);
  const float bb = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(p, bb));
  s = t;
  c += err + fmaf(wh, al, fmaf(wl, ah, pe));
}
// The first term of a dot product: (s, c) = (wh + wl)(ah + al).
__device__ __forceinline__ void ff_dot_first(float& s, float& c, float wh, float wl, float ah,
                                             float al) {
  s = __fmul_rn(wh, ah);
  c = fmaf(wh, al, fmaf(wl, ah, fmaf(wh, ah, -s)));
}

// s + c as a double, within one double ulp of |s + c|, on the FP32 and
// integer pipes: an error-free two-sum makes |r| <= 2^-24 |t| with
// t + r = s + c, then r's significand is shifted into the 53-bit
// significand of t (truncated below t's last double bit).  t = 0 (exact
// cancellation) or a subnormal t gives 0; a subnormal r is dropped; an
// infinite or NaN t gives NaN.
__device__ __forceinline__ double ff_to_double(float s, float c) {
  const float t = __fadd_rn(s, c);
  const float bb = __fsub_rn(t, s);
  const float r = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(c, bb));
  const unsigned tb = __float_as_uint(t), rb = __float_as_uint(r);
  const unsigned et = (tb >> 23) & 0xffu, er = (rb >> 23) & 0xffu;
  const unsigned long long B = (unsigned long long)((tb & 0x7fffffu) | 0x800000u) << 29;
  const unsigned d = et - er;   // >= 24 when r is normal and nonzero
  const unsigned long long Rm = (unsigned long long)((rb & 0x7fffffu) | 0x800000u) << 29;
  const unsigned long long Sm = (er == 0u || d > 52u) ? 0ull : (Rm >> d);
  unsigned long long R = ((tb ^ rb) >> 31) ? B - Sm : B + Sm;
  long long e = (long long)et + (1023 - 127);
  // only B = 2^52 minus a nonzero Sm (< 2^29) falls below 2^52: one shift
  const bool low = R < (1ull << 52);
  R = low ? (R << 1) : R;
  e = low ? e - 1 : e;
  const unsigned long long bits =
      ((unsigned long long)(tb >> 31) << 63) | ((unsigned long long)e << 52) | (R & ((1ull << 52) - 1));
  const double v = (et == 0xffu) ? __longlong_as_double(0x7ff8000000000000ll)
                                 : __longlong_as_double((long long)bits);
  return (et == 0u) ? 0.0 : v;
}

// A double constant as a float pair (compile time).
struct FFc {
  float hi, lo;
};
__host__ __device__ constexpr FFc make_ffc(double x) {
  return FFc{(float)x, (float)(x - (double)(float)x)};
}

}  // namespace
}  // namespace qcams
