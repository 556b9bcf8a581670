// The pair-force factor u = V'(r)/r of one pair at squared distance s, as
// the FP64 integrators form it (Sec. 3.2 potentials): the reciprocal square
// root and the exponential of elem64.cuh, 10 FP64 instructions for a Morse
// pair.  Shared by the one-thread-per-trajectory and the lane-group
// integrators.
#pragma once

#include <cuda_runtime.h>

#include "qcams_device.cuh"
#include "elem64.cuh"

namespace qcams {
namespace {

// The exponents' arguments take alpha r as (alpha s) (1/sqrt(s)): alpha s
// is formed while the reciprocal square root is refined, so the argument
// is one FP64 instruction after it instead of two (the same instruction
// count as forming r = s / sqrt(s) first).
template <bool MORSE>
__device__ __forceinline__ double pair_u(const DevPair& q, double s, const double* __restrict__ T) {
  float rf;   // FP32 estimate of r, for the exponential's table index
  const double ri = rsqrt_seeded(s, rf);
  if (MORSE) {
    // u = x (1 - x) / r, x = e^{-alpha (r - re)}; the factor 2 alpha De is in kf_morse
    const double as = q.c0 * s;
    const double x = texp_hint(fma(-as, ri, q.c1), fmaf(-q.ef0, rf, q.ef1), T);
    return fma(-x, x, x) * ri;
  }
  // generic kernels (mixed systems): u = V'(r)/r with the table exponential
  if (q.kind == QCAMS_MORSE) {
    const double as = q.c0 * s, c2ri = q.c2 * ri;
    const double x = texp_hint(fma(-as, ri, q.c1), fmaf(-q.ef0, rf, q.ef1), T);
    return fma(-x, x, x) * c2ri;
  }
  if (q.kind == QCAMS_BUCK) {
    // u = 6 C6 / r^8 - A B e^{-B r} / r, the exponential taking A B as the
    // offset ln(A B) of its argument: 9 FP64 instructions
    const double ri2 = ri * ri, ri4 = ri2 * ri2, bs = q.c1 * s;
    const double ex = texp_hint(fma(-bs, ri, q.lc2), fmaf(-q.ef0, rf, q.ef1), T);
    return fma(q.c3, ri4 * ri4, -(ex * ri));
  }
  return pot_g(q, ri, s * ri);
}

}  // namespace
}  // namespace qcams
