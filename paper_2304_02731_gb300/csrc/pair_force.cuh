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

template <bool MORSE>
__device__ __forceinline__ double pair_u(const DevPair& q, double s, const double* __restrict__ T) {
  float rf;   // FP32 estimate of r, for the exponential's table index
  const double ri = rsqrt_seeded(s, rf);
  const double r = s * ri;
  if (MORSE) {
    // u = x (1 - x) / r, x = e^{-alpha (r - re)}; the factor 2 alpha De is in kf_morse
    const double x = texp_hint(fma(-q.c0, r, q.c1), fmaf(-q.ef0, rf, q.ef1), T);
    return fma(-x, x, x) * ri;
  }
  // generic kernels (mixed systems): u = V'(r)/r with the table exponential
  if (q.kind == QCAMS_MORSE) {
    const double x = texp_hint(fma(-q.c0, r, q.c1), fmaf(-q.ef0, rf, q.ef1), T);
    return q.c2 * fma(-x, x, x) * ri;
  }
  if (q.kind == QCAMS_BUCK) {
    // u = 6 C6 / r^8 - A B e^{-B r} / r, the exponential taking A B as the
    // offset ln(A B) of its argument: 9 FP64 instructions
    const double ri2 = ri * ri, ri4 = ri2 * ri2;
    const double ex = texp_hint(fma(-q.c1, r, q.lc2), fmaf(-q.ef0, rf, q.ef1), T);
    return fma(q.c3, ri4 * ri4, -(ex * ri));
  }
  return pot_g(q, ri, r);
}

}  // namespace
}  // namespace qcams
