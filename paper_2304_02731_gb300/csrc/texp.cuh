// Table-driven FP64 exponential shared by the integrator and the product
// analysis.  Each translation unit that includes this header gets its own
// copy of the 16 KB table (internal linkage); kernels stage it in shared
// memory (__shared__ double sT[kExpTableSize]) with load_exp_table before
// the first texp call.
#pragma once

#include <cuda_runtime.h>

namespace qcams {
namespace {

#include "exp2_table.inc"

// e^x by Tang's table-driven method (P. T. P. Tang, ACM Trans. Math. Softw.
// 15 (1989) 144-157) with N = 2048: x = (N m + j) ln2/N + r, |r| <= ln2/(2N),
// then e^x = 2^m 2^(j/N) e^r with e^r - 1 = r + r^2/2 + r^3/6 (truncation
// r^4/24 < 3.5e-17 relative).  8 FP64 instructions.  Arguments below -700
// (e^x < 1e-304, far below any force term) give 2^-1010, chosen on the
// integer pipe from the high word; the caller guarantees x < 700.
__device__ __forceinline__ double texp(double x, const double* __restrict__ T) {
  const double kShift = 6755399441055744.0;  // 1.5 * 2^52: rounds to an integer
  const double t = fma(x, kExpInvL, kShift);
  const int k = __double2loint(t);
  const double kd = t - kShift;
  double r = fma(-kd, kExpL1, x);
  r = fma(-kd, kExpL2, r);
  double q = fma(r, 1.0 / 6.0, 0.5);
  q = q * r;
  const double p = fma(q, r, r);
  const double Tj = T[k & (kExpTableSize - 1)];
  const double y = fma(Tj, p, Tj);
  const double e = __hiloint2double(__double2hiint(y) + ((k >> 11) << 20), __double2loint(y));
  // high word above that of -700 as unsigned: x < -700, -inf or a negative NaN
  return ((unsigned)__double2hiint(x) > 0xC085E000u) ? 0x1.0p-1010 : e;
}

// Copies the table (16 KB) into shared memory (all threads of the block
// must call it: it ends with a barrier).
__device__ __forceinline__ void load_exp_table(double* sT) {
  for (int k = threadIdx.x; k < kExpTableSize; k += blockDim.x) sT[k] = kExp2Table[k];
  __syncthreads();
}

}  // namespace
}  // namespace qcams
