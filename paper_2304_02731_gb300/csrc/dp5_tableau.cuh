// Dormand & Prince 5(4) tableau and the Runge-Kutta-Nystrom coefficient
// products the integrators use, evaluated at compile time.  Shared by the
// FP64 (integrate.cu) and FP32 (integrate32.cu) integrators.
#pragma once

namespace qcams {

// ---------------------------------------------------------------------------
// Dormand & Prince (1980) 5(4) tableau (1-based stage indices) and the
// Runge-Kutta-Nystrom coefficient products derived from it at compile time.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr double dpA(int i, int j) {
  return (i == 2 && j == 1)   ? 1.0 / 5
         : (i == 3 && j == 1) ? 3.0 / 40
         : (i == 3 && j == 2) ? 9.0 / 40
         : (i == 4 && j == 1) ? 44.0 / 45
         : (i == 4 && j == 2) ? -56.0 / 15
         : (i == 4 && j == 3) ? 32.0 / 9
         : (i == 5 && j == 1) ? 19372.0 / 6561
         : (i == 5 && j == 2) ? -25360.0 / 2187
         : (i == 5 && j == 3) ? 64448.0 / 6561
         : (i == 5 && j == 4) ? -212.0 / 729
         : (i == 6 && j == 1) ? 9017.0 / 3168
         : (i == 6 && j == 2) ? -355.0 / 33
         : (i == 6 && j == 3) ? 46732.0 / 5247
         : (i == 6 && j == 4) ? 49.0 / 176
         : (i == 6 && j == 5) ? -5103.0 / 18656
         : (i == 7 && j == 1) ? 35.0 / 384
         : (i == 7 && j == 3) ? 500.0 / 1113
         : (i == 7 && j == 4) ? 125.0 / 192
         : (i == 7 && j == 5) ? -2187.0 / 6784
         : (i == 7 && j == 6) ? 11.0 / 84
                              : 0.0;
}
__host__ __device__ constexpr double dpC(int i) {
  return i == 2 ? 1.0 / 5 : i == 3 ? 3.0 / 10 : i == 4 ? 4.0 / 5 : i == 5 ? 8.0 / 9
         : (i >= 6) ? 1.0 : 0.0;
}
// 5th-order weights b = 7th row of A (FSAL); error weights e = b - b*.
__host__ __device__ constexpr double dpB(int j) { return dpA(7, j); }
__host__ __device__ constexpr double dpE(int j) {
  return j == 1 ? 71.0 / 57600 : j == 3 ? -71.0 / 16695 : j == 4 ? 71.0 / 1920
         : j == 5 ? -17253.0 / 339200 : j == 6 ? 22.0 / 525 : j == 7 ? -1.0 / 40 : 0.0;
}
__host__ __device__ constexpr double dpA2(int s, int q) {
  double acc = 0.0;
  for (int j = 1; j <= 7; ++j) acc += dpA(s, j) * dpA(j, q);
  return acc;
}
__host__ __device__ constexpr double dpEA(int q) {
  double acc = 0.0;
  for (int i = 1; i <= 7; ++i) acc += dpE(i) * dpA(i, q);
  return acc;
}

// Entries of A^2 and e^T A that are zero in exact arithmetic.  (A^2)_{s,q}
// needs q < j < s, so it vanishes for q >= s - 1.  (A^2)_{7,2} = sum_j b_j a_j2
// = b_2 (1 - c_2) = 0, since the last row of A is b and the tableau satisfies
// sum_i b_i a_ij = b_j (1 - c_j); (e^T A)_2 = 0 as well (both checked in
// rational arithmetic).  The double sums above leave rounding residues of
// about 1e-16 there, so the tables store exact zeros and the integrators
// skip those terms at compile time.
__host__ __device__ constexpr bool dpA2Zero(int s, int q) { return q >= s - 1 || (s == 7 && q == 2); }
__host__ __device__ constexpr bool dpEAZero(int q) { return q == 2 || q >= 7; }
static_assert(dpA2(7, 2) < 1e-15 && dpA2(7, 2) > -1e-15, "(A^2)_{7,2} is a rounding residue");
static_assert(dpEA(2) < 1e-15 && dpEA(2) > -1e-15, "(e^T A)_2 is a rounding residue");
static_assert(dpA2(7, 1) > 0.09 && dpEA(3) < -6e-3, "nonzero neighbours stay nonzero");

struct RknTab {
  double a2[8][8];  // (A^2)_{s,q}, s,q 1-based
  double c[8];
  double b[8];
  double e[8];
  double ea[8];     // (e^T A)_q
};
__host__ __device__ constexpr RknTab make_rkn_tab() {
  RknTab t{};
  for (int s = 1; s <= 7; ++s) {
    t.c[s] = dpC(s);
    t.b[s] = dpB(s);
    t.e[s] = dpE(s);
    t.ea[s] = dpEAZero(s) ? 0.0 : dpEA(s);
    for (int q = 1; q <= 7; ++q) t.a2[s][q] = dpA2Zero(s, q) ? 0.0 : dpA2(s, q);
  }
  return t;
}


}  // namespace qcams
