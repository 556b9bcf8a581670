// Device-side data structures and arithmetic shared by the QCT kernels.
//
// Physics: Koots & Perez-Rios, PyQCAMS (Comput. Phys. Commun.).  Pair
// potentials follow Sec. 3.2 items 1-3; Jacobi coordinates and reduced
// masses follow Sec. 2 (Eq. 2 and the definitions below it).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "qcams.h"

namespace qcams {

// ---------------------------------------------------------------------------
// Per-system constants, passed to every kernel by value (they live in the
// kernel-parameter constant bank, so warp-uniform reads are free).
// ---------------------------------------------------------------------------
struct DevPair {
  int32_t kind;   // QCAMS_MORSE / QCAMS_LJ / QCAMS_BUCK
  int32_t m, n;   // LJ exponents (integers)
  int32_t pad;
  double p[5];    // raw parameters (qcams_pair.p)
  // derived coefficients (set up on the host from p):
  //   Morse: c0 = alpha, c1 = alpha re, c2 = 2 alpha De, c3 = De
  //   LJ:    c0 = Cm, c1 = Cn, c2 = m Cm, c3 = n Cn
  //   Buck:  c0 = A, c1 = B, c2 = A B, c3 = 6 C6, c4 = C6
  double c0, c1, c2, c3, c4;
  double r_scale;  // a length near the well (root-search brackets)
  // FP32 copies of the exponent's coefficients, for the FP32 estimate of the
  // argument that the integrator's exponential rounds to its table index:
  //   Morse: ef0 = alpha, ef1 = alpha re (x = ef1 - ef0 r)
  //   Buck:  ef0 = B, ef1 = ln(A B) (x = ln(A B) - B r: the exponential
  //          returns A B e^{-B r} directly)
  float ef0, ef1;
  double lc2;     // Buck: ln(A B), the exponent's offset for A B e^{-B r}
  // c0..c4 rounded to FP32, for the FP32 root location of the product analysis
  float cf[5];
  int32_t pad2;
};

struct DevSys {
  double mu12, mu123;          // Jacobi reduced masses
  double inv_mu12, inv_mu123;
  double cA, cB;               // cA = mB/(mA+mB), cB = mA/(mA+mB)
  double mu_pair[3];           // reduced masses of the pairs AB, BC, CA
  double inv_mu_pair[3];       // their reciprocals
  double s2mu_pi[3];           // sqrt(2 mu_pair) / pi (Eq. 10's action-to-v' factor)
  DevPair pair[3];             // AB, BC, CA
  // Force coefficients: with u_k = V_k'(r_k)/r_k (generic) the accelerations
  // are a1 = kf[0] u0 r_AB + kf[1] u1 r_BC + kf[2] u2 r_CA and
  // a2 = kf[3] u1 r_BC + kf[4] u2 r_CA; kf_morse[] additionally folds the
  // Morse factor 2 alpha De, so that u_k = x(1 - x)/r with x = e^{-alpha(r-re)}.
  double kf[5];
  double kf_morse[5];
};

struct SysSet {
  DevSys s[QCAMS_MAX_SYS];
  int32_t n;
  int32_t pad;
};

// Shape of one pair potential, computed on the device once per call
// (kernel k_pair_shapes): beyond the well bottom r_eq, g(r) = r^3 V'(r)
// rises from 0 to a single maximum g_max at r_peak and decays to 0, so the
// effective potential V + L^2/(2 mu r^2) has a well and an outer barrier iff
// L^2/mu < g_max, at the two roots of g(r) = L^2/mu.
struct DevShape {
  double r_eq;     // minimum of V
  double r_peak;   // maximum of r^3 V'(r) beyond r_eq
  double g_max;    // r_peak^3 V'(r_peak)
  double r_b;      // Buckingham short-range maximum of V (0 for other kinds)
  double r_b2;     // r_b^2 (collapse test on squared distances)
  int32_t ok;
  int32_t pad;
};

struct DevLevel {
  double E, r_minus, r_plus, tau;
  int32_t ok;
  int32_t pad;
};

// Dense level table: [sys][v][j].
constexpr int kLevelV = QCAMS_V_MAX + 1;
constexpr int kLevelJ = QCAMS_J_MAX + 1;
constexpr int kLevelCells = QCAMS_MAX_SYS * kLevelV * kLevelJ;
__host__ __device__ inline int level_index(int s, int v, int j) {
  return (s * kLevelV + v) * kLevelJ + j;
}

// Batch pointers flattened for kernels (same meaning as qcams_batch).
struct DevBatch {
  int64_t n;
  const int32_t* sys_id;
  const int32_t* cell;
  const double* isw;
  double* y[12];
  double* t;
  double* h;
  double* t_scale;
  double* E0;
  double* Ecol;
  double* u[4];
  uint8_t* status;
  uint8_t* cls;
  int32_t* nsteps;
  int32_t* nrej;
  double* dE;
  double* vprime;
  double* jprime;
  double* gbw;
  int16_t* vt;
  int16_t* jt;
};

// ---------------------------------------------------------------------------
// Pair potentials (Sec. 3.2): V(r), V'(r).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double ipow(double x, int n) {
  // x^n for 0 <= n <= 64 by binary exponentiation (n is warp-uniform)
  double r = 1.0;
  while (n) {
    if (n & 1) r *= x;
    x *= x;
    n >>= 1;
  }
  return r;
}

__device__ __forceinline__ double pot_V(const DevPair& q, double r) {
  if (q.kind == QCAMS_MORSE) {
    double x = exp(q.c1 - q.c0 * r);
    double u = 1.0 - x;
    return q.c3 * u * u - q.c3;
  }
  double ri = 1.0 / r;
  if (q.kind == QCAMS_LJ) return q.c0 * ipow(ri, q.m) - q.c1 * ipow(ri, q.n);
  double ri2 = ri * ri;
  return q.c0 * exp(-q.c1 * r) - q.c4 * ri2 * ri2 * ri2;
}

__device__ __forceinline__ double pot_dV(const DevPair& q, double r) {
  if (q.kind == QCAMS_MORSE) {
    double x = exp(q.c1 - q.c0 * r);
    return q.c2 * x * (1.0 - x);
  }
  double ri = 1.0 / r;
  if (q.kind == QCAMS_LJ) return (q.c3 * ipow(ri, q.n) - q.c2 * ipow(ri, q.m)) * ri;
  double ri2 = ri * ri;
  return q.c3 * ri2 * ri2 * ri2 * ri - q.c2 * exp(-q.c1 * r);
}

__device__ __forceinline__ double pot_d2V(const DevPair& q, double r) {
  if (q.kind == QCAMS_MORSE) {
    double x = exp(q.c1 - q.c0 * r);
    return q.c2 * q.c0 * x * (2.0 * x - 1.0);
  }
  double ri = 1.0 / r;
  if (q.kind == QCAMS_LJ)
    return ((q.m + 1.0) * q.c2 * ipow(ri, q.m) - (q.n + 1.0) * q.c3 * ipow(ri, q.n)) * ri * ri;
  double ri2 = ri * ri;
  return q.c2 * q.c1 * exp(-q.c1 * r) - 7.0 * q.c3 * ri2 * ri2 * ri2 * ri2;
}

// V'(r)/r from 1/r and r (the force factor of the pair, used by the RHS).
__device__ __forceinline__ double pot_g(const DevPair& q, double ri, double r) {
  if (q.kind == QCAMS_MORSE) {
    double x = exp(fma(-q.c0, r, q.c1));
    return q.c2 * x * (1.0 - x) * ri;
  }
  double ri2 = ri * ri;
  if (q.kind == QCAMS_LJ) {
    if (q.n == 6 && (q.m == 12 || q.m == 8)) {
      // LJ(12,6) and LJ(8,6) from shared powers of 1/r^2: 7 FP64
      // instructions instead of the 16 of two binary exponentiations
      const double ri4 = ri2 * ri2, ri6 = ri4 * ri2;
      const double h = q.m == 12 ? ri6 : ri4;
      return fma(q.c3, ri6, -q.c2 * (h * h)) * ri2;
    }
    return (q.c3 * ipow(ri, q.n) - q.c2 * ipow(ri, q.m)) * ri2;
  }
  double ri6 = ri2 * ri2 * ri2;
  return (q.c3 * ri6 * ri - q.c2 * exp(-q.c1 * r)) * ri;
}

__device__ __forceinline__ double veff(const DevPair& q, double mu, double L2, double r) {
  return pot_V(q, r) + L2 / (2.0 * mu * r * r);
}
__device__ __forceinline__ double dveff(const DevPair& q, double mu, double L2, double r) {
  return pot_dV(q, r) - L2 / (mu * r * r * r);
}
// g(r) = r^3 V'(r)
__device__ __forceinline__ double gfun(const DevPair& q, double r) {
  return r * r * r * pot_dV(q, r);
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): counter-based uniforms for the
// orientation angles and vibrational phase (Sec. 2.1).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__device__ __forceinline__ double u01(uint32_t w) {
  return (static_cast<double>(w) + 0.5) * 2.3283064365386962890625e-10;  // 2^-32
}

// ---------------------------------------------------------------------------
// Bracketed root finding (Illinois variant of regula falsi).  f(a), f(b)
// must differ in sign; returns the root to a relative width of ~4 ulp or
// after 100 iterations.
// ---------------------------------------------------------------------------
template <class F>
__device__ double illinois(F f, double a, double b, double fa, double fb) {
  int side = 0;
  for (int it = 0; it < 100; ++it) {
    double c = (fa * b - fb * a) / (fa - fb);
    if (!(c > fmin(a, b) && c < fmax(a, b))) c = 0.5 * (a + b);
    double fc = f(c);
    if (fc == 0.0) return c;
    if ((fc > 0) == (fb > 0)) {
      b = c; fb = fc;
      if (side == -1) fa *= 0.5;
      side = -1;
    } else {
      a = c; fa = fc;
      if (side == +1) fb *= 0.5;
      side = +1;
    }
    if (fabs(b - a) <= 4.0 * 2.220446049250313e-16 * fmax(fabs(a), fabs(b))) break;
  }
  return (fabs(fa) < fabs(fb)) ? a : b;
}

}  // namespace qcams
