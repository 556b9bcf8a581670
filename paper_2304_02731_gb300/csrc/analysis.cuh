// Product analysis of finished trajectories (Sec. 2.2-2.3) and the
// root-finding / quadrature machinery it shares with the Bohr-Sommerfeld
// level solver.  Included by the translation unit that launches both (api.cu).
// Everything here has internal linkage.
//
// Two arithmetic variants share the algorithms (TAB template argument):
//  * TAB = false, the level solver (a few hundred levels per call, cached):
//    CUDA's exp, FP64 Illinois root iterations, 128-point quadrature.
//  * TAB = true, the per-lane product analysis (every trajectory): the work
//    goes to the FP32 / integer pipes where 53 bits are not needed.  The
//    exponential is the integrator's table method with an FP32-rounded
//    index (3 FP64 instructions), 1/r an FP32 reciprocal finished by a
//    second-order FP64 series step (3), 1/sqrt an FP32 estimate finished in
//    float-float (2).  Roots are located by an FP32 Illinois iteration and
//    finished by FP64 Newton steps (two steps take the ~2^-21 FP32 root to
//    full precision); the bracket decisions stay FP64, and an FP64 Illinois
//    iteration takes over whenever a Newton iterate leaves the bracket or
//    does not converge.  The action integral uses a 32-point rule in the
//    sine-mapped variable (at the rounding floor of the action for the
//    studies' Morse and LJ wells, within 4e-11 in v' even 1e-8 below a
//    centrifugal barrier top).
#pragma once

#include <cuda_runtime.h>

#include "qcams.h"
#include "qcams_device.cuh"
#include "elem64.cuh"
#include "texp.cuh"

namespace qcams {
namespace {

constexpr double kPi = 3.14159265358979323846;

// Gauss-Legendre rules in the sine-mapped variable (positive half of the
// symmetric nodes, written by gen_gl_tables.py): 32 points for the per-lane
// action integral, 128 for the level solver.  Compile-time constants, so
// every entry point can use them without a context.
constexpr int kGL32 = 32, kGL128 = 128;
#include "gl_tables.inc"

// ---------------------------------------------------------------------------
// Conversions between FP64 and FP32 on the integer pipe (a conversion
// instruction would occupy the FP64 pipe).
// ---------------------------------------------------------------------------
// x rounded toward zero to FP32; |x| below 2^-126 gives +-0, |x| of 2^128
// and above (inf, NaN) gives +-inf.
__device__ __forceinline__ float f32_of(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned sg = hi & 0x80000000u, ha = hi & 0x7fffffffu;
  const unsigned b = __funnelshift_l(lo, ha - (896u << 20), 3);
  const unsigned m = ha < (897u << 20) ? 0u : (ha >= (1151u << 20) ? 0x7f800000u : b);
  return __uint_as_float(m | sg);
}
// f exactly as a double for normal f; zero and subnormals give 0, inf and
// NaN a finite 2^128-scale value (callers treat it as out of range).
__device__ __forceinline__ double f64_of(float f) {
  const unsigned b = __float_as_uint(f), sg = b & 0x80000000u, a = b & 0x7fffffffu;
  const double d = __hiloint2double((int)(((a >> 3) + (896u << 20)) | sg), (int)(a << 29));
  return a < 0x00800000u ? 0.0 : d;
}

// 1/r for r in the FP32 normal range: the FP32 hardware reciprocal y0
// (relative error e0 below 2^-22), e = 1 - r y0, y = y0 (1 + e + e^2):
// relative error e0^3 < 2^-66.  3 FP64 instructions.
__device__ __forceinline__ double rcp_seeded(double r, float rf) {
  float yf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(rf));
  const double y0 = f64_of(yf);
  const double e = fma(-r, y0, 1.0);
  return fma(y0, fma(e, e, e), y0);
}

// ---------------------------------------------------------------------------
// Potentials (Sec. 3.2 items 1-3).  The FP64 forms with the table
// exponential: V, V' and, on request, V'' at r, given 1/r (ri) and an FP32
// copy of r (rf) for the exponential's table index.
// ---------------------------------------------------------------------------
template <bool D2>
__device__ __forceinline__ void pot_tab(const DevPair& q, double r, double ri, float rf,
                                        const double* __restrict__ T, double* V, double* dV,
                                        double* d2V) {
  if (q.kind == QCAMS_MORSE) {
    // x = e^{-alpha (r - re)}: V = De x (x - 2), V' = 2 alpha De x (1 - x),
    // V'' = 2 alpha^2 De x (2x - 1)
    const double x = texp_hint(fma(-q.c0, r, q.c1), fmaf(-q.ef0, rf, q.ef1), T);
    *V = q.c3 * (x * (x - 2.0));
    *dV = q.c2 * fma(-x, x, x);
    if (D2) *d2V = (q.c2 * q.c0) * (x * fma(2.0, x, -1.0));
  } else if (q.kind == QCAMS_LJ) {
    const double rm = ipow(ri, q.m), rn = ipow(ri, q.n);
    *V = fma(q.c0, rm, -q.c1 * rn);
    *dV = fma(q.c3, rn, -q.c2 * rm) * ri;
    if (D2) *d2V = fma((q.m + 1.0) * q.c2, rm, -(q.n + 1.0) * q.c3 * rn) * (ri * ri);
  } else {
    const double ex = texp_hint(-q.c1 * r, -q.ef0 * rf, T);
    const double ri2 = ri * ri, ri6 = ri2 * ri2 * ri2;
    *V = fma(q.c0, ex, -q.c4 * ri6);
    *dV = fma(q.c3 * ri6, ri, -q.c2 * ex);
    if (D2) *d2V = fma(q.c2 * q.c1, ex, -7.0 * q.c3 * ri6 * ri2);
  }
}

// FP32 form of V_eff(r) - E (root location only: relative error ~1e-6).
__device__ __forceinline__ float ipowf_a(float x, int n) {
  float r = 1.0f;
  while (n) {
    if (n & 1) r *= x;
    x *= x;
    n >>= 1;
  }
  return r;
}
__device__ __forceinline__ float veffE_f(const DevPair& q, float a, float E, float r) {
  const float ri = __fdividef(1.0f, r);
  float V;
  if (q.kind == QCAMS_MORSE) {
    const float x = __expf(fmaf(-q.cf[0], r, q.cf[1]));
    V = q.cf[3] * (x * (x - 2.0f));
  } else if (q.kind == QCAMS_LJ) {
    V = q.cf[0] * ipowf_a(ri, q.m) - q.cf[1] * ipowf_a(ri, q.n);
  } else {
    const float ri2 = ri * ri;
    V = q.cf[0] * __expf(-q.cf[1] * r) - q.cf[4] * (ri2 * ri2 * ri2);
  }
  return fmaf(a, ri * ri, V) - E;
}
// FP32 form of g(r) - c = r^3 V'(r) - c.
__device__ __forceinline__ float gfunc_f(const DevPair& q, float c, float r) {
  const float ri = __fdividef(1.0f, r);
  float dV;
  if (q.kind == QCAMS_MORSE) {
    const float x = __expf(fmaf(-q.cf[0], r, q.cf[1]));
    dV = q.cf[2] * (x - x * x);
  } else if (q.kind == QCAMS_LJ) {
    dV = (q.cf[3] * ipowf_a(ri, q.n) - q.cf[2] * ipowf_a(ri, q.m)) * ri;
  } else {
    const float ri2 = ri * ri;
    dV = q.cf[3] * (ri2 * ri2 * ri2) * ri - q.cf[2] * __expf(-q.cf[1] * r);
  }
  return r * r * r * dV - c;
}

// ---------------------------------------------------------------------------
// Root location.  illinois_f: the Illinois iteration in FP32 to a bracket
// width of 2^-21 relative.  root_finish: from an FP64 bracket [a, b] with
// fa, fb of opposite signs, an FP32 Illinois root of f32, then two Newton
// steps on fd (FP64 value, derivative through *d1), the step f / f' taken
// in FP32 (its own relative error only scales the Newton error, which is
// already the square of the previous one).  If an iterate leaves the
// bracket, or the last step is not below 2^-30 of the root, the FP64
// Illinois iteration on f64 decides instead.
// ---------------------------------------------------------------------------
template <class F>
__device__ float illinois_f(F f, float a, float b, float fa, float fb) {
  int side = 0;
  for (int it = 0; it < 60; ++it) {
    float c = __fdividef(fa * b - fb * a, fa - fb);
    if (!(c > fminf(a, b) && c < fmaxf(a, b))) c = 0.5f * (a + b);
    const float fc = f(c);
    if (fc == 0.0f) return c;
    if ((fc > 0.0f) == (fb > 0.0f)) {
      b = c; fb = fc;
      if (side == -1) fa *= 0.5f;
      side = -1;
    } else {
      a = c; fa = fc;
      if (side == +1) fb *= 0.5f;
      side = +1;
    }
    if (fabsf(b - a) <= 4.8e-7f * fmaxf(fabsf(a), fabsf(b))) break;
  }
  return (fabsf(fa) < fabsf(fb)) ? a : b;
}

template <class F32, class FD, class F64>
__device__ double root_finish(F32 f32, FD fd, F64 f64, double a, double b, double fa, double fb) {
  const float af = f32_of(a), bf = f32_of(b);
  const float fa32 = f32(af), fb32 = f32(bf);
  if (!((fa32 > 0.0f) == (fa > 0.0) && (fb32 > 0.0f) == (fb > 0.0) &&
        (fa32 > 0.0f) != (fb32 > 0.0f)))
    return illinois(f64, a, b, fa, fb);
  double r = f64_of(illinois_f(f32, af, bf, fa32, fb32));
  const double lo = fmin(a, b), hi = fmax(a, b);
  float last = 0.0f;
  bool ok = r > lo && r < hi;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    double d1;
    const double f = fd(r, &d1);
    last = __fdividef(f32_of(f), f32_of(d1));
    const double rn = r - f64_of(last);
    ok = ok && rn > lo && rn < hi;
    r = rn;
  }
  ok = ok && fabsf(last) <= 9.3e-10f * f32_of(r);   // 2^-30
  return ok ? r : illinois(f64, a, b, fa, fb);
}

// Potentials with the exponential taken either from CUDA's exp (TAB =
// false: level solver) or from the shared-memory table T (TAB = true:
// product analysis).
template <bool TAB>
__device__ __forceinline__ double pot_V_(const DevPair& q, double r, const double* T) {
  if (!TAB) return pot_V(q, r);
  const float rf = f32_of(r);
  double V, dV;
  pot_tab<false>(q, r, rcp_seeded(r, rf), rf, T, &V, &dV, nullptr);
  return V;
}
// V_eff = V + L2/(2 mu r^2); inv_mu = 1/mu (used by TAB = true, which
// multiplies by host-computed reciprocals instead of dividing).
template <bool TAB>
__device__ __forceinline__ double veff_(const DevPair& q, double mu, double inv_mu, double L2,
                                        double r, const double* T) {
  if (!TAB) {
    const double ri = rsqrt(r * r);   // 1/r^2 from a reciprocal square root: no division
    return pot_V(q, r) + (0.5 * L2 / mu) * (ri * ri);
  }
  const float rf = f32_of(r);
  const double ri = rcp_seeded(r, rf);
  double V, dV;
  pot_tab<false>(q, r, ri, rf, T, &V, &dV, nullptr);
  return fma(0.5 * L2 * inv_mu, ri * ri, V);
}
// g(r) = r^3 V'(r)
template <bool TAB>
__device__ __forceinline__ double gfun_(const DevPair& q, double r, const double* T) {
  if (!TAB) return r * r * r * pot_dV(q, r);
  const float rf = f32_of(r);
  double V, dV;
  pot_tab<false>(q, r, rcp_seeded(r, rf), rf, T, &V, &dV, nullptr);
  return r * r * r * dV;
}

// Outer barrier of the effective potential V + L2/(2 mu r^2): the root
// r_top > r_peak of g(r) = L2/mu and the threshold V_eff(r_top).  r_top =
// +inf and threshold 0 when L2 = 0 or when the barrier lies beyond reach.
// Returns false when L2/mu >= g_max (no well).
template <bool TAB>
__device__ bool barrier_top(const DevPair& q, const DevShape& sh, double mu, double inv_mu,
                            double L2, const double* T, double* r_top, double* thr) {
  if (L2 <= 0.0) {
    *r_top = INFINITY;
    *thr = 0.0;
    return true;
  }
  const double c = TAB ? L2 * inv_mu : L2 / mu;
  if (!(c < sh.g_max)) return false;
  auto G = [&](double r) { return gfun_<TAB>(q, r, T) - c; };
  double a = sh.r_peak, b = 2.0 * sh.r_peak, gb = G(b);
  for (int it = 0; it < 60 && gb >= 0.0; ++it) {
    a = b;
    b *= 2.0;
    gb = G(b);
  }
  if (gb >= 0.0) {  // barrier beyond reach (vanishing L): threshold 0
    *r_top = INFINITY;
    *thr = 0.0;
    return true;
  }
  if (TAB) {
    const float cf = f32_of(c);
    auto G32 = [&](float r) { return gfunc_f(q, cf, r); };
    // G'(r) = r^2 (3 V'(r) + r V''(r))
    auto GD = [&](double r, double* d1) {
      const float rf = f32_of(r);
      double V, dV, d2V;
      pot_tab<true>(q, r, rcp_seeded(r, rf), rf, T, &V, &dV, &d2V);
      const double r2 = r * r;
      *d1 = r2 * fma(r, d2V, 3.0 * dV);
      return fma(r2 * r, dV, -c);
    };
    *r_top = root_finish(G32, GD, G, a, b, G(a), gb);
  } else {
    *r_top = illinois(G, a, b, G(a), gb);
  }
  *thr = veff_<TAB>(q, mu, inv_mu, L2, *r_top, T);
  return true;
}

// Well of the effective potential: bottom r_min and outer barrier (r_top,
// threshold).  Returns false when L2/mu >= g_max (no well).
__device__ bool eff_well(const DevPair& q, const DevShape& sh, double mu, double L2,
                         double* r_min, double* r_top, double* thr) {
  if (!barrier_top<false>(q, sh, mu, 0.0, L2, nullptr, r_top, thr)) return false;
  if (L2 <= 0.0) {
    *r_min = sh.r_eq;
    return true;
  }
  const double c = L2 / mu;
  auto G = [&](double r) { return gfun(q, r) - c; };
  *r_min = illinois(G, sh.r_eq, sh.r_peak, -c, sh.g_max - c);
  return true;
}

// Turning points of E = V_eff inside the well, bracketed by a split point
// r_in of the classically allowed region (V_eff(r_in) < E: the well bottom
// for the level solver, the pair's own separation in the analysis) and the
// barrier top.
template <bool TAB>
__device__ bool turning_points(const DevPair& q, const DevShape& sh, double mu, double inv_mu,
                               double L2, double E, double r_in, double r_top, const double* T,
                               double* rm, double* rp) {
  auto f = [&](double r) { return veff_<TAB>(q, mu, inv_mu, L2, r, T) - E; };
  double fin = f(r_in);
  if (!(fin < 0.0)) return false;
  // inner: V_eff rises steeply toward small r (Buckingham: up to r_b)
  double lo, flo;
  if (q.kind == QCAMS_BUCK) {
    lo = sh.r_b;
    flo = f(lo);
    if (!(flo > 0.0)) return false;
  } else {
    lo = 0.5 * r_in;
    flo = f(lo);
    for (int it = 0; it < 60 && flo <= 0.0; ++it) {
      lo *= 0.5;
      flo = f(lo);
    }
    if (!(flo > 0.0)) return false;
  }
  const double a2 = 0.5 * L2 * inv_mu;
  const float af = f32_of(a2), Ef = f32_of(E);
  auto f32 = [&](float r) { return veffE_f(q, af, Ef, r); };
  // f'(r) = V'(r) - 2 a / r^3
  auto fd = [&](double r, double* d1) {
    const float rf = f32_of(r);
    const double ri = rcp_seeded(r, rf), ri2 = ri * ri;
    double V, dV;
    pot_tab<false>(q, r, ri, rf, T, &V, &dV, nullptr);
    *d1 = fma(-2.0 * a2, ri2 * ri, dV);
    return fma(a2, ri2, V) - E;
  };
  *rm = TAB ? root_finish(f32, fd, f, lo, r_in, flo, fin) : illinois(f, lo, r_in, flo, fin);
  double hi, fhi;
  if (isfinite(r_top)) {
    hi = r_top;
    fhi = f(hi);
  } else {
    hi = 2.0 * r_in;
    fhi = f(hi);
    for (int it = 0; it < 60 && fhi <= 0.0; ++it) {
      hi *= 2.0;
      fhi = f(hi);
    }
  }
  if (!(fhi > 0.0)) return false;
  *rp = TAB ? root_finish(f32, fd, f, r_in, hi, fin, fhi) : illinois(f, r_in, hi, fin, fhi);
  return true;
}

// Action and period integrals by Gauss-Legendre in s after r = c + d sin(s)
// (the mapped integrands are smooth on the closed interval):
//   I_act = int sqrt(E - V_eff) dr,  I_per = int dr / sqrt(E - V_eff).
// The node sines and the weights times the map's cosine are tabulated.
// PERIOD = false skips the period sum (the product analysis needs only the
// action).  TAB = true evaluates the integrand with the table exponential,
// the seeded reciprocal and the seeded reciprocal square root (values of
// E - V_eff below 2^-126, where sqrt contributes below 1e-19, are dropped).
template <int NG, bool TAB, bool PERIOD>
__device__ void action_period(const DevPair& q, double mu, double inv_mu, double L2, double E,
                              double rm, double rp, const double* T, double* act, double* per) {
  const double c = 0.5 * (rp + rm), d = 0.5 * (rp - rm);
  const double a = TAB ? 0.5 * L2 * inv_mu : L2 / (2.0 * mu);
  double sa = 0.0, sp = 0.0;
#pragma unroll 4
  for (int k = 0; k < NG / 2; ++k) {
    const double sn = (NG == kGL32) ? kGL32S[k] : kGL128S[k];
    const double wc = (NG == kGL32) ? kGL32WC[k] : kGL128WC[k];
#pragma unroll
    for (int sgn = 0; sgn < 2; ++sgn) {
      const double r = sgn ? fma(-d, sn, c) : fma(d, sn, c);
      if (TAB) {
        const float rf = f32_of(r);
        const double ri = rcp_seeded(r, rf);
        double V, dV;
        pot_tab<false>(q, r, ri, rf, T, &V, &dV, nullptr);
        const double g = fma(-a, ri * ri, E) - V;
        if (g > 0x1.0p-126) {
          float gf;
          const double rg = rsqrt_seeded(g, gf);
          sa = fma(wc, g * rg, sa);
          if (PERIOD) sp = fma(wc, rg, sp);
        }
      } else {
        const double ri = rsqrt(r * r);   // 1/r and sqrt(g) from reciprocal square roots
        const double g = E - (pot_V(q, r) + a * ri * ri);
        if (g > 0.0) {
          const double rg = rsqrt(g);
          sa = fma(wc, g * rg, sa);
          if (PERIOD) sp = fma(wc, rg, sp);
        }
      }
    }
  }
  *act = 0.5 * kPi * d * sa;
  if (PERIOD) *per = 0.5 * kPi * d * sp;
}

// ---------------------------------------------------------------------------
// Product analysis (Sec. 2.2).
// ---------------------------------------------------------------------------
// Bound test of one pair (Sec. 2.2 with reading R13): E below the barrier
// threshold V_eff(r_top) and the pair inside its barrier (r < r_top; for
// Buckingham also outside the short-range maximum, r > r_b, and E below
// V_eff(r_b)).  Sets r_top for the turning-point search.  Two exact
// shortcuts skip the root search for unbound pairs:
//  * the barrier top lies beyond r_peak, where V < 0, so the threshold is
//    below L2/(2 mu r_peak^2): a pair at or above that energy is unbound;
//  * beyond r_peak, g(r) = r^3 V'(r) decreases through L2/mu exactly at
//    r_top (g is unimodal there), so g(r) < L2/mu at r > r_peak means
//    r > r_top: the pair is outside its barrier.
__device__ bool pair_bound(const DevPair& q, const DevShape& sh, double mu, double inv_mu,
                           double L2, double E, double r, const double* T, double* r_top) {
  *r_top = INFINITY;
  // E >= L2 / (2 mu r_peak^2), L2 / mu >= g_max and g(r) < L2 / mu, multiplied out
  if (!sh.ok || (2.0 * mu) * (sh.r_peak * sh.r_peak) * E >= L2) return false;
  if (!(L2 < sh.g_max * mu)) return false;
  if (r > sh.r_peak && gfun_<true>(q, r, T) * mu < L2) return false;
  double thr;
  if (!barrier_top<true>(q, sh, mu, inv_mu, L2, T, r_top, &thr)) return false;
  bool b = E < thr && r < *r_top;
  if (q.kind == QCAMS_BUCK) b = b && r > sh.r_b && E < veff_<true>(q, mu, inv_mu, L2, sh.r_b, T);
  return b;
}

// Product analysis of lane i: energy error, arrangement class by the unique
// bound pair, j' from its angular momentum, v' from its action (Eq. 10), the
// integer bins and the Gaussian-binning weight (Sec. 2.2-2.3).
// T: the exponential table staged in shared memory.
// gb_c1 = 1 / (2 sigma^2) and gb_c2 = 1 / (sigma sqrt(2 pi)) of the
// Gaussian-binning width sigma (host-computed).
__device__ void analyze_lane(const SysSet& sys, const DevShape* shapes, double gb_c1,
                             double gb_c2, const DevBatch& B, int64_t i,
                             const double* __restrict__ sT) {
  const int st = B.status[i];
  const int sid = B.sys_id[i];
  int cls = QCAMS_CLS_FAIL;
  double vp = 0.0, jp = 0.0, w = 0.0, dE = 0.0;
  int vt = 0, jt = 0;
  if (sid >= 0 && sid < sys.n && st != QCAMS_LANE_NO_LEVEL && st != QCAMS_LANE_INVALID) {
    const DevSys& S = sys.s[sid];
    double y[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) y[k] = B.y[k][i];
    // pair separations, energies and squared angular momenta; their
    // potentials also give the total energy (Eq. 2)
    double d[3], Ep[3], L2p[3], Vsum = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double ck = k == 0 ? 0.0 : (k == 1 ? -S.cB : S.cA);
      const double fk = k == 0 ? 0.0 : 1.0;
      double r[3], v[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double v1 = y[6 + a] * S.inv_mu12, v2 = y[9 + a] * S.inv_mu123;
        r[a] = k == 0 ? y[a] : fma(ck, y[a], y[3 + a]);
        v[a] = k == 0 ? v1 : fma(ck, v1, fk * v2);
      }
      const double mu = S.mu_pair[k];
      const double s2 = fma(r[0], r[0], fma(r[1], r[1], r[2] * r[2]));
      float rf;
      d[k] = s2 * rsqrt_seeded(s2, rf);
      // pairs beyond the FP32 range of r^2 (never met) fall back to sqrt
      if (!(d[k] == d[k])) d[k] = sqrt(s2);
      const double V = pot_V_<true>(S.pair[k], d[k], sT);
      Vsum += V;
      const double Lx = r[1] * v[2] - r[2] * v[1];
      const double Ly = r[2] * v[0] - r[0] * v[2];
      const double Lz = r[0] * v[1] - r[1] * v[0];
      Ep[k] = 0.5 * mu * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) + V;
      L2p[k] = mu * mu * (Lx * Lx + Ly * Ly + Lz * Lz);
    }
    const double Tkin = (y[6] * y[6] + y[7] * y[7] + y[8] * y[8]) * (0.5 * S.inv_mu12) +
                        (y[9] * y[9] + y[10] * y[10] + y[11] * y[11]) * (0.5 * S.inv_mu123);
    dE = (Tkin + Vsum) - B.E0[i];
    if (st == QCAMS_LANE_DONE_RSTOP || st == QCAMS_LANE_DONE_TMAX) {
      bool bd[3];
      double rtop[3];
#pragma unroll
      for (int k = 0; k < 3; ++k)
        bd[k] = pair_bound(S.pair[k], shapes[sid * 3 + k], S.mu_pair[k], S.inv_mu_pair[k],
                           L2p[k], Ep[k], d[k], sT, &rtop[k]);
      const int nb = (int)bd[0] + (int)bd[1] + (int)bd[2];
      if (nb == 0) {
        cls = QCAMS_CLS_D;
      } else if (nb > 1) {
        cls = QCAMS_CLS_AMBIG;
      } else {
        // the bound pair's quantities by selects (no dynamic register indexing)
        const int which = bd[0] ? 0 : (bd[1] ? 1 : 2);
        cls = which == 0 ? QCAMS_CLS_Q : which == 2 ? QCAMS_CLS_R_AC : QCAMS_CLS_R_BC;
        const double E = bd[0] ? Ep[0] : (bd[1] ? Ep[1] : Ep[2]);
        const double L2 = bd[0] ? L2p[0] : (bd[1] ? L2p[1] : L2p[2]);
        const double r = bd[0] ? d[0] : (bd[1] ? d[1] : d[2]);
        const double r_top = bd[0] ? rtop[0] : (bd[1] ? rtop[1] : rtop[2]);
        const double mu = S.mu_pair[which];
        const double inv_mu = S.inv_mu_pair[which];
        const DevPair& q = S.pair[which];
        const DevShape sh = shapes[sid * 3 + which];
        double r_in = r;
        if (!(veff_<true>(q, mu, inv_mu, L2, r, sT) < E)) {
          // at a turning point within rounding: split at the well bottom
          double rmin, rt, thr;
          if (!eff_well(q, sh, mu, L2, &rmin, &rt, &thr)) rmin = sh.r_eq;
          r_in = rmin;
        }
        double rm, rp, act, per;
        vp = -0.5;
        if (turning_points<true>(q, sh, mu, inv_mu, L2, E, r_in, r_top, sT, &rm, &rp)) {
          action_period<kGL32, true, false>(q, mu, inv_mu, L2, E, rm, rp, sT, &act, &per);
          vp = fma(S.s2mu_pi[which], act, -0.5);   // sqrt(2 mu) / pi * act - 1/2
        }
        {  // j' (j' + 1) = L2: j' = (sqrt(1 + 4 L2) - 1) / 2
          const double s4 = fma(4.0, L2, 1.0);
          float sf;
          double sq = s4 * rsqrt_seeded(s4, sf);
          if (!(sq == sq)) sq = sqrt(s4);
          jp = fma(0.5, sq, -0.5);
        }
        vt = (int)floor(vp + 0.5);
        if (vt < 0) vt = 0;
        jt = (int)floor(jp + 0.5);
        const double dv = vp - vt;
        w = gb_c2 * texp(-(dv * dv) * gb_c1, sT);
      }
    }
  }
  B.cls[i] = (uint8_t)cls;
  B.vprime[i] = vp;
  B.jprime[i] = jp;
  B.gbw[i] = w;
  B.vt[i] = (int16_t)(vt > 32767 ? 32767 : vt);
  B.jt[i] = (int16_t)(jt > 32767 ? 32767 : jt);
  B.dE[i] = dE;
}

}  // namespace
}  // namespace qcams
