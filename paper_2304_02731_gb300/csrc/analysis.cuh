// Product analysis of finished trajectories (Sec. 2.2-2.3) and the
// root-finding / quadrature machinery it shares with the Bohr-Sommerfeld
// level solver.  Included by the translation units that launch it: the
// stand-alone analysis kernel (api.cu) and the FP32 integrator, which
// analyses its own finished lanes (integrate32.cu).  Everything here has
// internal linkage, so each including unit gets its own copy of the
// constant tables.
#pragma once

#include <cuda_runtime.h>

#include "qcams.h"
#include "qcams_device.cuh"
#include "texp.cuh"

namespace qcams {
namespace {

constexpr double kPi = 3.14159265358979323846;

// Gauss-Legendre rules in the sine-mapped variable (positive half of the
// symmetric nodes, written by gen_gl_tables.py): 48 points for the per-lane
// action integral, 128 for the level solver.  Compile-time constants, so
// every entry point can use them without a context.
constexpr int kGL48 = 48, kGL128 = 128;
#include "gl_tables.inc"

// Potentials with the exponential taken either from CUDA's exp (TAB =
// false: level solver) or from the shared-memory table T (TAB = true:
// product analysis, one table-driven exp per evaluation).
template <bool TAB>
__device__ __forceinline__ double pot_V_(const DevPair& q, double r, const double* T) {
  if (!TAB || q.kind == QCAMS_LJ) return pot_V(q, r);
  if (q.kind == QCAMS_MORSE) {
    const double u = 1.0 - texp(q.c1 - q.c0 * r, T);
    return q.c3 * u * u - q.c3;
  }
  const double ri = 1.0 / r, ri2 = ri * ri;
  return q.c0 * texp(-q.c1 * r, T) - q.c4 * ri2 * ri2 * ri2;
}
template <bool TAB>
__device__ __forceinline__ double pot_dV_(const DevPair& q, double r, const double* T) {
  if (!TAB || q.kind == QCAMS_LJ) return pot_dV(q, r);
  if (q.kind == QCAMS_MORSE) {
    const double x = texp(q.c1 - q.c0 * r, T);
    return q.c2 * x * (1.0 - x);
  }
  const double ri = 1.0 / r, ri2 = ri * ri;
  return q.c3 * ri2 * ri2 * ri2 * ri - q.c2 * texp(-q.c1 * r, T);
}
// V_eff = V + L2/(2 mu r^2); the centrifugal term from 1/r^2 = rsqrt(r^2)^2
// (no division in the root-search loops).
template <bool TAB>
__device__ __forceinline__ double veff_(const DevPair& q, double mu, double L2, double r,
                                        const double* T) {
  const double ri = rsqrt(r * r);
  return pot_V_<TAB>(q, r, T) + (0.5 * L2 / mu) * (ri * ri);
}
template <bool TAB>
__device__ __forceinline__ double gfun_(const DevPair& q, double r, const double* T) {
  return r * r * r * pot_dV_<TAB>(q, r, T);
}

// Outer barrier of the effective potential V + L2/(2 mu r^2): the root
// r_top > r_peak of g(r) = L2/mu and the threshold V_eff(r_top).  r_top =
// +inf and threshold 0 when L2 = 0 or when the barrier lies beyond reach.
// Returns false when L2/mu >= g_max (no well).
template <bool TAB>
__device__ bool barrier_top(const DevPair& q, const DevShape& sh, double mu, double L2,
                            const double* T, double* r_top, double* thr) {
  if (L2 <= 0.0) {
    *r_top = INFINITY;
    *thr = 0.0;
    return true;
  }
  const double c = L2 / mu;
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
  *r_top = illinois(G, a, b, G(a), gb);
  *thr = veff_<TAB>(q, mu, L2, *r_top, T);
  return true;
}

// Well of the effective potential: bottom r_min and outer barrier (r_top,
// threshold).  Returns false when L2/mu >= g_max (no well).
__device__ bool eff_well(const DevPair& q, const DevShape& sh, double mu, double L2,
                         double* r_min, double* r_top, double* thr) {
  if (!barrier_top<false>(q, sh, mu, L2, nullptr, r_top, thr)) return false;
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
__device__ bool turning_points(const DevPair& q, const DevShape& sh, double mu, double L2, double E,
                               double r_in, double r_top, const double* T, double* rm,
                               double* rp) {
  auto f = [&](double r) { return veff_<TAB>(q, mu, L2, r, T) - E; };
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
  *rm = illinois(f, lo, r_in, flo, fin);
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
  *rp = illinois(f, r_in, hi, fin, fhi);
  return true;
}

// Action and period integrals by Gauss-Legendre in s after r = c + d sin(s)
// (the mapped integrands are smooth on the closed interval):
//   I_act = int sqrt(E - V_eff) dr,  I_per = int dr / sqrt(E - V_eff).
// The node sines and the weights times the map's cosine are tabulated.
// PERIOD = false skips the period sum (the product analysis needs only the
// action).
template <int NG, bool TAB, bool PERIOD>
__device__ void action_period(const DevPair& q, double mu, double L2, double E, double rm,
                              double rp, const double* T, double* act, double* per) {
  const double c = 0.5 * (rp + rm), d = 0.5 * (rp - rm);
  const double a = L2 / (2.0 * mu);
  double sa = 0.0, sp = 0.0;
#pragma unroll 4
  for (int k = 0; k < NG / 2; ++k) {
    const double sn = (NG == kGL48) ? kGL48S[k] : kGL128S[k];
    const double wc = (NG == kGL48) ? kGL48WC[k] : kGL128WC[k];
#pragma unroll
    for (int sgn = 0; sgn < 2; ++sgn) {
      const double r = sgn ? fma(-d, sn, c) : fma(d, sn, c);
      const double ri = rsqrt(r * r);   // 1/r and sqrt(g) from reciprocal square roots
      const double g = E - (pot_V_<TAB>(q, r, T) + a * ri * ri);
      if (g > 0.0) {
        const double rg = rsqrt(g);
        sa = fma(wc, g * rg, sa);
        if (PERIOD) sp = fma(wc, rg, sp);
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
__device__ bool pair_bound(const DevPair& q, const DevShape& sh, double mu, double L2, double E,
                           double r, const double* T, double* r_top) {
  *r_top = INFINITY;
  if (!sh.ok || E >= L2 / (2.0 * mu * sh.r_peak * sh.r_peak)) return false;
  if (!(L2 / mu < sh.g_max)) return false;
  if (r > sh.r_peak && gfun_<true>(q, r, T) < L2 / mu) return false;
  double thr;
  if (!barrier_top<true>(q, sh, mu, L2, T, r_top, &thr)) return false;
  bool b = E < thr && r < *r_top;
  if (q.kind == QCAMS_BUCK) b = b && r > sh.r_b && E < veff_<true>(q, mu, L2, sh.r_b, T);
  return b;
}

// Product analysis of lane i: energy error, arrangement class by the unique
// bound pair, j' from its angular momentum, v' from its action (Eq. 10), the
// integer bins and the Gaussian-binning weight (Sec. 2.2-2.3).
// T: the exponential table staged in shared memory.
__device__ void analyze_lane(const SysSet& sys, const DevShape* shapes, double gb_sigma,
                             const DevBatch& B, int64_t i, const double* __restrict__ sT) {
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
      d[k] = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
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
        bd[k] = pair_bound(S.pair[k], shapes[sid * 3 + k], S.mu_pair[k], L2p[k], Ep[k], d[k], sT,
                           &rtop[k]);
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
        const DevPair& q = S.pair[which];
        const DevShape sh = shapes[sid * 3 + which];
        double r_in = r;
        if (!(veff_<true>(q, mu, L2, r, sT) < E)) {
          // at a turning point within rounding: split at the well bottom
          double rmin, rt, thr;
          if (!eff_well(q, sh, mu, L2, &rmin, &rt, &thr)) rmin = sh.r_eq;
          r_in = rmin;
        }
        double rm, rp, act, per;
        vp = -0.5;
        if (turning_points<true>(q, sh, mu, L2, E, r_in, r_top, sT, &rm, &rp)) {
          action_period<kGL48, true, false>(q, mu, L2, E, rm, rp, sT, &act, &per);
          vp = -0.5 + sqrt(2.0 * mu) / kPi * act;
        }
        jp = -0.5 + 0.5 * sqrt(1.0 + 4.0 * L2);
        vt = (int)floor(vp + 0.5);
        if (vt < 0) vt = 0;
        jt = (int)floor(jp + 0.5);
        const double dv = vp - vt;
        w = exp(-dv * dv / (2.0 * gb_sigma * gb_sigma)) / (gb_sigma * sqrt(2.0 * kPi));
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
