// Trajectory integrator: Hamilton's equations (Sec. 2, Eqs. 3-4) in Jacobi
// coordinates, one trajectory per thread, Dormand-Prince 5(4) with a
// per-lane adaptive step (Sec. 3.2: SciPy's solve_ivp RK45 step control).
//
// GB300 design:
//  * The state (12 doubles) and the stage derivatives live in registers;
//    global memory is touched only to load a lane and to store it back.
//  * Runge-Kutta-Nystrom form.  Since d(rho)/dt = P/mu depends on P only,
//    every stage position of the classical method can be written with the
//    stage accelerations alone:
//        rho_s = rho + h c_s v + h^2 sum_q (A^2)_{sq} a_q ,   v = P/mu,
//    and the 5th-order update and the embedded error likewise use b^T A and
//    e^T A.  This is algebraically the same method as the 12-dimensional
//    Dormand-Prince step, with 6 (not 12) stored values per stage.
//  * The three pair distances of the last stage (FSAL, the new state) are
//    reused by the stop test, so the test costs no extra square roots.
//  * Step acceptance is a select, not a branch: all lanes of a warp run the
//    same instruction stream; only retirement diverges.
//  * Persistent mode: a finished lane takes the next trajectory index from a
//    device counter, with one atomicAdd per warp for all lanes that need
//    work (ballot + popc), so warps stay full until the queue drains.
//  * GB300 issues one warp-wide FP64 instruction per 64 cycles per SM
//    sub-partition (1/64 of the FP32 rate), so the kernel is bound by the
//    number of FP64-pipe instructions per step.  Everything that does not
//    need 53-bit arithmetic runs on the integer / FP32 pipes: the step-size
//    controller's error norm (magnitudes taken from the doubles' exponent and
//    leading mantissa bits, ratios in FP32), the stop tests (integer compares
//    of non-negative doubles) and the minimum-step test (exponent compare).
//  * Each pair force takes 1/sqrt(s) and e^x (elem64.cuh), 3 FP64
//    instructions each: the reciprocal square root is an FP32 hardware
//    estimate finished in FP64; the exponential is Tang's table method (a
//    2048-entry table of 2^(j/2048) in shared memory, the table index
//    rounded in FP32, the quadratic and cubic terms in float-float).
//  * Stages 6 and 7 (c = 1) share rho + h v, and the tableau entries that are
//    zero in exact arithmetic are skipped at compile time.
//  * Linear combinations that do not need an FP64 result run as float-float
//    compensated dot products on the FP32 / integer pipes (ff.cuh): the
//    acceleration corrections of stages 4-6 (one DADD each onto the FP64
//    base) and the embedded error estimate.  The new state (stage 7, v_n+1)
//    keeps its FP64 sums.
#include <cuda_runtime.h>

#include "qcams_device.cuh"
#include "qcams_internal.h"
#include "dp5_tableau.cuh"
#include "elem64.cuh"
#include "ff.cuh"
#include "step_ctrl.cuh"
#include "pair_force.cuh"

namespace qcams {
namespace {

// Coefficients in the constant bank: a DFMA takes a constant-bank operand at
// full rate, so indexing this table with compile-time indices costs nothing.
__constant__ RknTab kT = make_rkn_tab();

// The coefficients of the float-float sums as float pairs.
__constant__ RknTabFF kTff = make_rkn_tab_ff();

constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------------------
// Accelerations a = (dP1/dt / mu12, dP2/dt / mu123) at Jacobi positions x,
// and the squared pair distances (AB, BC, CA).
//   r_AB = rho1,  r_BC = rho2 - cB rho1,  r_CA = rho2 + cA rho1
//   dV/drho1 = g_AB r_AB - cB g_BC r_BC + cA g_CA r_CA,
//   dV/drho2 = g_BC r_BC + g_CA r_CA,          g = V'(r)/r.
// ---------------------------------------------------------------------------
template <bool MORSE>
__device__ __forceinline__ void accel(const DevSys& S, const double* __restrict__ T,
                                      const double* x, double* a, double* s2) {
  const double rab0 = x[0], rab1 = x[1], rab2 = x[2];
  const double rbc0 = fma(-S.cB, x[0], x[3]), rbc1 = fma(-S.cB, x[1], x[4]),
               rbc2 = fma(-S.cB, x[2], x[5]);
  const double rca0 = fma(S.cA, x[0], x[3]), rca1 = fma(S.cA, x[1], x[4]),
               rca2 = fma(S.cA, x[2], x[5]);
  s2[0] = fma(rab0, rab0, fma(rab1, rab1, rab2 * rab2));
  s2[1] = fma(rbc0, rbc0, fma(rbc1, rbc1, rbc2 * rbc2));
  s2[2] = fma(rca0, rca0, fma(rca1, rca1, rca2 * rca2));
  const double u0 = pair_u<MORSE>(S.pair[0], s2[0], T);
  const double u1 = pair_u<MORSE>(S.pair[1], s2[1], T);
  const double u2 = pair_u<MORSE>(S.pair[2], s2[2], T);
  const double f0 = (MORSE ? S.kf_morse[0] : S.kf[0]) * u0;
  const double f1 = (MORSE ? S.kf_morse[1] : S.kf[1]) * u1;
  const double f2 = (MORSE ? S.kf_morse[2] : S.kf[2]) * u2;
  const double h1 = (MORSE ? S.kf_morse[3] : S.kf[3]) * u1;
  const double h2 = (MORSE ? S.kf_morse[4] : S.kf[4]) * u2;
  a[0] = fma(f0, rab0, fma(f1, rbc0, f2 * rca0));
  a[1] = fma(f0, rab1, fma(f1, rbc1, f2 * rca1));
  a[2] = fma(f0, rab2, fma(f1, rbc2, f2 * rca2));
  a[3] = fma(h1, rbc0, h2 * rca0);
  a[4] = fma(h1, rbc1, h2 * rca1);
  a[5] = fma(h1, rbc2, h2 * rca2);
}

// Position of stage s (1-based, s >= 2) from base = rho + h c_s v.
// The stage's coefficients h^2 (A^2)_{sq} are formed once per stage rather
// than scaling each component's sum by h^2 (6 multiplies); entries that are
// zero in exact arithmetic are skipped (stage 2 has no acceleration term).
template <int s>
__device__ __forceinline__ void stage_x(const double* base, const double (*acc)[6], double hh,
                                        double* x) {
  double w[s > 2 ? s - 2 : 1];
#pragma unroll
  for (int q = 1; q <= s - 2; ++q) w[q - 1] = dpA2Zero(s, q) ? 0.0 : hh * kT.a2[s][q];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    double xi = base[i];
#pragma unroll
    for (int q = 1; q <= s - 2; ++q)
      if (!dpA2Zero(s, q)) xi = fma(w[q - 1], acc[q - 1][i], xi);
    x[i] = xi;
  }
}
// The same for stages 2 and 3 (c_s < 1), forming rho + h c_s v per component.
template <int s>
__device__ __forceinline__ void stage_x(const double* rho, const double* vel, const double (*acc)[6],
                                        double h, double hh, double* x) {
  static_assert(s == 2 || s == 3, "stages 4-6 use stage_x_ff, 7 the FP64 form");
  const double hc = h * dpC(s);
  double base[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) base[i] = fma(hc, vel[i], rho[i]);
  stage_x<s>(base, acc, hh, x);
}

// Position of stage s = 4, 5, 6: base + h^2 sum_q (A^2)_{sq} a_q, the sum
// as a float-float compensated dot product (FP32 / integer pipes) added to
// the FP64 base with one DADD.  Its error, ~1e-13 h^2 |a|, reaches the step's
// result through the stage force only, damped by (h omega)^3 below the FP64
// rounding of the result; the 5th-order position (stage 7) and velocity
// keep FP64 sums.
template <int s>
__device__ __forceinline__ void stage_x_ff(const double* base, const double (*acc)[6], float hhh,
                                           float hhl, double* x) {
  static_assert(s >= 4 && s <= 6, "stages 4-6");
  float wh[s - 2], wl[s - 2];
#pragma unroll
  for (int q = 1; q <= s - 2; ++q) {
    const FFc c = kTff.a2[s][q];
    wh[q - 1] = __fmul_rn(hhh, c.hi);
    wl[q - 1] = fmaf(hhh, c.hi, -wh[q - 1]) + fmaf(hhh, c.lo, hhl * c.hi);
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    float sm, cm, ah, al;
    split_ff(acc[0][i], ah, al);
    ff_dot_first(sm, cm, wh[0], wl[0], ah, al);
#pragma unroll
    for (int q = 2; q <= s - 2; ++q) {
      split_ff(acc[q - 1][i], ah, al);
      ff_dot_acc(sm, cm, wh[q - 1], wl[q - 1], ah, al);
    }
    x[i] = base[i] + ff_to_double(sm, cm);
  }
}

// One Dormand-Prince step of size h from (rho, vel) with acc[0] = a(rho).
// On return acc[1..6] hold the stage accelerations, xn / vn the 5th-order
// solution (acc[6] = a(xn), FSAL), er / ev the embedded error estimates of
// positions and velocities divided by h^2 and h (the error norm applies
// those factors in FP32), s2 the squared pair distances at xn.
//
// The error estimates are sums of ~1e-9 |a| from terms of ~0.05 |a|; the
// FP32 norm needs them to about 20 bits, so they are float-float
// compensated dot products (relative error ~1e-6 where the norm is near 1,
// the level of the norm's own 20-bit magnitudes) rather than FP64 sums.
template <bool MORSE>
__device__ __forceinline__ void dp_step(const DevSys& S, const double* __restrict__ T,
                                        const double* rho, const double* vel, double (*acc)[6],
                                        double h, double* xn, double* vn, float* er, float* ev,
                                        double* s2) {
  const double hh = h * h;
  float hhh, hhl;
  split_ff(hh, hhh, hhl);
  double x[6];
  stage_x<2>(rho, vel, acc, h, hh, x);
  accel<MORSE>(S, T, x, acc[1], s2);
  stage_x<3>(rho, vel, acc, h, hh, x);
  accel<MORSE>(S, T, x, acc[2], s2);
  double base[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) base[i] = fma(h * dpC(4), vel[i], rho[i]);
  stage_x_ff<4>(base, acc, hhh, hhl, x);
  accel<MORSE>(S, T, x, acc[3], s2);
#pragma unroll
  for (int i = 0; i < 6; ++i) base[i] = fma(h * dpC(5), vel[i], rho[i]);
  stage_x_ff<5>(base, acc, hhh, hhl, x);
  accel<MORSE>(S, T, x, acc[4], s2);
#pragma unroll
  for (int i = 0; i < 6; ++i) base[i] = fma(h, vel[i], rho[i]);   // c_6 = c_7 = 1
  stage_x_ff<6>(base, acc, hhh, hhl, x);
  accel<MORSE>(S, T, x, acc[5], s2);
  stage_x<7>(base, acc, hh, xn);
  accel<MORSE>(S, T, xn, acc[6], s2);
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    double vb = kT.b[1] * acc[0][i];
#pragma unroll
    for (int q = 3; q <= 6; ++q) vb = fma(kT.b[q], acc[q - 1][i], vb);
    vn[i] = fma(h, vb, vel[i]);
    // (e^T A)_2 = e_2 = 0 and (e^T A)_7 = 0: a_2 never enters, a_7 only ev
    float es, ec, rs, rc, ah, al;
    split_ff(acc[0][i], ah, al);
    ff_dot_first(es, ec, kTff.e[1].hi, kTff.e[1].lo, ah, al);
    ff_dot_first(rs, rc, kTff.ea[1].hi, kTff.ea[1].lo, ah, al);
#pragma unroll
    for (int q = 3; q <= 7; ++q) {
      split_ff(acc[q - 1][i], ah, al);
      ff_dot_acc(es, ec, kTff.e[q].hi, kTff.e[q].lo, ah, al);
      if (!dpEAZero(q)) ff_dot_acc(rs, rc, kTff.ea[q].hi, kTff.ea[q].lo, ah, al);
    }
    ev[i] = es + ec;
    er[i] = rs + rc;
  }
}

// Lane registers.
struct LaneState {
  double rho[6], vel[6];
  double acc[7][6];
  double t, h, tmax;
  int nacc, nrej, calls;   // calls = accepted + rejected in this launch
  int status;
  int sid;
  float atv[2];            // atol / mu of the two velocity blocks (FP32)
  bool rejected;           // the current step attempt follows a rejection
};

// Starting step (Hairer, Norsett & Wanner, Solving ODEs I, Sec. II.4), as
// used by SciPy's solve_ivp; error-estimator order 4, exponent 1/5.  Run once
// per trajectory, in FP64.
template <bool MORSE>
__device__ double initial_step(const DevSys& S, const double* __restrict__ T, const LaneState& L,
                               double rtol, double atol) {
  double atv[2] = {atol * S.inv_mu12, atol * S.inv_mu123};
  double d0 = 0.0, d1 = 0.0;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    double scr = atol + fabs(L.rho[i]) * rtol;
    double scv = atv[i / 3] + fabs(L.vel[i]) * rtol;
    double q0 = L.rho[i] / scr, q1 = L.vel[i] / scv;
    d0 += q0 * q0 + q1 * q1;
    double p0 = L.vel[i] / scr, p1 = L.acc[0][i] / scv;
    d1 += p0 * p0 + p1 * p1;
  }
  d0 = sqrt(d0 / 12.0);
  d1 = sqrt(d1 / 12.0);
  double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
  double x1[6], a1[6], s2[3];
#pragma unroll
  for (int i = 0; i < 6; ++i) x1[i] = fma(h0, L.vel[i], L.rho[i]);
  accel<MORSE>(S, T, x1, a1, s2);
  double d2 = 0.0;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    double scr = atol + fabs(L.rho[i]) * rtol;
    double scv = atv[i / 3] + fabs(L.vel[i]) * rtol;
    double p0 = h0 * L.acc[0][i] / scr, p1 = (a1[i] - L.acc[0][i]) / scv;
    d2 += p0 * p0 + p1 * p1;
  }
  d2 = sqrt(d2 / 12.0) / h0;
  double h1 = (d1 <= 1e-15 && d2 <= 1e-15) ? fmax(1e-6, h0 * 1e-3)
                                           : pow(0.01 / fmax(d1, d2), 0.2);
  return fmin(100.0 * h0, h1);
}

__device__ __forceinline__ bool runnable(int st) {
  return st == QCAMS_LANE_READY || st == QCAMS_LANE_RUNNING;
}

// Load lane i; returns false if it is not runnable.  Computes acc[0] and,
// if no step size is stored yet, the starting step.
template <bool MORSE>
__device__ bool lane_load(const SysSet& sys, const IntegParams& ip, const double* __restrict__ T,
                          const DevBatch& B, int64_t i, LaneState& L,
                          unsigned long long& rhs_count) {
  L.status = B.status[i];
  if (!runnable(L.status)) return false;
  L.sid = B.sys_id[i];
  if (L.sid < 0 || L.sid >= sys.n) {
    B.status[i] = QCAMS_LANE_INVALID;
    return false;
  }
  const DevSys& S = sys.s[L.sid];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    L.rho[k] = B.y[k][i];
    L.rho[3 + k] = B.y[3 + k][i];
    L.vel[k] = B.y[6 + k][i] * S.inv_mu12;
    L.vel[3 + k] = B.y[9 + k][i] * S.inv_mu123;
  }
  L.t = B.t[i];
  L.h = B.h[i];
  L.tmax = ip.t_stop * B.t_scale[i];
  L.nacc = B.nsteps[i];
  L.nrej = B.nrej[i];
  L.calls = 0;
  L.rejected = false;
  L.status = QCAMS_LANE_RUNNING;
  L.atv[0] = (float)(ip.atol * S.inv_mu12);
  L.atv[1] = (float)(ip.atol * S.inv_mu123);
  double s2[3];
  accel<MORSE>(S, T, L.rho, L.acc[0], s2);
  rhs_count += 1;
  if (!(L.h > 0.0)) {
    L.h = initial_step<MORSE>(S, T, L, ip.rtol, ip.atol);
    rhs_count += 1;
  }
  return true;
}

template <bool MORSE>
__device__ void lane_store(const SysSet& sys, const DevBatch& B, int64_t i, const LaneState& L) {
  const DevSys& S = sys.s[L.sid];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    B.y[k][i] = L.rho[k];
    B.y[3 + k][i] = L.rho[3 + k];
    B.y[6 + k][i] = L.vel[k] * S.mu12;
    B.y[9 + k][i] = L.vel[3 + k] * S.mu123;
  }
  B.t[i] = L.t;
  B.h[i] = L.h;
  B.status[i] = static_cast<uint8_t>(L.status);
  B.nsteps[i] = L.nacc;
  B.nrej[i] = L.nrej;
}

// One adaptive step attempt with SciPy's RK45 rules: RMS error norm with
// scale atol + rtol max(|y_n|, |y_n+1|); accept iff norm < 1; new step
// h * clamp(0.9 norm^(-1/5), 0.2, 10), with no growth on the attempt that
// follows a rejection.  After an accepted step the stop rules are applied
// (Sec. 3.1: r_stop while separating, or t >= t_max).
//
// Only the step itself (stages, 5th-order update) is FP64; the error vector
// comes as FP32 from float-float sums.  The norm is formed in FP32 from
// 20-bit magnitudes of the state and scale terms (relative error < 1e-6,
// irrelevant to a step-size controller); accept / reject is a select, so
// the warp does not diverge.  The minimum step is checked by exponents: h
// fails below 8-16 ulp(t).
template <bool MORSE>
__device__ __forceinline__ void lane_attempt(const SysSet& sys, const DevShape* shapes,
                                             const IntegParams& ip, const double* __restrict__ T,
                                             LaneState& L) {
  const DevSys& S = sys.s[L.sid];
  {
    const int eh = (__double2hiint(L.h) >> 20) & 0x7ff;
    const int et = (__double2hiint(L.t) >> 20) & 0x7ff;
    if (et - eh >= 49 || eh == 0) {
      L.status = QCAMS_LANE_FAIL_HMIN;
      return;
    }
  }
  double xn[6], vn[6], s2[3];
  float er[6], ev[6];
  dp_step<MORSE>(S, T, L.rho, L.vel, L.acc, L.h, xn, vn, er, ev, s2);
  unsigned bad = 0, ignore = 0;
  float sum = 0.f;
  const float rt = ip.rtol_f, at = ip.atol_f;
  const float atv0 = L.atv[0], atv1 = L.atv[1];
  const float hf = mag_f(L.h, ignore), hhf = hf * hf;   // h > 0
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const float scr = fmaf(rt, fmaxf(mag_f(L.rho[i], ignore), mag_f(xn[i], ignore)), at);
    const float qr = err_mag(er[i], bad) * hhf * rcp_approx(scr);
    sum = fmaf(qr, qr, sum);
    const float scv = fmaf(rt, fmaxf(mag_f(L.vel[i], ignore), mag_f(vn[i], ignore)),
                           i < 3 ? atv0 : atv1);
    const float qv = err_mag(ev[i], bad) * hf * rcp_approx(scv);
    sum = fmaf(qv, qv, sum);
  }
  const float en2 = sum * (1.0f / 12.0f);
  L.calls += 1;
  if (bad) {
    L.status = QCAMS_LANE_FAIL_NAN;
    return;
  }
  // en^(-1/5) = en2^(-1/10)
  const float fac = 0.9f * pow_m01(en2);
  const bool accept = en2 < 1.0f;
  float fa = (en2 == 0.0f) ? 10.0f : fminf(10.0f, fac);
  fa = L.rejected ? fminf(1.0f, fa) : fa;
  const float f = accept ? fa : fmaxf(0.2f, fac);
  const double tn = L.t + L.h;
  L.t = accept ? tn : L.t;
  L.h = L.h * static_cast<double>(f);
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    L.rho[i] = accept ? xn[i] : L.rho[i];
    L.vel[i] = accept ? vn[i] : L.vel[i];
    L.acc[0][i] = accept ? L.acc[6][i] : L.acc[0][i];
  }
  L.nacc += accept ? 1 : 0;
  L.nrej += accept ? 0 : 1;
  L.rejected = !accept;
  // stop rules on the accepted state (integer / FP32 compares)
  const long long smax = max(dbits(s2[0]), max(dbits(s2[1]), dbits(s2[2])));
  const float radial = fmaf(signed_f(L.rho[3]), signed_f(L.vel[3]),
                            fmaf(signed_f(L.rho[4]), signed_f(L.vel[4]),
                                 signed_f(L.rho[5]) * signed_f(L.vel[5])));
  bool collapse = false;
  if (!MORSE) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
      collapse |= S.pair[k].kind == QCAMS_BUCK &&
                  dbits(s2[k]) < dbits(shapes[L.sid * 3 + k].r_b2);
  }
  int st = L.status;
  st = (accept && dbits(L.t) >= dbits(L.tmax)) ? QCAMS_LANE_DONE_TMAX : st;
  st = (accept && smax > dbits(ip.r_stop2) && radial > 0.0f) ? QCAMS_LANE_DONE_RSTOP : st;
  st = (accept && collapse) ? QCAMS_LANE_FAIL_COLLAPSE : st;
  st = (st == QCAMS_LANE_RUNNING && (long long)(L.nacc + L.nrej) >= ip.max_steps)
           ? QCAMS_LANE_FAIL_MAXSTEPS : st;
  L.status = st;
}

__device__ __forceinline__ void flush_counters(unsigned long long rhs, unsigned long long steps,
                                               unsigned long long* counters) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rhs += __shfl_xor_sync(FULL, rhs, o);
    steps += __shfl_xor_sync(FULL, steps, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&counters[0], rhs);
    atomicAdd(&counters[1], steps);
  }
}

// One thread per trajectory.
template <bool MORSE, int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) k_integrate_plain(SysSet sys, const DevShape* shapes,
                                                         IntegParams ip, DevBatch B,
                                                         unsigned long long* counters) {
  __shared__ double sT[kExpTableSize];
  load_exp_table(sT);
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  unsigned long long rhs = 0, steps = 0;
  LaneState L;
  if (i < B.n && lane_load<MORSE>(sys, ip, sT, B, i, L, rhs)) {
    while (L.status == QCAMS_LANE_RUNNING) lane_attempt<MORSE>(sys, shapes, ip, sT, L);
    rhs += 6ull * L.calls;
    steps += L.calls;
    lane_store<MORSE>(sys, B, i, L);
  }
  flush_counters(rhs, steps, counters);
}

// Persistent refill-queue launch: each warp pops trajectory indices for all
// of its idle lanes with one atomicAdd (ballot + popc + shuffle).
template <bool MORSE, int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) k_integrate_persistent(SysSet sys, const DevShape* shapes,
                                                              IntegParams ip, DevBatch B,
                                                              unsigned long long* counters) {
  __shared__ double sT[kExpTableSize];
  load_exp_table(sT);
  const unsigned lane = threadIdx.x & 31u;
  unsigned long long rhs = 0, steps = 0;
  LaneState L;
  int64_t idx = -1;
  bool have = false, exhausted = false;
  for (;;) {
    const bool need = !have && !exhausted;
    const unsigned want = __ballot_sync(FULL, need);
    if (want) {
      const int leader = __ffs(want) - 1;
      unsigned long long base = 0;
      if ((int)lane == leader) base = atomicAdd(&counters[2], (unsigned long long)__popc(want));
      base = __shfl_sync(FULL, base, leader);
      if (need) {
        const int64_t k = (int64_t)(base + __popc(want & ((1u << lane) - 1u)));
        if (k >= B.n) {
          exhausted = true;
        } else {
          idx = k;
          have = lane_load<MORSE>(sys, ip, sT, B, idx, L, rhs);
        }
      }
    }
    if (__all_sync(FULL, exhausted && !have)) break;
    if (have) {
      lane_attempt<MORSE>(sys, shapes, ip, sT, L);
      if (L.status != QCAMS_LANE_RUNNING) {
        rhs += 6ull * L.calls;
        steps += L.calls;
        lane_store<MORSE>(sys, B, idx, L);
        have = false;
      }
    }
  }
  flush_counters(rhs, steps, counters);
}

// Fixed-step mode: exactly max_steps steps of size h_fixed, no control and
// no stop test (used to check the integrator against the reference steps).
template <bool MORSE>
__global__ void __launch_bounds__(128) k_integrate_fixed(SysSet sys, IntegParams ip, DevBatch B,
                                                         unsigned long long* counters) {
  __shared__ double sT[kExpTableSize];
  load_exp_table(sT);
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  unsigned long long rhs = 0, steps = 0;
  if (i < B.n) {
    int st = B.status[i];
    const int sid = B.sys_id[i];
    if (runnable(st) && (sid < 0 || sid >= sys.n)) B.status[i] = QCAMS_LANE_INVALID;
    if (runnable(st) && sid >= 0 && sid < sys.n) {
      LaneState L;
      L.sid = sid;
      const DevSys& S = sys.s[L.sid];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        L.rho[k] = B.y[k][i];
        L.rho[3 + k] = B.y[3 + k][i];
        L.vel[k] = B.y[6 + k][i] * S.inv_mu12;
        L.vel[3 + k] = B.y[9 + k][i] * S.inv_mu123;
      }
      double s2[3];
      accel<MORSE>(S, sT, L.rho, L.acc[0], s2);
      double t = B.t[i];
      const double h = ip.h_fixed;
      for (long long it = 0; it < ip.max_steps; ++it) {
        double xn[6], vn[6];
        float er[6], ev[6];
        dp_step<MORSE>(S, sT, L.rho, L.vel, L.acc, h, xn, vn, er, ev, s2);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          L.rho[q] = xn[q];
          L.vel[q] = vn[q];
          L.acc[0][q] = L.acc[6][q];
        }
        t += h;
      }
      L.t = t;
      L.h = h;
      L.status = QCAMS_LANE_RUNNING;
      L.nacc = B.nsteps[i] + (int)ip.max_steps;
      L.nrej = B.nrej[i];
      lane_store<MORSE>(sys, B, i, L);
      rhs = 1 + 6ull * ip.max_steps;
      steps = ip.max_steps;
    }
  }
  flush_counters(rhs, steps, counters);
}

__global__ void k_exp_check(const double* x, double* mine, double* ref, long long n) {
  __shared__ double sT[kExpTableSize];
  load_exp_table(sT);
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  mine[i] = texp(x[i], sT);
  ref[i] = exp(x[i]);
}

// The integrator's pair-force elementary functions on n squared distances s
// of one Morse pair (alpha = c0, alpha re = c1): 1/sqrt(s), the exponent's
// argument x = c1 - c0 r and e^x, exactly as the force law forms them.
__global__ void k_force_math_check(const double* s, double c0, double c1, float c0f, float c1f,
                                   double* ri_out, double* x_out, double* e_out, long long n) {
  __shared__ double sT[kExpTableSize];
  load_exp_table(sT);
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float rf;
  const double si = s[i];
  const double ri = rsqrt_seeded(si, rf);
  const double x = fma(-c0, si * ri, c1);
  ri_out[i] = ri;
  x_out[i] = x;
  e_out[i] = texp_hint(x, fmaf(-c0f, rf, c1f), sT);
}

// The integrator's float-float dot product on n rows of m <= 8 terms:
// out[i] = sum_q w[q] a[i m + q] formed as in the stage corrections (both
// operands split into float pairs, Dot2 accumulation, rebuilt as a double)
// and out_f[i] = the same sum rounded to FP32 as the error estimate takes it.
__global__ void k_ff_dot_check(const double* a, const double* w, int m, double* out,
                               float* out_f, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.0f, c = 0.0f;
  for (int q = 0; q < m; ++q) {
    float wh, wl, ah, al;
    split_ff(w[q], wh, wl);
    split_ff(a[i * m + q], ah, al);
    if (q == 0)
      ff_dot_first(s, c, wh, wl, ah, al);
    else
      ff_dot_acc(s, c, wh, wl, ah, al);
  }
  out[i] = ff_to_double(s, c);
  out_f[i] = s + c;
}

bool all_morse(const SysSet& s) {
  for (int k = 0; k < s.n; ++k)
    for (int p = 0; p < 3; ++p)
      if (s.s[k].pair[p].kind != QCAMS_MORSE) return false;
  return true;
}

// Launch-shape variants: threads per block and the resident blocks per SM
// each kernel is compiled for (__launch_bounds__ minimum, which caps the
// registers per thread).  At ~190 registers, 64-thread blocks fit 5 per SM
// (10 warps) where 128-thread blocks fit 2 (8 warps); the autotuner measures.
struct Variant {
  int block, minb;
};
constexpr Variant kVariants[] = {{128, 1}, {64, 1}, {128, 3}, {64, 6}, {64, 7}, {256, 1}};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

int find_variant(int block, int minb) {
  if (block <= 0) block = 128;
  if (minb <= 0) minb = 1;
  for (int v = 0; v < kNumVariants; ++v)
    if (kVariants[v].block == block && kVariants[v].minb == minb) return v;
  return -1;
}

template <bool MORSE, int BLOCK, int MINB>
cudaError_t launch_shape(const SysSet& sys, const DevShape* shapes, const IntegParams& ip,
                         const DevBatch& b, int persistent, Ctx& ctx, cudaStream_t st,
                         int* blocks_per_sm_out) {
  if (persistent) {
    cudaError_t e = cudaMemsetAsync(ctx.counters + 2, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, k_integrate_persistent<MORSE, BLOCK, MINB>, BLOCK, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (blocks_per_sm_out) *blocks_per_sm_out = per_sm;
    long long grid = (long long)per_sm * ctx.sm_count;
    const long long need = (b.n + BLOCK - 1) / BLOCK;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    k_integrate_persistent<MORSE, BLOCK, MINB><<<(unsigned)grid, BLOCK, 0, st>>>(
        sys, shapes, ip, b, ctx.counters);
    return cudaGetLastError();
  }
  const unsigned grid = (unsigned)((b.n + BLOCK - 1) / BLOCK);
  k_integrate_plain<MORSE, BLOCK, MINB><<<grid, BLOCK, 0, st>>>(sys, shapes, ip, b, ctx.counters);
  return cudaGetLastError();
}

template <bool MORSE>
cudaError_t launch_variant(int v, const SysSet& sys, const DevShape* shapes,
                           const IntegParams& ip, const DevBatch& b, int persistent, Ctx& ctx,
                           cudaStream_t st, int* bps) {
  switch (v) {
    case 0: return launch_shape<MORSE, 128, 1>(sys, shapes, ip, b, persistent, ctx, st, bps);
    case 1: return launch_shape<MORSE, 64, 1>(sys, shapes, ip, b, persistent, ctx, st, bps);
    case 2: return launch_shape<MORSE, 128, 3>(sys, shapes, ip, b, persistent, ctx, st, bps);
    case 3: return launch_shape<MORSE, 64, 6>(sys, shapes, ip, b, persistent, ctx, st, bps);
    case 4: return launch_shape<MORSE, 64, 7>(sys, shapes, ip, b, persistent, ctx, st, bps);
    case 5: return launch_shape<MORSE, 256, 1>(sys, shapes, ip, b, persistent, ctx, st, bps);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_exp_check(const double* x, double* mine, double* ref, long long n,
                             cudaStream_t st) {
  k_exp_check<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, mine, ref, n);
  return cudaGetLastError();
}

cudaError_t launch_force_math_check(const double* s, double c0, double c1, double* ri,
                                    double* x, double* e, long long n, cudaStream_t st) {
  k_force_math_check<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s, c0, c1, (float)c0,
                                                                  (float)c1, ri, x, e, n);
  return cudaGetLastError();
}

cudaError_t launch_ff_dot_check(const double* a, const double* w, int m, double* out,
                               float* out_f, long long n, cudaStream_t st) {
  k_ff_dot_check<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, w, m, out, out_f, n);
  return cudaGetLastError();
}

cudaError_t launch_integrate(const SysSet& sys, const DevShape* shapes, const IntegParams& ip,
                             const DevBatch& b, int precision, int persistent, int block,
                             int blocks_per_sm, Ctx& ctx, cudaStream_t st) {
  if (b.n == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(ctx.counters, 0, 2 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  const bool morse = all_morse(sys);
  if (precision == 32) return launch_integrate32(sys, shapes, ip, b, persistent, ctx, st, morse);
  if (ip.fixed_step) {
    const unsigned grid = (unsigned)((b.n + 127) / 128);
    if (morse) k_integrate_fixed<true><<<grid, 128, 0, st>>>(sys, ip, b, ctx.counters);
    else k_integrate_fixed<false><<<grid, 128, 0, st>>>(sys, ip, b, ctx.counters);
    return cudaGetLastError();
  }
  if (persistent == 2 || persistent == 3)
    return launch_integrate_grouped(sys, shapes, ip, b, persistent == 2 ? 3 : 6, ctx.counters, st,
                                    morse);
  const int v = find_variant(block, blocks_per_sm);
  if (v < 0) return cudaErrorInvalidValue;
  return morse ? launch_variant<true>(v, sys, shapes, ip, b, persistent, ctx, st, nullptr)
               : launch_variant<false>(v, sys, shapes, ip, b, persistent, ctx, st, nullptr);
}

int integrate_variant_count() { return kNumVariants; }

void integrate_variant_shape(int v, int* block, int* minb) {
  *block = kVariants[v].block;
  *minb = kVariants[v].minb;
}

bool integrate_shape_supported(int block, int blocks_per_sm) {
  return find_variant(block, blocks_per_sm) >= 0;
}

cudaError_t integrate_variant_regs(int v, bool morse, int* regs) {
  cudaFuncAttributes a;
  cudaError_t e = cudaErrorInvalidValue;
#define QCAMS_REGS(M, B, N) e = cudaFuncGetAttributes(&a, k_integrate_persistent<M, B, N>)
  switch (v) {
    case 0: if (morse) QCAMS_REGS(true, 128, 1); else QCAMS_REGS(false, 128, 1); break;
    case 1: if (morse) QCAMS_REGS(true, 64, 1); else QCAMS_REGS(false, 64, 1); break;
    case 2: if (morse) QCAMS_REGS(true, 128, 3); else QCAMS_REGS(false, 128, 3); break;
    case 3: if (morse) QCAMS_REGS(true, 64, 6); else QCAMS_REGS(false, 64, 6); break;
    case 4: if (morse) QCAMS_REGS(true, 64, 7); else QCAMS_REGS(false, 64, 7); break;
    case 5: if (morse) QCAMS_REGS(true, 256, 1); else QCAMS_REGS(false, 256, 1); break;
    default: break;
  }
#undef QCAMS_REGS
  if (e == cudaSuccess) *regs = a.numRegs;
  return e;
}

cudaError_t integrate_variant_occupancy(int v, bool morse, int* blocks_per_sm) {
  cudaError_t e = cudaErrorInvalidValue;
#define QCAMS_OCC(M, B, N) \
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_integrate_persistent<M, B, N>, B, 0)
  switch (v) {
    case 0: if (morse) QCAMS_OCC(true, 128, 1); else QCAMS_OCC(false, 128, 1); break;
    case 1: if (morse) QCAMS_OCC(true, 64, 1); else QCAMS_OCC(false, 64, 1); break;
    case 2: if (morse) QCAMS_OCC(true, 128, 3); else QCAMS_OCC(false, 128, 3); break;
    case 3: if (morse) QCAMS_OCC(true, 64, 6); else QCAMS_OCC(false, 64, 6); break;
    case 4: if (morse) QCAMS_OCC(true, 64, 7); else QCAMS_OCC(false, 64, 7); break;
    case 5: if (morse) QCAMS_OCC(true, 256, 1); else QCAMS_OCC(false, 256, 1); break;
    default: break;
  }
#undef QCAMS_OCC
  return e;
}

bool integrate_all_morse(const SysSet& sys) { return all_morse(sys); }

}  // namespace qcams
