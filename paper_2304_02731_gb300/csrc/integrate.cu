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
#include <cuda_runtime.h>

#include "qcams_device.cuh"
#include "qcams_internal.h"

namespace qcams {
namespace {

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
    t.ea[s] = dpEA(s);
    for (int q = 1; q <= 7; ++q) t.a2[s][q] = dpA2(s, q);
  }
  return t;
}
// Coefficients in the constant bank: a DFMA takes a constant-bank operand at
// full rate, so indexing this table with compile-time indices costs nothing.
__constant__ RknTab kT = make_rkn_tab();

constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------------------
// Accelerations a = (dP1/dt / mu12, dP2/dt / mu123) at Jacobi positions x,
// and the squared pair distances (AB, BC, CA).
//   r_AB = rho1,  r_BC = rho2 - cB rho1,  r_CA = rho2 + cA rho1
//   dV/drho1 = g_AB r_AB - cB g_BC r_BC + cA g_CA r_CA,
//   dV/drho2 = g_BC r_BC + g_CA r_CA,          g = V'(r)/r.
// ---------------------------------------------------------------------------
template <bool MORSE>
__device__ __forceinline__ double pair_g(const DevPair& q, double s) {
  double ri = rsqrt(s);
  double r = s * ri;
  if (MORSE) {
    double x = exp(fma(-q.c0, r, q.c1));
    return q.c2 * x * (1.0 - x) * ri;
  }
  return pot_g(q, ri, r);
}

template <bool MORSE>
__device__ __forceinline__ void accel(const DevSys& S, const double* x, double* a, double* s2) {
  double rab0 = x[0], rab1 = x[1], rab2 = x[2];
  double rbc0 = fma(-S.cB, x[0], x[3]), rbc1 = fma(-S.cB, x[1], x[4]), rbc2 = fma(-S.cB, x[2], x[5]);
  double rca0 = fma(S.cA, x[0], x[3]), rca1 = fma(S.cA, x[1], x[4]), rca2 = fma(S.cA, x[2], x[5]);
  s2[0] = fma(rab0, rab0, fma(rab1, rab1, rab2 * rab2));
  s2[1] = fma(rbc0, rbc0, fma(rbc1, rbc1, rbc2 * rbc2));
  s2[2] = fma(rca0, rca0, fma(rca1, rca1, rca2 * rca2));
  double g0 = pair_g<MORSE>(S.pair[0], s2[0]);
  double g1 = pair_g<MORSE>(S.pair[1], s2[1]);
  double g2 = pair_g<MORSE>(S.pair[2], s2[2]);
  double f0 = -g0 * S.inv_mu12, f1 = S.cB * g1 * S.inv_mu12, f2 = -S.cA * g2 * S.inv_mu12;
  a[0] = fma(f0, rab0, fma(f1, rbc0, f2 * rca0));
  a[1] = fma(f0, rab1, fma(f1, rbc1, f2 * rca1));
  a[2] = fma(f0, rab2, fma(f1, rbc2, f2 * rca2));
  double h1 = -g1 * S.inv_mu123, h2 = -g2 * S.inv_mu123;
  a[3] = fma(h1, rbc0, h2 * rca0);
  a[4] = fma(h1, rbc1, h2 * rca1);
  a[5] = fma(h1, rbc2, h2 * rca2);
}

// Position of stage s (1-based, s >= 2).
template <int s>
__device__ __forceinline__ void stage_x(const double* rho, const double* vel, const double (*acc)[6],
                                        double h, double hh, double* x) {
  const double hc = h * kT.c[s];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    double sum = 0.0;
#pragma unroll
    for (int q = 1; q <= s - 2; ++q) sum = fma(kT.a2[s][q], acc[q - 1][i], sum);
    x[i] = fma(hh, sum, fma(hc, vel[i], rho[i]));
  }
}

// One Dormand-Prince step of size h from (rho, vel) with acc[0] = a(rho).
// On return acc[1..6] hold the stage accelerations, xn / vn the 5th-order
// solution (acc[6] = a(xn), FSAL), er / ev the embedded error estimates of
// positions and velocities, s2 the squared pair distances at xn.
template <bool MORSE>
__device__ __forceinline__ void dp_step(const DevSys& S, const double* rho, const double* vel,
                                        double (*acc)[6], double h, double* xn, double* vn,
                                        double* er, double* ev, double* s2) {
  const double hh = h * h;
  double x[6];
  stage_x<2>(rho, vel, acc, h, hh, x);
  accel<MORSE>(S, x, acc[1], s2);
  stage_x<3>(rho, vel, acc, h, hh, x);
  accel<MORSE>(S, x, acc[2], s2);
  stage_x<4>(rho, vel, acc, h, hh, x);
  accel<MORSE>(S, x, acc[3], s2);
  stage_x<5>(rho, vel, acc, h, hh, x);
  accel<MORSE>(S, x, acc[4], s2);
  stage_x<6>(rho, vel, acc, h, hh, x);
  accel<MORSE>(S, x, acc[5], s2);
  stage_x<7>(rho, vel, acc, h, hh, xn);
  accel<MORSE>(S, xn, acc[6], s2);
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    double vb = kT.b[1] * acc[0][i];
#pragma unroll
    for (int q = 3; q <= 6; ++q) vb = fma(kT.b[q], acc[q - 1][i], vb);
    vn[i] = fma(h, vb, vel[i]);
    double e = kT.e[1] * acc[0][i];
#pragma unroll
    for (int q = 3; q <= 7; ++q) e = fma(kT.e[q], acc[q - 1][i], e);
    ev[i] = h * e;
    double ea = kT.ea[1] * acc[0][i];
#pragma unroll
    for (int q = 2; q <= 6; ++q) ea = fma(kT.ea[q], acc[q - 1][i], ea);
    er[i] = hh * ea;
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
  bool rejected;           // the current step attempt follows a rejection
};

__device__ __forceinline__ double rms_ratio(const double* e, const double* sc) {
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    double q = e[i] / sc[i];
    s = fma(q, q, s);
  }
  return s;
}

// Starting step (Hairer, Norsett & Wanner, Solving ODEs I, Sec. II.4), as
// used by SciPy's solve_ivp; error-estimator order 4, exponent 1/5.
template <bool MORSE>
__device__ double initial_step(const DevSys& S, const LaneState& L, double rtol, double atol) {
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
  accel<MORSE>(S, x1, a1, s2);
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
__device__ bool lane_load(const SysSet& sys, const IntegParams& ip, const DevBatch& B, int64_t i,
                          LaneState& L, unsigned long long& rhs_count) {
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
  double s2[3];
  accel<MORSE>(S, L.rho, L.acc[0], s2);
  rhs_count += 1;
  if (!(L.h > 0.0)) {
    L.h = initial_step<MORSE>(S, L, ip.rtol, ip.atol);
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
// (Sec. 3.1: r_stop while separating, or t >= t_max).  The controller's
// power is taken in FP32 (its result only scales the next step).
template <bool MORSE>
__device__ __forceinline__ void lane_attempt(const SysSet& sys, const DevShape* shapes,
                                             const IntegParams& ip, LaneState& L) {
  const DevSys& S = sys.s[L.sid];
  // minimum step: 10 ulp(t)
  double ulp_t = __longlong_as_double(__double_as_longlong(L.t) + 1) - L.t;
  if (L.h < 10.0 * ulp_t) {
    L.status = QCAMS_LANE_FAIL_HMIN;
    return;
  }
  double xn[6], vn[6], er[6], ev[6], s2[3];
  dp_step<MORSE>(S, L.rho, L.vel, L.acc, L.h, xn, vn, er, ev, s2);
  double sr[6], sv[6];
  const double atv0 = ip.atol * S.inv_mu12, atv1 = ip.atol * S.inv_mu123;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    sr[i] = fma(ip.rtol, fmax(fabs(L.rho[i]), fabs(xn[i])), ip.atol);
    sv[i] = fma(ip.rtol, fmax(fabs(L.vel[i]), fabs(vn[i])), i < 3 ? atv0 : atv1);
  }
  double en2 = (rms_ratio(er, sr) + rms_ratio(ev, sv)) * (1.0 / 12.0);
  L.calls += 1;
  if (!(en2 == en2)) {
    L.status = QCAMS_LANE_FAIL_NAN;
    return;
  }
  // en^(-1/5) = en2^(-1/10)
  float fac = __powf(static_cast<float>(en2), -0.1f) * 0.9f;
  bool accept = en2 < 1.0;
  if (accept) {
    float f = (en2 == 0.0) ? 10.0f : fminf(10.0f, fac);
    if (L.rejected) f = fminf(1.0f, f);
    L.t += L.h;
    L.h *= static_cast<double>(f);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      L.rho[i] = xn[i];
      L.vel[i] = vn[i];
      L.acc[0][i] = L.acc[6][i];
    }
    L.nacc += 1;
    L.rejected = false;
    // stop rules
    bool collapse = false;
    double smax = fmax(s2[0], fmax(s2[1], s2[2]));
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (S.pair[k].kind == QCAMS_BUCK && s2[k] < shapes[L.sid * 3 + k].r_b2) collapse = true;
    double radial = L.rho[3] * L.vel[3] + L.rho[4] * L.vel[4] + L.rho[5] * L.vel[5];
    if (collapse) L.status = QCAMS_LANE_FAIL_COLLAPSE;
    else if (smax > ip.r_stop2 && radial > 0.0) L.status = QCAMS_LANE_DONE_RSTOP;
    else if (L.t >= L.tmax) L.status = QCAMS_LANE_DONE_TMAX;
  } else {
    L.h *= static_cast<double>(fmaxf(0.2f, fac));
    L.nrej += 1;
    L.rejected = true;
  }
  if (L.status == QCAMS_LANE_RUNNING && (long long)(L.nacc + L.nrej) >= ip.max_steps)
    L.status = QCAMS_LANE_FAIL_MAXSTEPS;
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
template <bool MORSE>
__global__ void __launch_bounds__(128) k_integrate_plain(SysSet sys, const DevShape* shapes,
                                                         IntegParams ip, DevBatch B,
                                                         unsigned long long* counters) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  unsigned long long rhs = 0, steps = 0;
  LaneState L;
  if (i < B.n && lane_load<MORSE>(sys, ip, B, i, L, rhs)) {
    while (L.status == QCAMS_LANE_RUNNING) lane_attempt<MORSE>(sys, shapes, ip, L);
    rhs += 6ull * L.calls;
    steps += L.calls;
    lane_store<MORSE>(sys, B, i, L);
  }
  flush_counters(rhs, steps, counters);
}

// Persistent refill-queue launch: each warp pops trajectory indices for all
// of its idle lanes with one atomicAdd (ballot + popc + shuffle).
template <bool MORSE>
__global__ void __launch_bounds__(128) k_integrate_persistent(SysSet sys, const DevShape* shapes,
                                                              IntegParams ip, DevBatch B,
                                                              unsigned long long* counters) {
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
          have = lane_load<MORSE>(sys, ip, B, idx, L, rhs);
        }
      }
    }
    if (__all_sync(FULL, exhausted && !have)) break;
    if (have) {
      lane_attempt<MORSE>(sys, shapes, ip, L);
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
      accel<MORSE>(S, L.rho, L.acc[0], s2);
      double t = B.t[i];
      const double h = ip.h_fixed;
      for (long long it = 0; it < ip.max_steps; ++it) {
        double xn[6], vn[6], er[6], ev[6];
        dp_step<MORSE>(S, L.rho, L.vel, L.acc, h, xn, vn, er, ev, s2);
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

bool all_morse(const SysSet& s) {
  for (int k = 0; k < s.n; ++k)
    for (int p = 0; p < 3; ++p)
      if (s.s[k].pair[p].kind != QCAMS_MORSE) return false;
  return true;
}

template <bool MORSE>
cudaError_t launch_fp64(const SysSet& sys, const DevShape* shapes, const IntegParams& ip,
                        const DevBatch& b, int persistent, int block, int blocks_per_sm, Ctx& ctx,
                        cudaStream_t st) {
  if (block <= 0) block = 128;
  if (block > 128) block = 128;
  block = (block / 32) * 32;
  if (block == 0) block = 32;
  if (ip.fixed_step) {
    unsigned grid = (unsigned)((b.n + block - 1) / block);
    k_integrate_fixed<MORSE><<<grid, block, 0, st>>>(sys, ip, b, ctx.counters);
    return cudaGetLastError();
  }
  if (persistent) {
    cudaError_t e = cudaMemsetAsync(ctx.counters + 2, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    int per_sm = blocks_per_sm;
    if (per_sm <= 0) {
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_integrate_persistent<MORSE>,
                                                        block, 0);
      if (e != cudaSuccess) return e;
      if (per_sm < 1) per_sm = 1;
    }
    long long grid = (long long)per_sm * ctx.sm_count;
    long long need = (b.n + block - 1) / block;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    k_integrate_persistent<MORSE><<<(unsigned)grid, block, 0, st>>>(sys, shapes, ip, b,
                                                                    ctx.counters);
    return cudaGetLastError();
  }
  unsigned grid = (unsigned)((b.n + block - 1) / block);
  k_integrate_plain<MORSE><<<grid, block, 0, st>>>(sys, shapes, ip, b, ctx.counters);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_integrate(const SysSet& sys, const DevShape* shapes, const IntegParams& ip,
                             const DevBatch& b, int precision, int persistent, int block,
                             int blocks_per_sm, Ctx& ctx, cudaStream_t st) {
  if (b.n == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(ctx.counters, 0, 2 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  (void)precision;
  if (all_morse(sys))
    return launch_fp64<true>(sys, shapes, ip, b, persistent, block, blocks_per_sm, ctx, st);
  return launch_fp64<false>(sys, shapes, ip, b, persistent, block, blocks_per_sm, ctx, st);
}

}  // namespace qcams
