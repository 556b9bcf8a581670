// FP64 trajectory integrator for small batches: three lanes per trajectory.
//
// The same method as integrate.cu (Hamilton's equations in Jacobi
// coordinates, Sec. 2 Eqs. 3-4; Dormand-Prince 5(4) in Runge-Kutta-Nystrom
// form with SciPy's RK45 step control, Sec. 3.2; the stop rules of
// Sec. 3.1), laid out for latency instead of throughput.
//
// GB300 issues a warp-wide FP64 instruction in 64 cycles per SM
// sub-partition however many of its lanes are active.  A batch too small to
// give every sub-partition full warps (the 1,000-trajectory plain study runs
// 32 warps on 608 sub-partitions) therefore takes as long as its longest
// trajectory's chain of warp-wide FP64 instructions, 516 per step in the
// one-thread-per-trajectory kernel.  Here lane j = 0, 1, 2 of a trajectory's
// triplet holds spatial component j of both Jacobi vectors, their velocities
// and the stage accelerations, and evaluates the force of pair j (AB, BC,
// CA).  The triplet exchanges the squared pair distances, the pair force
// factors and the error norm's partial sums by warp shuffles.  A step costs
// about 200 warp-wide FP64 instructions, so the longest trajectory of a
// small batch finishes about 2.5x sooner; a warp carries 10 trajectories
// instead of 32, so large batches belong to the one-thread kernels.
//
// Every quantity the step control and the stop rules decide on (error norm,
// largest pair distance, radial velocity, collapse) is reduced in the same
// lane order in all three lanes, so the triplet's lanes take identical
// decisions.  Lanes 30 and 31 repeat components 0 and 1 of the warp's last
// triplet and store nothing; a lane whose trajectory is done or absent keeps
// executing the warp's instructions (FP64 costs the same either way) with
// its state frozen, so every shuffle runs on the full warp.
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

__constant__ RknTab kT3 = make_rkn_tab();
__constant__ RknTabFF kTff3 = make_rkn_tab_ff();

constexpr unsigned FULL = 0xffffffffu;
constexpr int kTriPerWarp = 10;   // triplets in lanes 0..29
constexpr int kTriBlock = 32;     // one warp per block: small batches spread over the SMs

// The lane's place in its triplet and the constants of its pair.
struct Tri {
  int j;        // spatial component and pair index (0 = AB, 1 = BC, 2 = CA)
  int base;     // lane of component 0
  DevPair q;    // pair j of the trajectory's system
  double kf;    // dP1-force factor of pair j (f_j = kf u_j)
  double kh;    // dP2-force factor (h_1, h_2; 0 for pair AB)
};

// Sum over the triplet of a per-lane value, in lane order (identical in the
// three lanes).
__device__ __forceinline__ float tri_sum(float v, int base) {
  const float a = __shfl_sync(FULL, v, base), b = __shfl_sync(FULL, v, base + 1),
              c = __shfl_sync(FULL, v, base + 2);
  return (a + b) + c;
}
__device__ __forceinline__ double tri_sum(double v, int base) {
  const double a = __shfl_sync(FULL, v, base), b = __shfl_sync(FULL, v, base + 1),
               c = __shfl_sync(FULL, v, base + 2);
  return (a + b) + c;
}
__device__ __forceinline__ unsigned tri_or(unsigned v, int base) {
  return __shfl_sync(FULL, v, base) | __shfl_sync(FULL, v, base + 1) |
         __shfl_sync(FULL, v, base + 2);
}
__device__ __forceinline__ long long tri_max(long long v, int base) {
  const long long a = __shfl_sync(FULL, v, base), b = __shfl_sync(FULL, v, base + 1),
                  c = __shfl_sync(FULL, v, base + 2);
  return max(a, max(b, c));
}

// Components j of the accelerations (a1 = dP1/dt / mu12, a2 = dP2/dt / mu123)
// at Jacobi positions with components x1, x2 in the triplet's lanes, and the
// squared distance of pair j.  The pair vectors are those of accel() in
// integrate.cu:
//   r_AB = rho1,  r_BC = rho2 - cB rho1,  r_CA = rho2 + cA rho1.
// Lane j gathers the three squared components of pair j (two shuffles, each
// lane sending the square that the receiving lane's pair needs), evaluates
// u_j = V'(r_j)/r_j, and the triplet exchanges f_j = kf u_j and h_j = kh u_j.
template <bool MORSE>
__device__ __forceinline__ void accel_tri(const DevSys& S, const Tri& L,
                                          const double* __restrict__ T, double x1, double x2,
                                          double& a1, double& a2, double& s_own) {
  const double rab = x1, rbc = fma(-S.cB, x1, x2), rca = fma(S.cA, x1, x2);
  const double q0 = rab * rab, q1 = rbc * rbc, q2 = rca * rca;
  double s = L.j == 0 ? q0 : (L.j == 1 ? q1 : q2);
#pragma unroll
  for (int r = 1; r <= 2; ++r) {
    // this lane, as sender, holds component (j) of every pair; the lane that
    // pulls from it in round r has pair index (j - r) mod 3
    const int want = (L.j + 3 - r) % 3;
    const double v = want == 0 ? q0 : (want == 1 ? q1 : q2);
    s += __shfl_sync(FULL, v, L.base + (L.j + r) % 3);
  }
  s_own = s;
  const double u = pair_u<MORSE>(L.q, s, T);
  const double f = L.kf * u, h = L.kh * u;
  const double f0 = __shfl_sync(FULL, f, L.base), f1 = __shfl_sync(FULL, f, L.base + 1),
               f2 = __shfl_sync(FULL, f, L.base + 2);
  const double h1 = __shfl_sync(FULL, h, L.base + 1), h2 = __shfl_sync(FULL, h, L.base + 2);
  a1 = fma(f0, rab, fma(f1, rbc, f2 * rca));
  a2 = fma(h1, rbc, h2 * rca);
}

// Stage positions for this lane's two components (index 0: rho1_j, 1:
// rho2_j), the formulas of integrate.cu's stage_x / stage_x_ff.
// Stage s from base = rho + h c_s v, FP64 sums (stages 2, 3 and 7).
template <int s>
__device__ __forceinline__ void stage_x2(const double* base, const double (*acc)[2], double hh,
                                         double* x) {
  double w[s > 2 ? s - 2 : 1];
#pragma unroll
  for (int q = 1; q <= s - 2; ++q) w[q - 1] = dpA2Zero(s, q) ? 0.0 : hh * kT3.a2[s][q];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    double xi = base[i];
#pragma unroll
    for (int q = 1; q <= s - 2; ++q)
      if (!dpA2Zero(s, q)) xi = fma(w[q - 1], acc[q - 1][i], xi);
    x[i] = xi;
  }
}
// Stages 4-6: the acceleration correction as a float-float dot product
// added to the FP64 base with one DADD.
template <int s>
__device__ __forceinline__ void stage_x2_ff(const double* base, const double (*acc)[2], float hhh,
                                            float hhl, double* x) {
  float wh[s - 2], wl[s - 2];
#pragma unroll
  for (int q = 1; q <= s - 2; ++q) {
    const FFc c = kTff3.a2[s][q];
    wh[q - 1] = __fmul_rn(hhh, c.hi);
    wl[q - 1] = fmaf(hhh, c.hi, -wh[q - 1]) + fmaf(hhh, c.lo, hhl * c.hi);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
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

// One Dormand-Prince step of size h for this lane's components, with
// acc[0] = a(rho).  On return acc[1..6] hold the stage accelerations, xn /
// vn the 5th-order solution, er / ev the embedded error estimates divided by
// h^2 and h, s_own the squared distance of pair j at xn (the same
// arithmetic per component as integrate.cu's dp_step).
template <bool MORSE>
__device__ __forceinline__ void dp_step_tri(const DevSys& S, const Tri& L,
                                            const double* __restrict__ T, const double* rho,
                                            const double* vel, double (*acc)[2], double h,
                                            double* xn, double* vn, float* er, float* ev,
                                            double& s_own) {
  const double hh = h * h;
  float hhh, hhl;
  split_ff(hh, hhh, hhl);
  double x[2], base[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) base[i] = fma(h * dpC(2), vel[i], rho[i]);
  stage_x2<2>(base, acc, hh, x);
  accel_tri<MORSE>(S, L, T, x[0], x[1], acc[1][0], acc[1][1], s_own);
#pragma unroll
  for (int i = 0; i < 2; ++i) base[i] = fma(h * dpC(3), vel[i], rho[i]);
  stage_x2<3>(base, acc, hh, x);
  accel_tri<MORSE>(S, L, T, x[0], x[1], acc[2][0], acc[2][1], s_own);
#pragma unroll
  for (int i = 0; i < 2; ++i) base[i] = fma(h * dpC(4), vel[i], rho[i]);
  stage_x2_ff<4>(base, acc, hhh, hhl, x);
  accel_tri<MORSE>(S, L, T, x[0], x[1], acc[3][0], acc[3][1], s_own);
#pragma unroll
  for (int i = 0; i < 2; ++i) base[i] = fma(h * dpC(5), vel[i], rho[i]);
  stage_x2_ff<5>(base, acc, hhh, hhl, x);
  accel_tri<MORSE>(S, L, T, x[0], x[1], acc[4][0], acc[4][1], s_own);
#pragma unroll
  for (int i = 0; i < 2; ++i) base[i] = fma(h, vel[i], rho[i]);   // c_6 = c_7 = 1
  stage_x2_ff<6>(base, acc, hhh, hhl, x);
  accel_tri<MORSE>(S, L, T, x[0], x[1], acc[5][0], acc[5][1], s_own);
  stage_x2<7>(base, acc, hh, xn);
  accel_tri<MORSE>(S, L, T, xn[0], xn[1], acc[6][0], acc[6][1], s_own);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    double vb = kT3.b[1] * acc[0][i];
#pragma unroll
    for (int q = 3; q <= 6; ++q) vb = fma(kT3.b[q], acc[q - 1][i], vb);
    vn[i] = fma(h, vb, vel[i]);
    // (e^T A)_2 = e_2 = 0 and (e^T A)_7 = 0: a_2 never enters, a_7 only ev
    float es, ec, rs, rc, ah, al;
    split_ff(acc[0][i], ah, al);
    ff_dot_first(es, ec, kTff3.e[1].hi, kTff3.e[1].lo, ah, al);
    ff_dot_first(rs, rc, kTff3.ea[1].hi, kTff3.ea[1].lo, ah, al);
#pragma unroll
    for (int q = 3; q <= 7; ++q) {
      split_ff(acc[q - 1][i], ah, al);
      ff_dot_acc(es, ec, kTff3.e[q].hi, kTff3.e[q].lo, ah, al);
      if (!dpEAZero(q)) ff_dot_acc(rs, rc, kTff3.ea[q].hi, kTff3.ea[q].lo, ah, al);
    }
    ev[i] = es + ec;
    er[i] = rs + rc;
  }
}

// A trajectory's state in one lane of its triplet: components j of both
// Jacobi vectors (index 0: rho1, 1: rho2), their velocities P / mu and the
// stage accelerations; the scalars are the same in the three lanes.
struct TriLane {
  double rho[2], vel[2];
  double acc[7][2];
  double t, h, tmax;
  int nacc, nrej, calls, status;
  float atv[2];            // atol / mu of the two velocity blocks (FP32)
  bool rejected;
};

__device__ __forceinline__ bool runnable(int st) {
  return st == QCAMS_LANE_READY || st == QCAMS_LANE_RUNNING;
}

// Starting step (Hairer, Norsett & Wanner, Solving ODEs I, Sec. II.4, as
// SciPy's solve_ivp takes it), the norms summed over the triplet.
template <bool MORSE>
__device__ double initial_step_tri(const DevSys& S, const Tri& L, const double* __restrict__ T,
                                   const TriLane& X, double rtol, double atol) {
  const double atv[2] = {atol * S.inv_mu12, atol * S.inv_mu123};
  double d0 = 0.0, d1 = 0.0;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const double scr = atol + fabs(X.rho[i]) * rtol;
    const double scv = atv[i] + fabs(X.vel[i]) * rtol;
    const double q0 = X.rho[i] / scr, q1 = X.vel[i] / scv;
    d0 += q0 * q0 + q1 * q1;
    const double p0 = X.vel[i] / scr, p1 = X.acc[0][i] / scv;
    d1 += p0 * p0 + p1 * p1;
  }
  d0 = sqrt(tri_sum(d0, L.base) / 12.0);
  d1 = sqrt(tri_sum(d1, L.base) / 12.0);
  const double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
  double a1[2], s_dummy;
  accel_tri<MORSE>(S, L, T, fma(h0, X.vel[0], X.rho[0]), fma(h0, X.vel[1], X.rho[1]), a1[0],
                   a1[1], s_dummy);
  double d2 = 0.0;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const double scr = atol + fabs(X.rho[i]) * rtol;
    const double scv = atv[i] + fabs(X.vel[i]) * rtol;
    const double p0 = h0 * X.acc[0][i] / scr, p1 = (a1[i] - X.acc[0][i]) / scv;
    d2 += p0 * p0 + p1 * p1;
  }
  d2 = sqrt(tri_sum(d2, L.base) / 12.0) / h0;
  const double h1 = (d1 <= 1e-15 && d2 <= 1e-15) ? fmax(1e-6, h0 * 1e-3)
                                                 : pow(0.01 / fmax(d1, d2), 0.2);
  return fmin(100.0 * h0, h1);
}

// One adaptive step attempt with SciPy's RK45 rules, as integrate.cu's
// lane_attempt: RMS error norm with scale atol + rtol max(|y_n|, |y_n+1|)
// (FP32, from 20-bit magnitudes), accept iff norm < 1, new step
// h clamp(0.9 norm^(-1/5), 0.2, 10) with no growth right after a rejection,
// then the stop rules on the accepted state (Sec. 3.1).  Lanes whose
// trajectory is not running execute it with their state frozen.
template <bool MORSE>
__device__ __forceinline__ void attempt_tri(const DevSys& S, const Tri& L, const DevShape* shapes,
                                            int sid, const IntegParams& ip,
                                            const double* __restrict__ T, TriLane& X) {
  bool go = X.status == QCAMS_LANE_RUNNING;
  {
    const int eh = (__double2hiint(X.h) >> 20) & 0x7ff;
    const int et = (__double2hiint(X.t) >> 20) & 0x7ff;
    const bool fail_h = go && (et - eh >= 49 || eh == 0);
    X.status = fail_h ? QCAMS_LANE_FAIL_HMIN : X.status;
    go = go && !fail_h;
  }
  double xn[2], vn[2], s_new;
  float er[2], ev[2];
  dp_step_tri<MORSE>(S, L, T, X.rho, X.vel, X.acc, X.h, xn, vn, er, ev, s_new);
  unsigned bad = 0, ignore = 0;
  float part = 0.f;
  const float rt = ip.rtol_f, at = ip.atol_f;
  const float hf = mag_f(X.h, ignore), hhf = hf * hf;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float scr = fmaf(rt, fmaxf(mag_f(X.rho[i], ignore), mag_f(xn[i], ignore)), at);
    const float qr = err_mag(er[i], bad) * hhf * rcp_approx(scr);
    part = fmaf(qr, qr, part);
    const float scv = fmaf(rt, fmaxf(mag_f(X.vel[i], ignore), mag_f(vn[i], ignore)), X.atv[i]);
    const float qv = err_mag(ev[i], bad) * hf * rcp_approx(scv);
    part = fmaf(qv, qv, part);
  }
  const float en2 = tri_sum(part, L.base) * (1.0f / 12.0f);
  bad = tri_or(bad, L.base);
  X.calls += go ? 1 : 0;
  X.status = (go && bad) ? QCAMS_LANE_FAIL_NAN : X.status;
  go = go && !bad;
  const float fac = 0.9f * pow_m01(en2);
  const bool accept = go && en2 < 1.0f;
  float fa = (en2 == 0.0f) ? 10.0f : fminf(10.0f, fac);
  fa = X.rejected ? fminf(1.0f, fa) : fa;
  const float f = accept ? fa : fmaxf(0.2f, fac);
  const double tn = X.t + X.h;
  X.t = accept ? tn : X.t;
  X.h = go ? X.h * static_cast<double>(f) : X.h;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    X.rho[i] = accept ? xn[i] : X.rho[i];
    X.vel[i] = accept ? vn[i] : X.vel[i];
    X.acc[0][i] = accept ? X.acc[6][i] : X.acc[0][i];
  }
  X.nacc += accept ? 1 : 0;
  X.nrej += (go && !accept) ? 1 : 0;
  X.rejected = go ? !accept : X.rejected;
  // stop rules on the accepted state, reduced over the triplet
  const long long smax = tri_max(dbits(s_new), L.base);
  const float radial = tri_sum(signed_f(X.rho[1]) * signed_f(X.vel[1]), L.base);
  unsigned collapse = 0;
  if (!MORSE)
    collapse = (L.q.kind == QCAMS_BUCK && dbits(s_new) < dbits(shapes[sid * 3 + L.j].r_b2)) ? 1u : 0u;
  collapse = tri_or(collapse, L.base);
  int st = X.status;
  st = (accept && dbits(X.t) >= dbits(X.tmax)) ? QCAMS_LANE_DONE_TMAX : st;
  st = (accept && smax > dbits(ip.r_stop2) && radial > 0.0f) ? QCAMS_LANE_DONE_RSTOP : st;
  st = (accept && collapse) ? QCAMS_LANE_FAIL_COLLAPSE : st;
  st = (go && st == QCAMS_LANE_RUNNING && (long long)(X.nacc + X.nrej) >= ip.max_steps)
           ? QCAMS_LANE_FAIL_MAXSTEPS : st;
  X.status = st;
}

// One warp per block, ten trajectories per warp (lanes 3k .. 3k + 2 for
// trajectory 10 w + k of warp w), no refill: every lane runs until the last
// trajectory of its warp is done.
template <bool MORSE>
__global__ void __launch_bounds__(kTriBlock) k_integrate_tri(SysSet sys, const DevShape* shapes,
                                                             IntegParams ip, DevBatch B,
                                                             unsigned long long* counters) {
  __shared__ double sT[kExpTableSize];
  load_exp_table(sT);
  const int lane = threadIdx.x & 31;
  Tri L;
  L.j = lane < 30 ? lane % 3 : lane - 30;
  L.base = lane < 30 ? lane - L.j : 27;
  const int64_t i =
      ((int64_t)blockIdx.x * (kTriBlock / 32) + (threadIdx.x >> 5)) * kTriPerWarp + L.base / 3;
  const bool owner = lane < 30 && i < B.n;   // stores its components
  const int64_t ir = i < B.n ? i : B.n - 1;  // lanes past the batch mirror its last trajectory
  const int status0 = B.status[ir];
  int sid = B.sys_id[ir];
  const bool sid_ok = sid >= 0 && sid < sys.n;
  if (owner && L.j == 0 && runnable(status0) && !sid_ok) B.status[i] = QCAMS_LANE_INVALID;
  const bool active = owner && runnable(status0) && sid_ok;
  if (!sid_ok) sid = 0;   // keep the frozen lanes' arithmetic defined
  const DevSys& S = sys.s[sid];
  L.q = S.pair[L.j];
  L.kf = MORSE ? S.kf_morse[L.j] : S.kf[L.j];
  L.kh = L.j == 0 ? 0.0 : (MORSE ? S.kf_morse[2 + L.j] : S.kf[2 + L.j]);

  TriLane X;
  X.rho[0] = B.y[L.j][ir];
  X.rho[1] = B.y[3 + L.j][ir];
  X.vel[0] = B.y[6 + L.j][ir] * S.inv_mu12;
  X.vel[1] = B.y[9 + L.j][ir] * S.inv_mu123;
  X.t = B.t[ir];
  X.h = B.h[ir];
  X.tmax = ip.t_stop * B.t_scale[ir];
  X.nacc = B.nsteps[ir];
  X.nrej = B.nrej[ir];
  X.calls = 0;
  X.rejected = false;
  X.status = active ? QCAMS_LANE_RUNNING : QCAMS_LANE_INVALID;
  X.atv[0] = (float)(ip.atol * S.inv_mu12);
  X.atv[1] = (float)(ip.atol * S.inv_mu123);
  double s_dummy;
  accel_tri<MORSE>(S, L, sT, X.rho[0], X.rho[1], X.acc[0][0], X.acc[0][1], s_dummy);
  unsigned long long rhs = active ? 1 : 0, steps = 0;
  const bool need_h = active && !(X.h > 0.0);
  if (__any_sync(FULL, need_h)) {
    const double h0 = initial_step_tri<MORSE>(S, L, sT, X, ip.rtol, ip.atol);
    X.h = need_h ? h0 : X.h;
    rhs += need_h ? 1 : 0;
  }
  while (__any_sync(FULL, X.status == QCAMS_LANE_RUNNING))
    attempt_tri<MORSE>(S, L, shapes, sid, ip, sT, X);
  if (active) {
    B.y[L.j][i] = X.rho[0];
    B.y[3 + L.j][i] = X.rho[1];
    B.y[6 + L.j][i] = X.vel[0] * S.mu12;
    B.y[9 + L.j][i] = X.vel[1] * S.mu123;
    if (L.j == 0) {
      B.t[i] = X.t;
      B.h[i] = X.h;
      B.status[i] = static_cast<uint8_t>(X.status);
      B.nsteps[i] = X.nacc;
      B.nrej[i] = X.nrej;
    }
  }
  // counters per trajectory, from its component-0 lane
  rhs = (active && L.j == 0) ? rhs + 6ull * X.calls : 0;
  steps = (active && L.j == 0) ? (unsigned long long)X.calls : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rhs += __shfl_xor_sync(FULL, rhs, o);
    steps += __shfl_xor_sync(FULL, steps, o);
  }
  if (lane == 0) {
    atomicAdd(&counters[0], rhs);
    atomicAdd(&counters[1], steps);
  }
}

}  // namespace

cudaError_t launch_integrate_tri(const SysSet& sys, const DevShape* shapes, const IntegParams& ip,
                                 const DevBatch& b, unsigned long long* counters,
                                 cudaStream_t st, bool all_morse) {
  if (b.n == 0) return cudaSuccess;
  const long long warps = (b.n + kTriPerWarp - 1) / kTriPerWarp;
  const unsigned grid = (unsigned)((warps + kTriBlock / 32 - 1) / (kTriBlock / 32));
  if (all_morse)
    k_integrate_tri<true><<<grid, kTriBlock, 0, st>>>(sys, shapes, ip, b, counters);
  else
    k_integrate_tri<false><<<grid, kTriBlock, 0, st>>>(sys, shapes, ip, b, counters);
  return cudaGetLastError();
}

}  // namespace qcams
