// FP64 trajectory integrator for small batches: three or six lanes per
// trajectory.
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
// one-thread-per-trajectory kernel.  Here a group of G lanes carries one
// trajectory: each lane holds 6 / G of the six position components (and
// the matching velocities and stage accelerations) and evaluates the force
// of pair c mod 3 (AB, BC, CA) of its lane index c.
//   G = 3: lane j holds component j of both Jacobi vectors; a step takes
//          183 warp-wide FP64 instructions, 10 trajectories a warp.
//   G = 6: lane c holds one component (c < 3: rho1, else rho2), the two
//          halves of the group evaluate the three pair forces twice; 152
//          instructions a step, 5 trajectories a warp.
// The group exchanges pair-vector components, the pair force factors and
// the error norm's partial sums by warp shuffles.  Large batches belong
// to the one-thread kernels, which carry 32 trajectories a warp.
//
// Every quantity the step control and the stop rules decide on (error norm,
// largest pair distance, radial velocity, collapse) is reduced in the same
// lane order in all lanes of a group, so they take identical decisions.
// The lanes left over at the end of a warp repeat the first lanes of its
// last group and store nothing; a lane whose trajectory is done or absent
// keeps executing the warp's instructions (FP64 costs the same either way)
// with its state frozen, so every shuffle runs on the full warp.
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
constexpr int kGrpBlock = 32;   // one warp per block: small batches spread over the SMs

// A lane's place in its group and the constants of its pair.
template <int G>
struct Grp {
  static constexpr int K = 6 / G;          // position components per lane
  static constexpr int PER_WARP = 32 / G;  // trajectories per warp
  int c;        // lane index in the group, 0 .. G-1
  int j;        // pair index c mod 3 (0 = AB, 1 = BC, 2 = CA)
  int base;     // lane of group index 0
  DevPair q;    // pair j of the trajectory's system
  double kf;    // dP1-force factor of pair j (f_j = kf u_j)
  double kh;    // dP2-force factor of pair j (h_1, h_2; 0 for pair AB)
  // global position component (0-2: rho1, 3-5: rho2) of local component k
  __device__ __forceinline__ int comp(int k) const { return G == 3 ? (k == 0 ? j : 3 + j) : c; }
};

// Sum over the group of a per-lane value, in lane order (identical in all
// lanes of the group).
template <int G, typename V>
__device__ __forceinline__ V grp_sum(V v, int base) {
  V s = __shfl_sync(FULL, v, base);
#pragma unroll
  for (int k = 1; k < G; ++k) s += __shfl_sync(FULL, v, base + k);
  return s;
}
template <int G>
__device__ __forceinline__ unsigned grp_or(unsigned v, int base) {
  unsigned s = 0;
#pragma unroll
  for (int k = 0; k < G; ++k) s |= __shfl_sync(FULL, v, base + k);
  return s;
}
template <int G>
__device__ __forceinline__ long long grp_max(long long v, int base) {
  long long s = __shfl_sync(FULL, v, base);
#pragma unroll
  for (int k = 1; k < G; ++k) s = max(s, __shfl_sync(FULL, v, base + k));
  return s;
}

// The lane's acceleration components (dP1/dt / mu12 or dP2/dt / mu123 for
// its position components x) and the squared distance of pair j.  The pair
// vectors are those of accel() in integrate.cu:
//   r_AB = rho1,  r_BC = rho2 - cB rho1,  r_CA = rho2 + cA rho1.
// Each lane forms component j of the three pair vectors (with G = 6, from
// its own component and its partner's across the two halves), gathers
// components j+1, j+2 of pair j's vector from the lanes holding them in its
// half (each sender choosing the pair its receiver needs), forms the
// squared distance with one multiply and two FMAs, evaluates
// u_j = V'(r_j)/r_j, and the group exchanges f_j = kf u_j and h_j = kh u_j.
template <bool MORSE, int G>
__device__ __forceinline__ void accel_grp(const DevSys& S, const Grp<G>& L,
                                          const double* __restrict__ T, const double* x,
                                          double* a, double& s_own) {
  double x1, x2;
  if (G == 3) {
    x1 = x[0];
    x2 = x[1];
  } else {
    const double other = __shfl_sync(FULL, x[0], L.base + (L.c + 3) % 6);
    x1 = L.c < 3 ? x[0] : other;
    x2 = L.c < 3 ? other : x[0];
  }
  const double rab = x1, rbc = fma(-S.cB, x1, x2), rca = fma(S.cA, x1, x2);
  const int half = L.base + (L.c - L.j);   // lane of component 0 in this lane's half
  double rk[2];
#pragma unroll
  for (int r = 1; r <= 2; ++r) {
    // in round r a lane receives from the lane of component (j + r) mod 3,
    // which sends its component of pair (its j - r) mod 3: the receiver's pair
    const int want = (L.j + 3 - r) % 3;
    const double v = want == 0 ? rab : (want == 1 ? rbc : rca);
    rk[r - 1] = __shfl_sync(FULL, v, half + (L.j + r) % 3);
  }
  const double rj = L.j == 0 ? rab : (L.j == 1 ? rbc : rca);
  const double s = fma(rj, rj, fma(rk[0], rk[0], rk[1] * rk[1]));
  s_own = s;
  const double u = pair_u<MORSE>(L.q, s, T);
  const double f = L.kf * u, h = L.kh * u;
  const double f0 = __shfl_sync(FULL, f, L.base), f1 = __shfl_sync(FULL, f, L.base + 1),
               f2 = __shfl_sync(FULL, f, L.base + 2);
  const double h1 = __shfl_sync(FULL, h, L.base + 1), h2 = __shfl_sync(FULL, h, L.base + 2);
  if (G == 3) {
    a[0] = fma(f0, rab, fma(f1, rbc, f2 * rca));
    a[1] = fma(h1, rbc, h2 * rca);
  } else {
    const bool first = L.c < 3;
    a[0] = fma(first ? f0 : 0.0, rab, fma(first ? f1 : h1, rbc, (first ? f2 : h2) * rca));
  }
}

// Stage positions for the lane's K components, the formulas of
// integrate.cu's stage_x / stage_x_ff.  Stage s from base = rho + h c_s v,
// FP64 sums (stages 2, 3 and 7).
template <int s, int K>
__device__ __forceinline__ void stage_xk(const double* base, const double (*acc)[K], double hh,
                                         double* x) {
  double w[s > 2 ? s - 2 : 1];
#pragma unroll
  for (int q = 1; q <= s - 2; ++q) w[q - 1] = dpA2Zero(s, q) ? 0.0 : hh * kT3.a2[s][q];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    double xi = base[i];
#pragma unroll
    for (int q = 1; q <= s - 2; ++q)
      if (!dpA2Zero(s, q)) xi = fma(w[q - 1], acc[q - 1][i], xi);
    x[i] = xi;
  }
}
// Stages 4-6: the acceleration correction as a float-float dot product
// added to the FP64 base with one DADD.
template <int s, int K>
__device__ __forceinline__ void stage_xk_ff(const double* base, const double (*acc)[K], float hhh,
                                            float hhl, double* x) {
  float wh[s - 2], wl[s - 2];
#pragma unroll
  for (int q = 1; q <= s - 2; ++q) {
    const FFc c = kTff3.a2[s][q];
    wh[q - 1] = __fmul_rn(hhh, c.hi);
    wl[q - 1] = fmaf(hhh, c.hi, -wh[q - 1]) + fmaf(hhh, c.lo, hhl * c.hi);
  }
#pragma unroll
  for (int i = 0; i < K; ++i) {
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

// One Dormand-Prince step of size h for the lane's components, with
// acc[0] = a(rho).  On return acc[1..6] hold the stage accelerations, xn /
// vn the 5th-order solution, er / ev the embedded error estimates divided by
// h^2 and h, s_own the squared distance of pair j at xn (per component the
// arithmetic of integrate.cu's dp_step).
template <bool MORSE, int G>
__device__ __forceinline__ void dp_step_grp(const DevSys& S, const Grp<G>& L,
                                            const double* __restrict__ T, const double* rho,
                                            const double* vel, double (*acc)[Grp<G>::K],
                                            double h, double* xn, double* vn, float* er,
                                            float* ev, double& s_own) {
  constexpr int K = Grp<G>::K;
  const double hh = h * h;
  float hhh, hhl;
  split_ff(hh, hhh, hhl);
  double x[K], base[K];
#pragma unroll
  for (int i = 0; i < K; ++i) base[i] = fma(h * dpC(2), vel[i], rho[i]);
  stage_xk<2, K>(base, acc, hh, x);
  accel_grp<MORSE, G>(S, L, T, x, acc[1], s_own);
#pragma unroll
  for (int i = 0; i < K; ++i) base[i] = fma(h * dpC(3), vel[i], rho[i]);
  stage_xk<3, K>(base, acc, hh, x);
  accel_grp<MORSE, G>(S, L, T, x, acc[2], s_own);
#pragma unroll
  for (int i = 0; i < K; ++i) base[i] = fma(h * dpC(4), vel[i], rho[i]);
  stage_xk_ff<4, K>(base, acc, hhh, hhl, x);
  accel_grp<MORSE, G>(S, L, T, x, acc[3], s_own);
#pragma unroll
  for (int i = 0; i < K; ++i) base[i] = fma(h * dpC(5), vel[i], rho[i]);
  stage_xk_ff<5, K>(base, acc, hhh, hhl, x);
  accel_grp<MORSE, G>(S, L, T, x, acc[4], s_own);
#pragma unroll
  for (int i = 0; i < K; ++i) base[i] = fma(h, vel[i], rho[i]);   // c_6 = c_7 = 1
  stage_xk_ff<6, K>(base, acc, hhh, hhl, x);
  accel_grp<MORSE, G>(S, L, T, x, acc[5], s_own);
  stage_xk<7, K>(base, acc, hh, xn);
  accel_grp<MORSE, G>(S, L, T, xn, acc[6], s_own);
#pragma unroll
  for (int i = 0; i < K; ++i) {
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

// A trajectory's state in one lane of its group: the lane's K position
// components, their velocities P / mu and stage accelerations; the scalars
// are the same in all lanes of the group.
template <int K>
struct GrpLane {
  double rho[K], vel[K];
  double acc[7][K];
  double t, h, tmax;
  double inv_mu[K];        // 1 / mu12 or 1 / mu123 of each component
  float atv[K];            // atol / mu of each component (FP32)
  int nacc, nrej, calls, status;
  bool rejected;
};

__device__ __forceinline__ bool runnable(int st) {
  return st == QCAMS_LANE_READY || st == QCAMS_LANE_RUNNING;
}

// Starting step (Hairer, Norsett & Wanner, Solving ODEs I, Sec. II.4, as
// SciPy's solve_ivp takes it), the norms summed over the group.
template <bool MORSE, int G>
__device__ double initial_step_grp(const DevSys& S, const Grp<G>& L, const double* __restrict__ T,
                                   const GrpLane<Grp<G>::K>& X, double rtol, double atol) {
  constexpr int K = Grp<G>::K;
  double d0 = 0.0, d1 = 0.0;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const double scr = atol + fabs(X.rho[i]) * rtol;
    const double scv = atol * X.inv_mu[i] + fabs(X.vel[i]) * rtol;
    const double q0 = X.rho[i] / scr, q1 = X.vel[i] / scv;
    d0 += q0 * q0 + q1 * q1;
    const double p0 = X.vel[i] / scr, p1 = X.acc[0][i] / scv;
    d1 += p0 * p0 + p1 * p1;
  }
  d0 = sqrt(grp_sum<G>(d0, L.base) / 12.0);
  d1 = sqrt(grp_sum<G>(d1, L.base) / 12.0);
  const double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
  double x1[K], a1[K], s_dummy;
#pragma unroll
  for (int i = 0; i < K; ++i) x1[i] = fma(h0, X.vel[i], X.rho[i]);
  accel_grp<MORSE, G>(S, L, T, x1, a1, s_dummy);
  double d2 = 0.0;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const double scr = atol + fabs(X.rho[i]) * rtol;
    const double scv = atol * X.inv_mu[i] + fabs(X.vel[i]) * rtol;
    const double p0 = h0 * X.acc[0][i] / scr, p1 = (a1[i] - X.acc[0][i]) / scv;
    d2 += p0 * p0 + p1 * p1;
  }
  d2 = sqrt(grp_sum<G>(d2, L.base) / 12.0) / h0;
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
template <bool MORSE, int G>
__device__ __forceinline__ void attempt_grp(const DevSys& S, const Grp<G>& L,
                                            const DevShape* shapes, int sid,
                                            const IntegParams& ip, const double* __restrict__ T,
                                            GrpLane<Grp<G>::K>& X) {
  constexpr int K = Grp<G>::K;
  bool go = X.status == QCAMS_LANE_RUNNING;
  {
    const int eh = (__double2hiint(X.h) >> 20) & 0x7ff;
    const int et = (__double2hiint(X.t) >> 20) & 0x7ff;
    const bool fail_h = go && (et - eh >= 49 || eh == 0);
    X.status = fail_h ? QCAMS_LANE_FAIL_HMIN : X.status;
    go = go && !fail_h;
  }
  double xn[K], vn[K], s_new;
  float er[K], ev[K];
  dp_step_grp<MORSE, G>(S, L, T, X.rho, X.vel, X.acc, X.h, xn, vn, er, ev, s_new);
  unsigned bad = 0, ignore = 0;
  float part = 0.f;
  const float rt = ip.rtol_f, at = ip.atol_f;
  const float hf = mag_f(X.h, ignore), hhf = hf * hf;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const float scr = fmaf(rt, fmaxf(mag_f(X.rho[i], ignore), mag_f(xn[i], ignore)), at);
    const float qr = err_mag(er[i], bad) * hhf * rcp_approx(scr);
    part = fmaf(qr, qr, part);
    const float scv = fmaf(rt, fmaxf(mag_f(X.vel[i], ignore), mag_f(vn[i], ignore)), X.atv[i]);
    const float qv = err_mag(ev[i], bad) * hf * rcp_approx(scv);
    part = fmaf(qv, qv, part);
  }
  const float en2 = grp_sum<G>(part, L.base) * (1.0f / 12.0f);
  bad = grp_or<G>(bad, L.base);
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
  for (int i = 0; i < K; ++i) {
    X.rho[i] = accept ? xn[i] : X.rho[i];
    X.vel[i] = accept ? vn[i] : X.vel[i];
    X.acc[0][i] = accept ? X.acc[6][i] : X.acc[0][i];
  }
  X.nacc += accept ? 1 : 0;
  X.nrej += (go && !accept) ? 1 : 0;
  X.rejected = go ? !accept : X.rejected;
  // stop rules on the accepted state, reduced over the group
  const long long smax = grp_max<G>(dbits(s_new), L.base);
  float rad = 0.0f;   // rho2 . P2 / mu123 from the lane's rho2 components
#pragma unroll
  for (int i = 0; i < K; ++i)
    rad += L.comp(i) >= 3 ? signed_f(X.rho[i]) * signed_f(X.vel[i]) : 0.0f;
  const float radial = grp_sum<G>(rad, L.base);
  unsigned collapse = 0;
  if (!MORSE)
    collapse = (L.q.kind == QCAMS_BUCK && dbits(s_new) < dbits(shapes[sid * 3 + L.j].r_b2)) ? 1u : 0u;
  collapse = grp_or<G>(collapse, L.base);
  int st = X.status;
  st = (accept && dbits(X.t) >= dbits(X.tmax)) ? QCAMS_LANE_DONE_TMAX : st;
  st = (accept && smax > dbits(ip.r_stop2) && radial > 0.0f) ? QCAMS_LANE_DONE_RSTOP : st;
  st = (accept && collapse) ? QCAMS_LANE_FAIL_COLLAPSE : st;
  st = (go && st == QCAMS_LANE_RUNNING && (long long)(X.nacc + X.nrej) >= ip.max_steps)
           ? QCAMS_LANE_FAIL_MAXSTEPS : st;
  X.status = st;
}

// One warp per block, 32 / G trajectories per warp (lanes G k .. G k + G - 1
// for trajectory (32 / G) w + k of warp w), no refill: every lane runs
// until the last trajectory of its warp is done.
template <bool MORSE, int G>
__global__ void __launch_bounds__(kGrpBlock) k_integrate_grp(SysSet sys, const DevShape* shapes,
                                                             IntegParams ip, DevBatch B,
                                                             unsigned long long* counters) {
  constexpr int K = Grp<G>::K, PER_WARP = Grp<G>::PER_WARP;
  __shared__ double sT[kExpTableSize];
  load_exp_table(sT);
  const int lane = threadIdx.x & 31;
  const int used = PER_WARP * G;   // lanes of whole groups; the rest mirror the last group
  Grp<G> L;
  L.c = lane < used ? lane % G : lane - used;
  L.base = lane < used ? lane - L.c : used - G;
  L.j = L.c % 3;
  const int64_t i =
      ((int64_t)blockIdx.x * (kGrpBlock / 32) + (threadIdx.x >> 5)) * PER_WARP + L.base / G;
  const bool owner = lane < used && i < B.n;   // stores its components
  const int64_t ir = i < B.n ? i : B.n - 1;    // lanes past the batch mirror its last trajectory
  const int status0 = B.status[ir];
  int sid = B.sys_id[ir];
  const bool sid_ok = sid >= 0 && sid < sys.n;
  if (owner && L.c == 0 && runnable(status0) && !sid_ok) B.status[i] = QCAMS_LANE_INVALID;
  const bool active = owner && runnable(status0) && sid_ok;
  if (!sid_ok) sid = 0;   // keep the frozen lanes' arithmetic defined
  const DevSys& S = sys.s[sid];
  L.q = S.pair[L.j];
  L.kf = MORSE ? S.kf_morse[L.j] : S.kf[L.j];
  L.kh = L.j == 0 ? 0.0 : (MORSE ? S.kf_morse[2 + L.j] : S.kf[2 + L.j]);

  GrpLane<K> X;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int cg = L.comp(k);
    X.inv_mu[k] = cg < 3 ? S.inv_mu12 : S.inv_mu123;
    X.atv[k] = (float)(ip.atol * X.inv_mu[k]);
    X.rho[k] = B.y[cg][ir];
    X.vel[k] = B.y[6 + cg][ir] * X.inv_mu[k];
  }
  X.t = B.t[ir];
  X.h = B.h[ir];
  X.tmax = ip.t_stop * B.t_scale[ir];
  X.nacc = B.nsteps[ir];
  X.nrej = B.nrej[ir];
  X.calls = 0;
  X.rejected = false;
  X.status = active ? QCAMS_LANE_RUNNING : QCAMS_LANE_INVALID;
  double s_dummy;
  accel_grp<MORSE, G>(S, L, sT, X.rho, X.acc[0], s_dummy);
  unsigned long long rhs = active ? 1 : 0, steps = 0;
  const bool need_h = active && !(X.h > 0.0);
  if (__any_sync(FULL, need_h)) {
    const double h0 = initial_step_grp<MORSE, G>(S, L, sT, X, ip.rtol, ip.atol);
    X.h = need_h ? h0 : X.h;
    rhs += need_h ? 1 : 0;
  }
  while (__any_sync(FULL, X.status == QCAMS_LANE_RUNNING))
    attempt_grp<MORSE, G>(S, L, shapes, sid, ip, sT, X);
  if (active) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int cg = L.comp(k);
      B.y[cg][i] = X.rho[k];
      B.y[6 + cg][i] = X.vel[k] * (cg < 3 ? S.mu12 : S.mu123);
    }
    if (L.c == 0) {
      B.t[i] = X.t;
      B.h[i] = X.h;
      B.status[i] = static_cast<uint8_t>(X.status);
      B.nsteps[i] = X.nacc;
      B.nrej[i] = X.nrej;
    }
  }
  // counters per trajectory, from its group-index-0 lane
  rhs = (active && L.c == 0) ? rhs + 6ull * X.calls : 0;
  steps = (active && L.c == 0) ? (unsigned long long)X.calls : 0;
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

template <int G>
cudaError_t launch_grp(const SysSet& sys, const DevShape* shapes, const IntegParams& ip,
                       const DevBatch& b, unsigned long long* counters, cudaStream_t st,
                       bool all_morse) {
  const long long warps = (b.n + Grp<G>::PER_WARP - 1) / Grp<G>::PER_WARP;
  const unsigned grid = (unsigned)((warps + kGrpBlock / 32 - 1) / (kGrpBlock / 32));
  if (all_morse)
    k_integrate_grp<true, G><<<grid, kGrpBlock, 0, st>>>(sys, shapes, ip, b, counters);
  else
    k_integrate_grp<false, G><<<grid, kGrpBlock, 0, st>>>(sys, shapes, ip, b, counters);
  return cudaGetLastError();
}

}  // namespace

cudaError_t grouped_func_info(int lanes, bool all_morse, int* regs, int* blocks_per_sm) {
  cudaFuncAttributes a;
  cudaError_t e = cudaErrorInvalidValue;
#define QCAMS_GRP_INFO(M, G)                                                               \
  e = cudaFuncGetAttributes(&a, k_integrate_grp<M, G>);                                    \
  if (e == cudaSuccess)                                                                    \
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_integrate_grp<M, G>, \
                                                      kGrpBlock, 0)
  if (lanes == 3) {
    if (all_morse) { QCAMS_GRP_INFO(true, 3); } else { QCAMS_GRP_INFO(false, 3); }
  } else if (lanes == 6) {
    if (all_morse) { QCAMS_GRP_INFO(true, 6); } else { QCAMS_GRP_INFO(false, 6); }
  }
#undef QCAMS_GRP_INFO
  if (e == cudaSuccess) *regs = a.numRegs;
  return e;
}

cudaError_t launch_integrate_grouped(const SysSet& sys, const DevShape* shapes,
                                     const IntegParams& ip, const DevBatch& b, int lanes,
                                     unsigned long long* counters, cudaStream_t st,
                                     bool all_morse) {
  if (b.n == 0) return cudaSuccess;
  if (lanes == 3) return launch_grp<3>(sys, shapes, ip, b, counters, st, all_morse);
  if (lanes == 6) return launch_grp<6>(sys, shapes, ip, b, counters, st, all_morse);
  return cudaErrorInvalidValue;
}

}  // namespace qcams
