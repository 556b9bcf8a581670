// FP32 trajectory integrator with compensated (Kahan) state updates.
//
// Same method as the FP64 integrator (Hamilton's equations in Jacobi
// coordinates, Sec. 2 Eqs. 3-4; Dormand-Prince 5(4) with SciPy's RK45 step
// control, Sec. 3.2; stop rules of Sec. 3.1) in single precision, for the
// FP32 study of the sweep.  GB300 runs FP32 at 64x its FP64 rate, so this
// path trades accuracy (tolerances ~1e-6) for throughput.
//
//  * Stages, forces and the error norm are FP32 (the hardware 1/sqrt and
//    2^x of x log2 e, relative error below 2 + 1.2 |x| ulp; the
//    exponentials of the force law have |x| < 2 where the force matters and
//    up to ~35 only for pairs far apart, whose forces are negligible).
//  * Each step adds a small increment to a large state (|rho| ~ 30 bohr,
//    increments ~1e-2), so plain FP32 accumulation would lose ~1e-7 |y| per
//    step.  Positions and velocities are therefore kept as Kahan pairs
//    (value, compensation): y_true = y - c, and every update y += d folds the
//    rounding error of the previous updates back in (Kahan, CACM 8 (1965) 40).
//  * Time is FP64 (one add per step).  Initial conditions, the level table,
//    the energy bookkeeping and the product analysis stay FP64: the kernel
//    loads the FP64 state as (float, compensation) and stores y - c in FP64.
#include <cuda_runtime.h>

#include "dp5_tableau.cuh"
#include "qcams_device.cuh"
#include "qcams_internal.h"

namespace qcams {
namespace {

struct RknTabF {
  float a2[8][8], c[8], b[8], e[8], ea[8];
};
__host__ __device__ constexpr RknTabF make_rkn_tab_f() {
  RknTabF f{};
  for (int s = 1; s <= 7; ++s) {
    f.c[s] = (float)dpC(s);
    f.b[s] = (float)dpB(s);
    f.e[s] = (float)dpE(s);
    f.ea[s] = dpEAZero(s) ? 0.0f : (float)dpEA(s);
    for (int q = 1; q <= 7; ++q) f.a2[s][q] = dpA2Zero(s, q) ? 0.0f : (float)dpA2(s, q);
  }
  return f;
}
__constant__ RknTabF kTf = make_rkn_tab_f();

constexpr unsigned FULL = 0xffffffffu;

// Approximate reciprocal (one MUFU instruction, about 1 ulp): the error norm
// needs only a few significant bits, and the scales it divides by are
// positive and far from the FP32 range limits (atol > 0).
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// 2^x (one MUFU instruction, relative error about 2^-22): the force law's
// exponentials e^y are taken as 2^(y log2 e) with the constants of y
// pre-scaled by log2 e on the host, so no multiply precedes the MUFU.
__device__ __forceinline__ float ex2_approx(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// 1/sqrt(s) (one MUFU instruction, about 1 ulp).  Flush-to-zero: s is a
// squared pair distance, subnormal only for pairs closer than 1e-19 bohr,
// where the lane fails on the infinite force it gets.
__device__ __forceinline__ float rsqrt_approx(float s) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(s));
  return r;
}

// x^(-1/10) for the step-size factor, as 2^(-log2(x) / 10) (two MUFU
// instructions and a multiply).  x = 0 or subnormal gives +inf, which the
// controller caps at the maximum growth factor as it does for a zero norm.
__device__ __forceinline__ float pow_m01(float x) {
  float l, r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(x));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(-0.1f * l));
  return r;
}

// FP32 copies of the per-system constants (built on the host, so the kernel
// never converts doubles in its inner loop).
struct PairF {
  int kind, m, n, pad;
  float c0, c1, c2, c3, c4;
  float l0, l1;   // exponent constants times log2 e: Morse c0, c1; Buckingham
                  // ln(A B) (l0) and B (l1), so that 2^(l0 - l1 r) = A B e^{-B r}
};
struct SysF {
  float cA, cB, inv_mu12, inv_mu123, mu12, mu123;
  float kf[5], kf_morse[5];
  double mu12d, mu123d;
  PairF pair[3];
};
struct SysSetF {
  SysF s[QCAMS_MAX_SYS];
  int n, pad;
};

__device__ __forceinline__ float ipowf_(float x, int n) {
  float r = 1.0f;
  while (n) {
    if (n & 1) r *= x;
    x *= x;
    n >>= 1;
  }
  return r;
}

// u = V'(r)/r (generic) or x (1 - x)/r (all-Morse kernels: the factor
// 2 alpha De is folded into kf_morse)
template <bool MORSE>
__device__ __forceinline__ float pair_u(const PairF& q, float s) {
  const float ri = rsqrt_approx(s);
  const float r = s * ri;
  if (MORSE) {
    const float x = ex2_approx(fmaf(-q.l0, r, q.l1));   // e^{-alpha (r - re)}
    return fmaf(-x, x, x) * ri;
  }
  if (q.kind == QCAMS_MORSE) {   // a Morse pair of a mixed system: V'/r = 2 alpha De x (1 - x) / r
    const float x = ex2_approx(fmaf(-q.l0, r, q.l1));
    return q.c2 * fmaf(-x, x, x) * ri;
  }
  const float ri2 = ri * ri;
  if (q.kind == QCAMS_LJ) {
    if (q.n == 6 && (q.m == 12 || q.m == 8)) {   // shared powers of 1/r^2
      const float ri4 = ri2 * ri2, ri6 = ri4 * ri2;
      const float h = q.m == 12 ? ri6 : ri4;
      return fmaf(q.c3, ri6, -q.c2 * (h * h)) * ri2;
    }
    return (q.c3 * ipowf_(ri, q.n) - q.c2 * ipowf_(ri, q.m)) * ri2;
  }
  // Buckingham: 6 C6 / r^8 - A B e^{-B r} / r
  const float ri4 = ri2 * ri2;
  return fmaf(q.c3, ri4 * ri4, -(ex2_approx(fmaf(-q.l1, r, q.l0)) * ri));
}

template <bool MORSE>
__device__ __forceinline__ void accel(const SysF& S, const float* x, float* a, float* s2) {
  const float rbc0 = fmaf(-S.cB, x[0], x[3]), rbc1 = fmaf(-S.cB, x[1], x[4]),
              rbc2 = fmaf(-S.cB, x[2], x[5]);
  const float rca0 = fmaf(S.cA, x[0], x[3]), rca1 = fmaf(S.cA, x[1], x[4]),
              rca2 = fmaf(S.cA, x[2], x[5]);
  s2[0] = fmaf(x[0], x[0], fmaf(x[1], x[1], x[2] * x[2]));
  s2[1] = fmaf(rbc0, rbc0, fmaf(rbc1, rbc1, rbc2 * rbc2));
  s2[2] = fmaf(rca0, rca0, fmaf(rca1, rca1, rca2 * rca2));
  const float u0 = pair_u<MORSE>(S.pair[0], s2[0]);
  const float u1 = pair_u<MORSE>(S.pair[1], s2[1]);
  const float u2 = pair_u<MORSE>(S.pair[2], s2[2]);
  const float f0 = (MORSE ? S.kf_morse[0] : S.kf[0]) * u0;
  const float f1 = (MORSE ? S.kf_morse[1] : S.kf[1]) * u1;
  const float f2 = (MORSE ? S.kf_morse[2] : S.kf[2]) * u2;
  const float h1 = (MORSE ? S.kf_morse[3] : S.kf[3]) * u1;
  const float h2 = (MORSE ? S.kf_morse[4] : S.kf[4]) * u2;
  a[0] = fmaf(f0, x[0], fmaf(f1, rbc0, f2 * rca0));
  a[1] = fmaf(f0, x[1], fmaf(f1, rbc1, f2 * rca1));
  a[2] = fmaf(f0, x[2], fmaf(f1, rbc2, f2 * rca2));
  a[3] = fmaf(h1, rbc0, h2 * rca0);
  a[4] = fmaf(h1, rbc1, h2 * rca1);
  a[5] = fmaf(h1, rbc2, h2 * rca2);
}

struct Lane32 {
  float rho[6], vel[6];   // state (true value = state - compensation)
  float crho[6], cvel[6]; // Kahan compensations
  float acc[7][6];
  double t, tmax;
  float h;
  float atv[2];
  float rb2[3];           // Buckingham collapse radii squared (0 for other kinds)
  int nacc, nrej, calls, status, sid;
  bool rejected;
};

// One adaptive attempt (SciPy RK45 rules, as in the FP64 integrator), all
// stages in FP32; the accepted increments are added with compensation.
// ONE: the batch has a single system, so its constants are read with a
// compile-time index (constant-bank operands, no per-lane indexed loads).
template <bool MORSE, bool ONE>
__device__ __forceinline__ void attempt(const SysSetF& sys, const IntegParams& ip, Lane32& L) {
  const SysF& S = sys.s[ONE ? 0 : L.sid];
  {
    const int eh = (__float_as_int(L.h) >> 23) & 0xff;
    const int et = (__double2hiint(L.t) >> 20) & 0x7ff;
    if ((et - 1023) - (eh - 127) >= 49 || eh == 0) {
      L.status = QCAMS_LANE_FAIL_HMIN;
      return;
    }
  }
  const float h = L.h, hh = h * h;
  float x[6], s2[3];
#define QCAMS_STAGE(sIdx)                                                            \
  {                                                                                  \
    const float hc = h * (float)dpC(sIdx); /* folded: c_6 = 1 */                     \
    float w[(sIdx) - 2];                                                             \
    _Pragma("unroll") for (int q = 1; q <= (sIdx) - 2; ++q)                          \
        w[q - 1] = hh * kTf.a2[sIdx][q];                                             \
    _Pragma("unroll") for (int i = 0; i < 6; ++i) {                                  \
      float xi = fmaf(hc, L.vel[i], L.rho[i]);                                       \
      _Pragma("unroll") for (int q = 1; q <= (sIdx) - 2; ++q)                        \
          if (!dpA2Zero(sIdx, q)) xi = fmaf(w[q - 1], L.acc[q - 1][i], xi);          \
      x[i] = xi;                                                                     \
    }                                                                                \
    accel<MORSE>(S, x, L.acc[(sIdx) - 1], s2);                                       \
  }
  {  // stage 2: (A^2)_{2q} = 0, no acceleration term
    const float hc = h * (float)dpC(2);
#pragma unroll
    for (int i = 0; i < 6; ++i) x[i] = fmaf(hc, L.vel[i], L.rho[i]);
    accel<MORSE>(S, x, L.acc[1], s2);
  }
  QCAMS_STAGE(3)
  QCAMS_STAGE(4)
  QCAMS_STAGE(5)
  QCAMS_STAGE(6)
#undef QCAMS_STAGE
  // stage 7 = the new state: increment d = h v + h^2 sum (b^T A)_q a_q,
  // compensated sum x7 = rho + (d - c)
  float yr[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    float sum = 0.0f;
#pragma unroll
    for (int q = 1; q <= 5; ++q)
      if (!dpA2Zero(7, q)) sum = fmaf(kTf.a2[7][q], L.acc[q - 1][i], sum);
    const float d = fmaf(hh, sum, h * L.vel[i]);
    yr[i] = d - L.crho[i];
    x[i] = L.rho[i] + yr[i];
  }
  accel<MORSE>(S, x, L.acc[6], s2);
  float dv[6], er[6], ev[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    float vb = kTf.b[1] * L.acc[0][i];
#pragma unroll
    for (int q = 3; q <= 6; ++q) vb = fmaf(kTf.b[q], L.acc[q - 1][i], vb);
    dv[i] = h * vb;
    float e = kTf.e[1] * L.acc[0][i];
#pragma unroll
    for (int q = 3; q <= 7; ++q) e = fmaf(kTf.e[q], L.acc[q - 1][i], e);
    ev[i] = e;   // velocity error / h
    float ea = kTf.ea[1] * L.acc[0][i];
#pragma unroll
    for (int q = 2; q <= 6; ++q)
      if (!dpEAZero(q)) ea = fmaf(kTf.ea[q], L.acc[q - 1][i], ea);
    er[i] = ea;  // position error / h^2
  }
  // the factors h and h^2 multiply the two partial sums of squares once
  float sum_r = 0.0f, sum_v = 0.0f;
  float vn[6], yv[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    yv[i] = dv[i] - L.cvel[i];
    vn[i] = L.vel[i] + yv[i];
    const float scr = fmaf(ip.rtol_f, fmaxf(fabsf(L.rho[i]), fabsf(x[i])), ip.atol_f);
    const float qr = er[i] * rcp_approx(scr);
    const float scv = fmaf(ip.rtol_f, fmaxf(fabsf(L.vel[i]), fabsf(vn[i])), L.atv[i / 3]);
    const float qv = ev[i] * rcp_approx(scv);
    sum_r = fmaf(qr, qr, sum_r);
    sum_v = fmaf(qv, qv, sum_v);
  }
  const float en2 = fmaf(hh, sum_v, (hh * hh) * sum_r) * (1.0f / 12.0f);
  L.calls += 1;
  if (!(en2 == en2)) {   // NaN fails the lane; an overflowing norm just rejects
    L.status = QCAMS_LANE_FAIL_NAN;
    return;
  }
  const float fac = 0.9f * pow_m01(en2);
  const bool accept = en2 < 1.0f;
  float fa = (en2 == 0.0f) ? 10.0f : fminf(10.0f, fac);
  fa = L.rejected ? fminf(1.0f, fa) : fa;
  const float f = accept ? fa : fmaxf(0.2f, fac);
  const double tn = L.t + (double)L.h;
  L.t = accept ? tn : L.t;
  L.h = L.h * f;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const float cr = (x[i] - L.rho[i]) - yr[i];
    const float cv = (vn[i] - L.vel[i]) - yv[i];
    L.crho[i] = accept ? cr : L.crho[i];
    L.cvel[i] = accept ? cv : L.cvel[i];
    L.rho[i] = accept ? x[i] : L.rho[i];
    L.vel[i] = accept ? vn[i] : L.vel[i];
    L.acc[0][i] = accept ? L.acc[6][i] : L.acc[0][i];
  }
  L.nacc += accept ? 1 : 0;
  L.nrej += accept ? 0 : 1;
  L.rejected = !accept;
  const float smax = fmaxf(s2[0], fmaxf(s2[1], s2[2]));
  const float radial = fmaf(L.rho[3], L.vel[3], fmaf(L.rho[4], L.vel[4], L.rho[5] * L.vel[5]));
  bool collapse = false;
  if (!MORSE) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
      collapse |= s2[k] < L.rb2[k];
  }
  int st = L.status;
  st = (accept && __double_as_longlong(L.t) >= __double_as_longlong(L.tmax))
           ? QCAMS_LANE_DONE_TMAX : st;
  st = (accept && smax > (float)ip.r_stop2 && radial > 0.0f) ? QCAMS_LANE_DONE_RSTOP : st;
  st = (accept && collapse) ? QCAMS_LANE_FAIL_COLLAPSE : st;
  st = (st == QCAMS_LANE_RUNNING && (long long)(L.nacc + L.nrej) >= ip.max_steps)
           ? QCAMS_LANE_FAIL_MAXSTEPS : st;
  L.status = st;
}

// Starting step (Hairer, Norsett & Wanner), in FP32.
template <bool MORSE>
__device__ float initial_step(const SysF& S, const Lane32& L, float rtol, float atol) {
  float d0 = 0.f, d1 = 0.f;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const float scr = atol + fabsf(L.rho[i]) * rtol;
    const float scv = L.atv[i / 3] + fabsf(L.vel[i]) * rtol;
    const float q0 = L.rho[i] / scr, q1 = L.vel[i] / scv;
    d0 += q0 * q0 + q1 * q1;
    const float p0 = L.vel[i] / scr, p1 = L.acc[0][i] / scv;
    d1 += p0 * p0 + p1 * p1;
  }
  d0 = sqrtf(d0 / 12.f);
  d1 = sqrtf(d1 / 12.f);
  const float h0 = (d0 < 1e-5f || d1 < 1e-5f) ? 1e-6f : 0.01f * d0 / d1;
  float x1[6], a1[6], s2[3];
#pragma unroll
  for (int i = 0; i < 6; ++i) x1[i] = fmaf(h0, L.vel[i], L.rho[i]);
  accel<MORSE>(S, x1, a1, s2);
  float d2 = 0.f;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const float scr = atol + fabsf(L.rho[i]) * rtol;
    const float scv = L.atv[i / 3] + fabsf(L.vel[i]) * rtol;
    const float p0 = h0 * L.acc[0][i] / scr, p1 = (a1[i] - L.acc[0][i]) / scv;
    d2 += p0 * p0 + p1 * p1;
  }
  d2 = sqrtf(d2 / 12.f) / h0;
  const float h1 = (d1 <= 1e-15f && d2 <= 1e-15f) ? fmaxf(1e-6f, h0 * 1e-3f)
                                                 : powf(0.01f / fmaxf(d1, d2), 0.2f);
  return fminf(100.f * h0, h1);
}

__device__ __forceinline__ bool runnable(int st) {
  return st == QCAMS_LANE_READY || st == QCAMS_LANE_RUNNING;
}

template <bool MORSE, bool ONE>
__device__ bool load(const SysSetF& sys, const DevShape* shapes, const IntegParams& ip,
                     const DevBatch& B, int64_t i, Lane32& L, unsigned long long& rhs) {
  L.status = B.status[i];
  if (!runnable(L.status)) return false;
  L.sid = B.sys_id[i];
  if (L.sid < 0 || L.sid >= sys.n) {
    B.status[i] = QCAMS_LANE_INVALID;
    return false;
  }
  const SysF& S = sys.s[ONE ? 0 : L.sid];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const double r = B.y[k][i];
    const double v = B.y[6 + k][i] * (k < 3 ? 1.0 / S.mu12d : 1.0 / S.mu123d);
    L.rho[k] = (float)r;
    L.crho[k] = (float)((double)L.rho[k] - r);
    L.vel[k] = (float)v;
    L.cvel[k] = (float)((double)L.vel[k] - v);
  }
  L.t = B.t[i];
  L.h = (float)B.h[i];
  L.tmax = ip.t_stop * B.t_scale[i];
  L.nacc = B.nsteps[i];
  L.nrej = B.nrej[i];
  L.calls = 0;
  L.rejected = false;
  L.status = QCAMS_LANE_RUNNING;
  L.atv[0] = ip.atol_f * S.inv_mu12;
  L.atv[1] = ip.atol_f * S.inv_mu123;
#pragma unroll
  for (int k = 0; k < 3; ++k)
    L.rb2[k] = (!MORSE && S.pair[k].kind == QCAMS_BUCK) ? (float)shapes[L.sid * 3 + k].r_b2 : 0.0f;
  float s2[3];
  accel<MORSE>(S, L.rho, L.acc[0], s2);
  rhs += 1;
  if (!(L.h > 0.0f)) {
    L.h = initial_step<MORSE>(S, L, ip.rtol_f, ip.atol_f);
    rhs += 1;
  }
  return true;
}

template <bool ONE>
__device__ void store(const SysSetF& sys, const DevBatch& B, int64_t i, const Lane32& L) {
  const SysF& S = sys.s[ONE ? 0 : L.sid];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    B.y[k][i] = (double)L.rho[k] - (double)L.crho[k];
    B.y[6 + k][i] = ((double)L.vel[k] - (double)L.cvel[k]) * (k < 3 ? S.mu12d : S.mu123d);
  }
  B.t[i] = L.t;
  B.h[i] = (double)L.h;
  B.status[i] = (uint8_t)L.status;
  B.nsteps[i] = L.nacc;
  B.nrej[i] = L.nrej;
}

__device__ __forceinline__ void flush(unsigned long long rhs, unsigned long long steps,
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

template <bool MORSE, bool ONE>
__global__ void __launch_bounds__(128) k_integrate32_plain(SysSetF sys, const DevShape* shapes,
                                                           IntegParams ip, DevBatch B,
                                                           unsigned long long* counters) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  unsigned long long rhs = 0, steps = 0;
  Lane32 L;
  if (i < B.n && load<MORSE, ONE>(sys, shapes, ip, B, i, L, rhs)) {
    while (L.status == QCAMS_LANE_RUNNING) attempt<MORSE, ONE>(sys, ip, L);
    rhs += 6ull * L.calls;
    steps += L.calls;
    store<ONE>(sys, B, i, L);
  }
  flush(rhs, steps, counters);
}

template <bool MORSE, bool ONE>
__global__ void __launch_bounds__(128) k_integrate32_persistent(SysSetF sys,
                                                                const DevShape* shapes,
                                                                IntegParams ip, DevBatch B,
                                                                unsigned long long* counters) {
  const unsigned lane = threadIdx.x & 31u;
  unsigned long long rhs = 0, steps = 0;
  Lane32 L;
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
        if (k >= B.n) exhausted = true;
        else {
          idx = k;
          have = load<MORSE, ONE>(sys, shapes, ip, B, idx, L, rhs);
        }
      }
    }
    if (__all_sync(FULL, exhausted && !have)) break;
    if (have) {
      attempt<MORSE, ONE>(sys, ip, L);
      if (L.status != QCAMS_LANE_RUNNING) {
        rhs += 6ull * L.calls;
        steps += L.calls;
        store<ONE>(sys, B, idx, L);
        have = false;
      }
    }
  }
  flush(rhs, steps, counters);
}

SysSetF to_float(const SysSet& in) {
  SysSetF o{};
  o.n = in.n;
  for (int s = 0; s < in.n; ++s) {
    const DevSys& d = in.s[s];
    SysF& f = o.s[s];
    f.cA = (float)d.cA;
    f.cB = (float)d.cB;
    f.inv_mu12 = (float)d.inv_mu12;
    f.inv_mu123 = (float)d.inv_mu123;
    f.mu12 = (float)d.mu12;
    f.mu123 = (float)d.mu123;
    f.mu12d = d.mu12;
    f.mu123d = d.mu123;
    for (int k = 0; k < 5; ++k) {
      f.kf[k] = (float)d.kf[k];
      f.kf_morse[k] = (float)d.kf_morse[k];
    }
    for (int p = 0; p < 3; ++p) {
      const DevPair& q = d.pair[p];
      PairF& g = f.pair[p];
      g.kind = q.kind;
      g.m = q.m;
      g.n = q.n;
      g.c0 = (float)q.c0;
      g.c1 = (float)q.c1;
      g.c2 = (float)q.c2;
      g.c3 = (float)q.c3;
      g.c4 = (float)q.c4;
      const double log2e = 1.4426950408889634;
      g.l0 = (float)((q.kind == QCAMS_BUCK ? q.lc2 : q.c0) * log2e);
      g.l1 = (float)(q.c1 * log2e);
    }
  }
  return o;
}

template <bool MORSE, bool ONE>
cudaError_t launch32(const SysSetF& sf, const DevShape* shapes, const IntegParams& ip,
                     const DevBatch& b, int persistent, Ctx& ctx, cudaStream_t st) {
  const int block = 128;
  if (persistent) {
    cudaError_t e = cudaMemsetAsync(ctx.counters + 2, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm,
                                                      k_integrate32_persistent<MORSE, ONE>, block, 0);
    if (e != cudaSuccess) return e;
    long long grid = (long long)(per_sm < 1 ? 1 : per_sm) * ctx.sm_count;
    const long long need_blocks = (b.n + block - 1) / block;
    if (grid > need_blocks) grid = need_blocks;
    if (grid < 1) grid = 1;
    k_integrate32_persistent<MORSE, ONE><<<(unsigned)grid, block, 0, st>>>(sf, shapes, ip, b,
                                                                          ctx.counters);
    return cudaGetLastError();
  }
  const unsigned grid = (unsigned)((b.n + block - 1) / block);
  k_integrate32_plain<MORSE, ONE><<<grid, block, 0, st>>>(sf, shapes, ip, b, ctx.counters);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_integrate32(const SysSet& sys, const DevShape* shapes, const IntegParams& ip,
                               const DevBatch& b, int persistent, Ctx& ctx, cudaStream_t st,
                               bool all_morse) {
  const SysSetF sf = to_float(sys);
  const bool one = sys.n == 1;
  if (all_morse)
    return one ? launch32<true, true>(sf, shapes, ip, b, persistent, ctx, st)
               : launch32<true, false>(sf, shapes, ip, b, persistent, ctx, st);
  return one ? launch32<false, true>(sf, shapes, ip, b, persistent, ctx, st)
             : launch32<false, false>(sf, shapes, ip, b, persistent, ctx, st);
}

}  // namespace qcams
