// QCT oracle: a plain, slow, single-threaded FP64 restatement of the
// quasi-classical trajectory method of Koots & Perez-Rios, "PyQCAMS: Python
// Quasi-Classical Atom-Molecule Scattering" (Comput. Phys. Commun.).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
// call this file; only tests/, __graft_entry__.smoke() and bench.py's CPU
// baseline / reference legs do.  It shares no header, table, helper or
// constant with the CUDA library: every formula below is written again from
// the paper (sections and equations cited at each function) and, where the
// paper defers to a published method, from that method's own definition.
//
// Build: g++ -std=c++17 -O2 -ffp-contract=off -shared -fPIC (no FMA
// contraction, so x86-64 and aarch64 produce the same bits).
//
// Units: atomic units throughout (hbar = 1, masses in electron masses,
// energies in hartree, lengths in bohr).
//
// Parity status of each function is listed in its comment; every function
// here is pinned by a CPU test (tests/test_oracle_*.py).

#include <cmath>
#include <cstdint>
#include <cstring>
#include <algorithm>

namespace {

const double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// Data layout shared with the Python wrapper (oracle/__init__.py).
// ---------------------------------------------------------------------------
struct OPair {
  int32_t kind;   // 0 Morse {De, re, alpha}; 1 generalized LJ {m, n, Cm, Cn, r_scale};
                  // 2 Buckingham {A, B, C6, r_max_guess}
  int32_t pad;
  double p[5];
};
struct OSystem {
  double m[3];    // masses of atoms A, B, C (electron masses)
  OPair pair[3];  // AB, BC, CA
};
struct OInteg {
  double rtol, atol, r_stop, t_stop, h_fixed, gb_sigma;
  int64_t max_steps;
};
struct OLevel {
  int32_t ok;      // 1 = level exists
  int32_t pad;
  double E;        // internal energy E_{v,j}
  double r_minus;  // inner turning point
  double r_plus;   // outer turning point
  double tau;      // vibrational period
  double r_min;    // minimum of the effective potential
  double r_top;    // outermost maximum of the effective potential (0 if none)
  double E_top;    // dissociation threshold used for the level search
};
struct OResult {
  int32_t status;  // lane status (see kStatus*)
  int32_t cls;     // outcome class (see kCls*)
  int32_t vt, jt;  // integer bins
  double vprime, jprime, gbw;
  double dE;       // H(final) - E0
  double t;        // final time
  int32_t nsteps, nrej;
  double Epair[3]; // pair internal energies E_ab (AB, BC, CA)
  double L2pair[3];
  int32_t bound[3];
  int32_t pad;
};

// Lane status and outcome class codes (documented interface values).
enum { kStatusReady = 0, kStatusRunning = 1, kStatusRstop = 2, kStatusTmax = 3,
       kStatusMaxSteps = 4, kStatusHmin = 5, kStatusNaN = 6, kStatusCollapse = 7,
       kStatusNoLevel = 8, kStatusInvalid = 9 };
enum { kClsQ = 0, kClsRAC = 1, kClsRBC = 2, kClsD = 3, kClsAmbig = 4, kClsFail = 5 };

// ---------------------------------------------------------------------------
// Pair potentials, Sec. 3.2 (Main Code), items 1-3: V(r) and dV/dr.
// ---------------------------------------------------------------------------
double pot_V(const OPair& q, double r) {
  if (q.kind == 0) {  // Morse: De (1 - exp(-alpha (r - re)))^2 - De
    double De = q.p[0], re = q.p[1], a = q.p[2];
    double one_minus = 1.0 - std::exp(-a * (r - re));
    return De * one_minus * one_minus - De;
  }
  if (q.kind == 1) {  // generalized LJ: Cm / r^m - Cn / r^n
    double m = q.p[0], n = q.p[1], Cm = q.p[2], Cn = q.p[3];
    return Cm / std::pow(r, m) - Cn / std::pow(r, n);
  }
  // Buckingham: A exp(-B r) - C6 / r^6
  double A = q.p[0], B = q.p[1], C6 = q.p[2];
  return A * std::exp(-B * r) - C6 / std::pow(r, 6.0);
}

double pot_dV(const OPair& q, double r) {
  if (q.kind == 0) {
    double De = q.p[0], re = q.p[1], a = q.p[2];
    double x = std::exp(-a * (r - re));
    return 2.0 * a * De * (1.0 - x) * x;
  }
  if (q.kind == 1) {
    double m = q.p[0], n = q.p[1], Cm = q.p[2], Cn = q.p[3];
    return -m * Cm / std::pow(r, m + 1.0) + n * Cn / std::pow(r, n + 1.0);
  }
  double A = q.p[0], B = q.p[1], C6 = q.p[2];
  return -A * B * std::exp(-B * r) + 6.0 * C6 / std::pow(r, 7.0);
}

// Effective potential with angular momentum squared L2 (hbar^2 j(j+1) for a
// level; |r x p|^2 for a product pair), Sec. 2.1 (tau integrand) and
// Sec. 2.2 (bound-pair criterion).
double Veff(const OPair& q, double mu, double L2, double r) {
  return pot_V(q, r) + L2 / (2.0 * mu * r * r);
}
double dVeff(const OPair& q, double mu, double L2, double r) {
  return pot_dV(q, r) - L2 / (mu * r * r * r);
}

// ---------------------------------------------------------------------------
// Stationary points of V_eff by brute-force scan on a logarithmic grid plus
// bisection.  Defines: r_min = the outermost local minimum (the well); r_top =
// the first local maximum beyond it (the centrifugal barrier, "r_0" of the
// bound-pair criterion, Sec. 2.2); r_inner = the last local maximum inside the
// well (the Buckingham short-range maximum, Sec. 3.2 item 3) or the scan start.
// ---------------------------------------------------------------------------
const double kScanHi = 1000.0;
const int kScanN = 8000;

double scan_lo(const OPair& q) {
  double scale = 1.0;
  if (q.kind == 0) scale = q.p[1];
  else if (q.kind == 1) scale = q.p[4] > 0 ? q.p[4] : 1.0;
  else scale = q.p[3] > 0 ? q.p[3] : 1.0;
  return std::min(0.25, 0.2 * scale);
}

struct Stationary {
  bool has_well;
  double r_min;
  bool has_top;      // a maximum was found inside the scan range
  double r_top;
  double r_inner;
};

template <class F>
double bisect(F f, double a, double b) {
  // f(a) and f(b) have opposite signs; halve until the interval cannot shrink.
  double fa = f(a);
  for (int it = 0; it < 200; ++it) {
    double m = 0.5 * (a + b);
    if (m <= a || m >= b) break;
    double fm = f(m);
    if ((fm < 0) == (fa < 0)) { a = m; fa = fm; } else { b = m; }
  }
  return 0.5 * (a + b);
}

Stationary stationary_points(const OPair& q, double mu, double L2) {
  Stationary st{false, 0.0, false, 0.0, 0.0};
  const double lo = scan_lo(q);
  const double dl = std::log(kScanHi / lo) / kScanN;
  auto g = [&](double r) { return dVeff(q, mu, L2, r); };
  st.r_inner = lo;
  // first pass: record all sign changes
  int last_min = -1;
  double prev_r = lo, prev = g(lo);
  // keep the crossings in a small ring (potentials here have at most 3)
  int nc = 0;
  int kind_c[16];
  double a_c[16], b_c[16];
  for (int k = 1; k <= kScanN; ++k) {
    double r = lo * std::exp(dl * k);
    double cur = g(r);
    if ((prev < 0) != (cur < 0) && nc < 16) {
      kind_c[nc] = (prev < 0) ? +1 : -1;  // +1: minimum (- to +), -1: maximum (+ to -)
      a_c[nc] = prev_r; b_c[nc] = r; ++nc;
    }
    prev = cur; prev_r = r;
  }
  for (int i = 0; i < nc; ++i) if (kind_c[i] == +1) last_min = i;
  if (last_min < 0) return st;
  st.has_well = true;
  st.r_min = bisect(g, a_c[last_min], b_c[last_min]);
  for (int i = last_min + 1; i < nc; ++i) {
    if (kind_c[i] == -1) { st.has_top = true; st.r_top = bisect(g, a_c[i], b_c[i]); break; }
  }
  for (int i = last_min - 1; i >= 0; --i) {
    if (kind_c[i] == -1) { st.r_inner = bisect(g, a_c[i], b_c[i]); break; }
  }
  return st;
}

// Dissociation threshold of the well: V_eff at the outer maximum; with no
// angular momentum V_eff tends to 0 from below, so the threshold is 0
// (Sec. 2.2, criterion for j' = 0).  If the barrier lies beyond the scan
// range, V_eff at the scan end is used (a value within L2/(2 mu 1000^2) of it).
double threshold(const OPair& q, double mu, double L2, const Stationary& st) {
  if (L2 == 0.0) return 0.0;
  if (st.has_top) return Veff(q, mu, L2, st.r_top);
  return Veff(q, mu, L2, kScanHi);
}

// Turning points of E = V_eff inside the well [r_inner, r_outer].
void turning_points(const OPair& q, double mu, double L2, double E, double r_inner,
                    double r_min, double r_outer, double* rm, double* rp) {
  auto f = [&](double r) { return Veff(q, mu, L2, r) - E; };
  *rm = bisect(f, r_inner, r_min);
  *rp = bisect(f, r_min, r_outer);
}

// Trapezoid rule in s over [-pi/2, pi/2] after r = c + d sin(s).  The mapped
// integrands of the action and of the period extend to smooth periodic
// functions, so the trapezoid sums converge geometrically; the panel count is
// doubled until two successive sums agree to 1e-14 relative.  Because the
// error falls geometrically, the successive differences shrink by large
// factors until they reach the round-off floor next to the turning points
// (where E - V_eff is a difference of nearly equal numbers); when a doubling
// no longer halves the difference, the floor has been reached and the
// coarser sum, which samples less of that noise, is returned.
template <class F>
double trap_s(F f, double f_lo, double f_hi) {
  int n = 16;
  double hs = kPi / n;
  double sum = 0.5 * (f_lo + f_hi);
  for (int k = 1; k < n; ++k) sum += f(-0.5 * kPi + k * hs);
  double I = hs * sum;
  double prev_diff = INFINITY;
  for (int level = 0; level < 12; ++level) {
    n *= 2; hs *= 0.5;
    for (int k = 1; k < n; k += 2) sum += f(-0.5 * kPi + k * hs);
    double In = hs * sum;
    double diff = std::fabs(In - I);
    if (diff <= 1e-14 * std::fabs(In)) return In;
    if (n >= 64 && diff > 0.5 * prev_diff) return I;
    prev_diff = diff;
    I = In;
  }
  return I;
}

// Action integral  int_{r-}^{r+} sqrt(E - V_eff) dr  (Eq. for v', Sec. 2.2).
double action_integral(const OPair& q, double mu, double L2, double E, double rm, double rp) {
  double c = 0.5 * (rp + rm), d = 0.5 * (rp - rm);
  auto f = [&](double s) {
    double r = c + d * std::sin(s);
    double w = E - Veff(q, mu, L2, r);
    return (w > 0 ? std::sqrt(w) : 0.0) * d * std::cos(s);
  };
  return trap_s(f, 0.0, 0.0);
}

// Period integral  int_{r-}^{r+} [E - V_eff]^{-1/2} dr  (Eq. for tau, Sec. 2.1).
double period_integral(const OPair& q, double mu, double L2, double E, double rm, double rp) {
  double c = 0.5 * (rp + rm), d = 0.5 * (rp - rm);
  auto f = [&](double s) {
    double r = c + d * std::sin(s);
    double w = E - Veff(q, mu, L2, r);
    return w > 0 ? d * std::cos(s) / std::sqrt(w) : 0.0;
  };
  // endpoint limits: sqrt(2 d / |V_eff'(r_pm)|)
  double flo = std::sqrt(2.0 * d / std::fabs(dVeff(q, mu, L2, rm)));
  double fhi = std::sqrt(2.0 * d / std::fabs(dVeff(q, mu, L2, rp)));
  return trap_s(f, flo, fhi);
}

// Continuous vibrational quantum number v(E) = -1/2 + sqrt(2 mu)/pi * action
// (Eq. for v', Sec. 2.2; the same Bohr-Sommerfeld rule quantises the initial
// state, Sec. 2).
double v_of_E(const OPair& q, double mu, double L2, double E, const Stationary& st,
              double r_outer, double* rm, double* rp) {
  turning_points(q, mu, L2, E, st.r_inner, st.r_min, r_outer, rm, rp);
  return -0.5 + std::sqrt(2.0 * mu) / kPi * action_integral(q, mu, L2, E, *rm, *rp);
}

// Bohr-Sommerfeld level (v, j) of pair q with reduced mass mu: solve
// v(E) = v by bisection on (V_eff(r_min), E_top).
OLevel solve_level(const OPair& q, double mu, int v, int j) {
  OLevel L{};
  L.ok = 0;
  const double L2 = double(j) * double(j + 1);
  Stationary st = stationary_points(q, mu, L2);
  if (!st.has_well) return L;
  double Etop = threshold(q, mu, L2, st);
  double r_outer = st.has_top ? st.r_top : kScanHi;
  double Emin = Veff(q, mu, L2, st.r_min);
  double rm, rp;
  double vtop = v_of_E(q, mu, L2, Etop, st, r_outer, &rm, &rp);
  if (vtop < v) return L;
  double a = Emin, b = Etop;
  for (int it = 0; it < 200; ++it) {
    double m = 0.5 * (a + b);
    if (m <= a || m >= b) break;
    double vm = v_of_E(q, mu, L2, m, st, r_outer, &rm, &rp);
    if (vm < v) a = m; else b = m;
  }
  double E = 0.5 * (a + b);
  v_of_E(q, mu, L2, E, st, r_outer, &rm, &rp);
  L.ok = 1;
  L.E = E;
  L.r_minus = rm;
  L.r_plus = rp;
  L.tau = std::sqrt(2.0 * mu) * period_integral(q, mu, L2, E, rm, rp);
  L.r_min = st.r_min;
  L.r_top = st.has_top ? st.r_top : 0.0;
  L.E_top = Etop;
  return L;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 counter-based generator, from its published definition
// (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
// SC'11): ten rounds of two 32x32->64 multiplies with a Weyl-sequence key
// schedule.
// ---------------------------------------------------------------------------
void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint64_t p0 = uint64_t(0xD2511F53u) * c0;
    uint64_t p1 = uint64_t(0xCD9E8D57u) * c2;
    uint32_t hi0 = uint32_t(p0 >> 32), lo0 = uint32_t(p0);
    uint32_t hi1 = uint32_t(p1 >> 32), lo1 = uint32_t(p1);
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// ---------------------------------------------------------------------------
// Masses and Jacobi coordinates, Sec. 2 (Eq. 2 and the definitions of mu12,
// mu123 below it).  rho1 = r_B - r_A, rho2 = r_C - (centre of mass of AB).
// ---------------------------------------------------------------------------
struct Masses {
  double mu12, mu123, cA, cB;   // cA = mB/(mA+mB), cB = mA/(mA+mB)
  double mu_pair[3];            // reduced masses of the pairs AB, BC, CA
};
Masses masses(const OSystem& s) {
  Masses M;
  double mA = s.m[0], mB = s.m[1], mC = s.m[2];
  M.mu12 = 1.0 / (1.0 / mA + 1.0 / mB);
  M.mu123 = 1.0 / (1.0 / mC + 1.0 / (mA + mB));
  M.cA = mB / (mA + mB);
  M.cB = mA / (mA + mB);
  M.mu_pair[0] = mA * mB / (mA + mB);
  M.mu_pair[1] = mB * mC / (mB + mC);
  M.mu_pair[2] = mC * mA / (mC + mA);
  return M;
}

// Pair separation vectors from the Jacobi vectors: AB = rho1,
// BC = r_C - r_B = rho2 - cB rho1, CA = r_C - r_A = rho2 + cA rho1.
void pair_vectors(const Masses& M, const double* rho1, const double* rho2, double r[3][3]) {
  for (int a = 0; a < 3; ++a) {
    r[0][a] = rho1[a];
    r[1][a] = rho2[a] - M.cB * rho1[a];
    r[2][a] = rho2[a] + M.cA * rho1[a];
  }
}

double norm3(const double* x) { return std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]); }

// Total energy, Eq. 2: P1^2/2mu12 + P2^2/2mu123 + V_AB + V_BC + V_CA.
double hamiltonian(const OSystem& s, const double* y) {
  Masses M = masses(s);
  const double *rho1 = y, *rho2 = y + 3, *P1 = y + 6, *P2 = y + 9;
  double r[3][3];
  pair_vectors(M, rho1, rho2, r);
  double T = (P1[0] * P1[0] + P1[1] * P1[1] + P1[2] * P1[2]) / (2.0 * M.mu12) +
             (P2[0] * P2[0] + P2[1] * P2[1] + P2[2] * P2[2]) / (2.0 * M.mu123);
  double V = 0.0;
  for (int k = 0; k < 3; ++k) V += pot_V(s.pair[k], norm3(r[k]));
  return T + V;
}

// Hamilton's equations, Eqs. 3-4, in the Jacobi coordinates of Eq. 2.
// y = (rho1, rho2, P1, P2).  The chain rule through the pair vectors gives
//   dV/drho1 = g_AB r_AB - cB g_BC r_BC + cA g_CA r_CA
//   dV/drho2 =             g_BC r_BC +    g_CA r_CA,     g = V'(r)/r.
void rhs_jacobi(const OSystem& s, const Masses& M, const double* y, double* dy) {
  const double *rho1 = y, *rho2 = y + 3, *P1 = y + 6, *P2 = y + 9;
  double r[3][3], g[3];
  pair_vectors(M, rho1, rho2, r);
  for (int k = 0; k < 3; ++k) {
    double d = norm3(r[k]);
    g[k] = pot_dV(s.pair[k], d) / d;
  }
  for (int a = 0; a < 3; ++a) {
    dy[a] = P1[a] / M.mu12;
    dy[3 + a] = P2[a] / M.mu123;
    double dVd1 = g[0] * r[0][a] - M.cB * g[1] * r[1][a] + M.cA * g[2] * r[2][a];
    double dVd2 = g[1] * r[1][a] + g[2] * r[2][a];
    dy[6 + a] = -dVd1;
    dy[9 + a] = -dVd2;
  }
}

// Cartesian form, Eq. 1: 3 atoms, x = (r_A, r_B, r_C, p_A, p_B, p_C).
// Used only to cross-check the Jacobi equations (Runge-Kutta methods commute
// with the linear change of variables between the two forms).
void rhs_cartesian(const OSystem& s, const double* x, double* dx) {
  const double* rA = x; const double* rB = x + 3; const double* rC = x + 6;
  double pairs[3][3];  // AB: rB - rA; BC: rC - rB; CA: rA - rC
  for (int a = 0; a < 3; ++a) {
    pairs[0][a] = rB[a] - rA[a];
    pairs[1][a] = rC[a] - rB[a];
    pairs[2][a] = rA[a] - rC[a];
  }
  double g[3];
  for (int k = 0; k < 3; ++k) {
    double d = norm3(pairs[k]);
    g[k] = pot_dV(s.pair[k], d) / d;
  }
  for (int a = 0; a < 3; ++a) {
    for (int i = 0; i < 3; ++i) dx[3 * i + a] = x[9 + 3 * i + a] / s.m[i];
    // force on A: from AB (pulls along rB - rA) and CA (rA - rC)
    double FA = g[0] * pairs[0][a] - g[2] * pairs[2][a];
    double FB = -g[0] * pairs[0][a] + g[1] * pairs[1][a];
    double FC = -g[1] * pairs[1][a] + g[2] * pairs[2][a];
    dx[9 + a] = FA;
    dx[12 + a] = FB;
    dx[15 + a] = FC;
  }
}

void jacobi_to_cartesian(const OSystem& s, const double* y, double* x) {
  Masses M = masses(s);
  double mA = s.m[0], mB = s.m[1], mC = s.m[2], Mt = mA + mB + mC;
  const double *rho1 = y, *rho2 = y + 3, *P1 = y + 6, *P2 = y + 9;
  for (int a = 0; a < 3; ++a) {
    double Rab = -(mC / Mt) * rho2[a];          // centre of mass of AB (total COM at 0)
    x[a] = Rab - M.cA * rho1[a];                // r_A
    x[3 + a] = Rab + M.cB * rho1[a];            // r_B
    x[6 + a] = Rab + rho2[a];                   // r_C
    double v1 = P1[a] / M.mu12, v2 = P2[a] / M.mu123;
    double Vab = -(mC / Mt) * v2;
    x[9 + a] = mA * (Vab - M.cA * v1);
    x[12 + a] = mB * (Vab + M.cB * v1);
    x[15 + a] = mC * (Vab + v2);
  }
}

void cartesian_to_jacobi(const OSystem& s, const double* x, double* y) {
  Masses M = masses(s);
  double mA = s.m[0], mB = s.m[1], mC = s.m[2];
  for (int a = 0; a < 3; ++a) {
    double rA = x[a], rB = x[3 + a], rC = x[6 + a];
    double vA = x[9 + a] / mA, vB = x[12 + a] / mB, vC = x[15 + a] / mC;
    y[a] = rB - rA;
    y[3 + a] = rC - (mA * rA + mB * rB) / (mA + mB);
    y[6 + a] = M.mu12 * (vB - vA);
    y[9 + a] = M.mu123 * (vC - (mA * vA + mB * vB) / (mA + mB));
  }
}

// ---------------------------------------------------------------------------
// Dormand-Prince 5(4) Runge-Kutta pair (J. R. Dormand & P. J. Prince, J. Comp.
// Appl. Math. 6 (1980) 19-26), the method behind SciPy's solve_ivp RK45 that
// the paper integrates Hamilton's equations with (Sec. 3.2).
// ---------------------------------------------------------------------------
const double DP_C[7] = {0.0, 1.0 / 5, 3.0 / 10, 4.0 / 5, 8.0 / 9, 1.0, 1.0};
const double DP_A[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5, 0, 0, 0, 0, 0},
    {3.0 / 40, 9.0 / 40, 0, 0, 0, 0},
    {44.0 / 45, -56.0 / 15, 32.0 / 9, 0, 0, 0},
    {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729, 0, 0},
    {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656, 0},
    {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}};
const double DP_B[7] = {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84, 0};
const double DP_BS[7] = {5179.0 / 57600, 0, 7571.0 / 16695, 393.0 / 640,
                         -92097.0 / 339200, 187.0 / 2100, 1.0 / 40};

// One Dormand-Prince step of size h from (t, y) with k1 = f(t, y) known.
// Writes the 5th-order solution, its derivative (FSAL) and the embedded error
// estimate h * sum (b_i - b*_i) k_i.
template <int D, class F>
void dopri5_step(F& f, double t, const double* y, const double* k1, double h,
                 double* ynew, double* knew, double* err) {
  double k[7][D];
  double tmp[D];
  for (int i = 0; i < D; ++i) k[0][i] = k1[i];
  for (int s = 1; s < 7; ++s) {
    for (int i = 0; i < D; ++i) {
      double acc = 0.0;
      for (int q = 0; q < s; ++q) acc += DP_A[s][q] * k[q][i];
      tmp[i] = y[i] + h * acc;
    }
    f(t + DP_C[s] * h, tmp, k[s]);
  }
  // stage 7 was evaluated at y + h sum a_7q k_q = the 5th-order solution
  for (int i = 0; i < D; ++i) {
    double acc = 0.0, eacc = 0.0;
    for (int q = 0; q < 7; ++q) {
      acc += DP_B[q] * k[q][i];
      eacc += (DP_B[q] - DP_BS[q]) * k[q][i];
    }
    ynew[i] = y[i] + h * acc;
    knew[i] = k[6][i];
    err[i] = h * eacc;
  }
}

// RMS norm used by SciPy's solve_ivp error control.
template <int D>
double rms(const double* v) {
  double s = 0.0;
  for (int i = 0; i < D; ++i) s += v[i] * v[i];
  return std::sqrt(s / D);
}

// Starting step size: the algorithm of Hairer, Norsett & Wanner, "Solving
// Ordinary Differential Equations I", Sec. II.4, as SciPy's solve_ivp uses it
// (error-estimator order 4, so exponent 1/5).
template <int D, class F>
double initial_step(F& f, double t0, const double* y0, const double* f0, double rtol, double atol) {
  double sc[D], tmp[D], y1[D], f1[D];
  for (int i = 0; i < D; ++i) sc[i] = atol + std::fabs(y0[i]) * rtol;
  for (int i = 0; i < D; ++i) tmp[i] = y0[i] / sc[i];
  double d0 = rms<D>(tmp);
  for (int i = 0; i < D; ++i) tmp[i] = f0[i] / sc[i];
  double d1 = rms<D>(tmp);
  double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
  for (int i = 0; i < D; ++i) y1[i] = y0[i] + h0 * f0[i];
  f(t0 + h0, y1, f1);
  for (int i = 0; i < D; ++i) tmp[i] = (f1[i] - f0[i]) / sc[i];
  double d2 = rms<D>(tmp) / h0;
  double h1;
  if (d1 <= 1e-15 && d2 <= 1e-15) h1 = std::max(1e-6, h0 * 1e-3);
  else h1 = std::pow(0.01 / std::max(d1, d2), 1.0 / 5.0);
  return std::min(100.0 * h0, h1);
}

// ---------------------------------------------------------------------------
// Stop rule (Sec. 3.1, t_stop and r_stop): stop after the first accepted step
// at which the largest pair distance exceeds r_stop while the atom-molecule
// distance grows (rho2 . P2 > 0), or t >= t_max = t_stop * R / v_rel.
// ---------------------------------------------------------------------------
bool separated(const Masses& M, const double* y, double r_stop) {
  double r[3][3];
  pair_vectors(M, y, y + 3, r);
  double rmax = std::max(norm3(r[0]), std::max(norm3(r[1]), norm3(r[2])));
  double radial = y[3] * y[9] + y[4] * y[10] + y[5] * y[11];
  return rmax > r_stop && radial > 0.0;
}

// Buckingham short-range maximum ("max", Sec. 3.2 item 3): the inner root of
// V'(r) = 0 below the well; a Buckingham pair closer than this has fallen into
// the unphysical collapse region.  Returns 0 for other kinds.
double buck_inner_barrier(const OPair& q) {
  if (q.kind != 2) return 0.0;
  Stationary st = stationary_points(q, 1.0, 0.0);
  return st.has_well ? st.r_inner : 0.0;
}

bool collapsed(const OSystem& s, const Masses& M, const double* y, const double* rb) {
  double r[3][3];
  pair_vectors(M, y, y + 3, r);
  for (int k = 0; k < 3; ++k)
    if (s.pair[k].kind == 2 && norm3(r[k]) < rb[k]) return true;
  return false;
}

struct JacobiRHS {
  const OSystem* s;
  Masses M;
  long nrhs = 0;
  void operator()(double, const double* y, double* dy) { ++nrhs; rhs_jacobi(*s, M, y, dy); }
};
struct CartRHS {
  const OSystem* s;
  void operator()(double, const double* x, double* dx) { rhs_cartesian(*s, x, dx); }
};

// Adaptive integration of one trajectory with SciPy's RK45 step-size
// controller: RMS error norm with scale atol + rtol max(|y_n|, |y_n+1|);
// accept iff norm < 1; factor 0.9 norm^(-1/5) clamped to [0.2, 10], and no
// growth on the step that follows a rejection within the same step attempt.
int integrate_adaptive(const OSystem& s, const OInteg& in, double* y, double t_scale,
                       double* t_out, int32_t* nsteps, int32_t* nrej) {
  JacobiRHS f{&s, masses(s)};
  double rb[3];
  for (int k = 0; k < 3; ++k) rb[k] = buck_inner_barrier(s.pair[k]);
  const double t_max = in.t_stop * t_scale;
  double t = 0.0;
  double k1[12], ynew[12], knew[12], err[12], sc[12];
  f(t, y, k1);
  double h = initial_step<12>(f, t, y, k1, in.rtol, in.atol);
  int32_t acc = 0, rej = 0;
  int status = kStatusRunning;
  while (status == kStatusRunning) {
    bool step_rejected = false;
    for (;;) {
      double min_step = 10.0 * (std::nextafter(t, INFINITY) - t);
      if (h < min_step) { status = kStatusHmin; break; }
      dopri5_step<12>(f, t, y, k1, h, ynew, knew, err);
      for (int i = 0; i < 12; ++i)
        sc[i] = in.atol + std::max(std::fabs(y[i]), std::fabs(ynew[i])) * in.rtol;
      double e2[12];
      for (int i = 0; i < 12; ++i) e2[i] = err[i] / sc[i];
      double en = rms<12>(e2);
      if (!(en == en)) { status = kStatusNaN; break; }
      if (en < 1.0) {
        double factor = (en == 0.0) ? 10.0 : std::min(10.0, 0.9 * std::pow(en, -0.2));
        if (step_rejected) factor = std::min(1.0, factor);
        t = t + h;
        h = h * factor;
        for (int i = 0; i < 12; ++i) { y[i] = ynew[i]; k1[i] = knew[i]; }
        ++acc;
        break;
      }
      h = h * std::max(0.2, 0.9 * std::pow(en, -0.2));
      step_rejected = true;
      ++rej;
      if (acc + rej >= in.max_steps) break;
    }
    if (status != kStatusRunning) break;
    if (collapsed(s, f.M, y, rb)) status = kStatusCollapse;
    else if (separated(f.M, y, in.r_stop)) status = kStatusRstop;
    else if (t >= t_max) status = kStatusTmax;
    else if (acc + rej >= in.max_steps) status = kStatusMaxSteps;
  }
  *t_out = t;
  *nsteps = acc;
  *nrej = rej;
  return status;
}

// ---------------------------------------------------------------------------
// Product analysis, Sec. 2.2: pair energies, bound-pair criterion, j', v',
// Gaussian binning weight.
// ---------------------------------------------------------------------------
struct PairState { double E, L2, r; };

void pair_states(const OSystem& s, const double* y, PairState ps[3]) {
  Masses M = masses(s);
  const double *P1 = y + 6, *P2 = y + 9;
  double r[3][3], v[3][3];
  pair_vectors(M, y, y + 3, r);
  for (int a = 0; a < 3; ++a) {
    double v1 = P1[a] / M.mu12, v2 = P2[a] / M.mu123;
    v[0][a] = v1;                // d(rho1)/dt
    v[1][a] = v2 - M.cB * v1;    // d(r_C - r_B)/dt
    v[2][a] = v2 + M.cA * v1;    // d(r_C - r_A)/dt
  }
  for (int k = 0; k < 3; ++k) {
    double mu = M.mu_pair[k];
    double v2 = v[k][0] * v[k][0] + v[k][1] * v[k][1] + v[k][2] * v[k][2];
    double d = norm3(r[k]);
    ps[k].r = d;
    ps[k].E = 0.5 * mu * v2 + pot_V(s.pair[k], d);
    double Lx = mu * (r[k][1] * v[k][2] - r[k][2] * v[k][1]);
    double Ly = mu * (r[k][2] * v[k][0] - r[k][0] * v[k][2]);
    double Lz = mu * (r[k][0] * v[k][1] - r[k][1] * v[k][0]);
    ps[k].L2 = Lx * Lx + Ly * Ly + Lz * Lz;
  }
}

void analyze(const OSystem& s, const OInteg& in, const double* y, double E0, int status,
             OResult* out) {
  Masses M = masses(s);
  PairState ps[3];
  pair_states(s, y, ps);
  out->dE = hamiltonian(s, y) - E0;
  out->vprime = 0.0; out->jprime = 0.0; out->gbw = 0.0; out->vt = 0; out->jt = 0;
  int nb = 0, which = -1;
  Stationary sts[3];
  for (int k = 0; k < 3; ++k) {
    out->Epair[k] = ps[k].E;
    out->L2pair[k] = ps[k].L2;
    sts[k] = stationary_points(s.pair[k], M.mu_pair[k], ps[k].L2);
    // Bound (Sec. 2.2): E_ab below V_eff at its outer maximum r_0 (0 when
    // L = 0).  Reading: the pair must also lie inside that maximum
    // (r_inner < r_ab < r_0); a pair outside the centrifugal barrier is
    // separating, whatever its energy.  A Buckingham pair must in addition
    // sit below its short-range maximum.
    bool bound = false;
    if (sts[k].has_well) {
      double mu = M.mu_pair[k];
      double thr = threshold(s.pair[k], mu, ps[k].L2, sts[k]);
      double r_out = sts[k].has_top ? sts[k].r_top : kScanHi;
      bound = ps[k].E < thr && ps[k].r < r_out && ps[k].r > sts[k].r_inner;
      if (bound && s.pair[k].kind == 2 &&
          ps[k].E >= Veff(s.pair[k], mu, ps[k].L2, sts[k].r_inner))
        bound = false;
    }
    out->bound[k] = bound ? 1 : 0;
    if (bound) { ++nb; which = k; }
  }
  if (status != kStatusRstop && status != kStatusTmax) { out->cls = kClsFail; return; }
  if (nb == 0) { out->cls = kClsD; return; }
  if (nb > 1) { out->cls = kClsAmbig; return; }
  out->cls = (which == 0) ? kClsQ : (which == 2) ? kClsRAC : kClsRBC;
  const OPair& q = s.pair[which];
  double mu = M.mu_pair[which], L2 = ps[which].L2, E = ps[which].E;
  const Stationary& st = sts[which];
  double r_outer = st.has_top ? st.r_top : kScanHi;
  double rm, rp;
  double vp = v_of_E(q, mu, L2, E, st, r_outer, &rm, &rp);
  double jp = -0.5 + 0.5 * std::sqrt(1.0 + 4.0 * L2);
  int vt = int(std::floor(vp + 0.5));
  if (vt < 0) vt = 0;
  int jt = int(std::floor(jp + 0.5));
  double sg = in.gb_sigma;
  double dv = vp - vt;
  out->vprime = vp;
  out->jprime = jp;
  out->vt = vt;
  out->jt = jt;
  out->gbw = std::exp(-dv * dv / (2.0 * sg * sg)) / (sg * std::sqrt(2.0 * kPi));
}

// ---------------------------------------------------------------------------
// Initial conditions, Sec. 2.1 (P1 components, Eq. 5; start distance, Eq. 6).
// Uniforms from Philox4x32-10 with key = seed and counter = (id, 0, 0):
// u_k = (word_k + 1/2) 2^-32; cos(theta) = 2 u0 - 1, phi = 2 pi u1,
// eta = 2 pi u2, chi = u3.
// ---------------------------------------------------------------------------
int init_lane(const OSystem& s, const OLevel& lev, double Ecol, double b, int j, double R0,
              uint64_t seed, uint64_t id, const double* u_in, double* y, double* t_scale,
              double* E0, double* u_out) {
  Masses M = masses(s);
  double u[4];
  if (u_in) {
    for (int k = 0; k < 4; ++k) u[k] = u_in[k];
  } else {
    uint32_t ctr[4] = {uint32_t(id), uint32_t(id >> 32), 0u, 0u};
    uint32_t key[2] = {uint32_t(seed), uint32_t(seed >> 32)};
    uint32_t w[4];
    philox4x32_10(ctr, key, w);
    for (int k = 0; k < 4; ++k) u[k] = (double(w[k]) + 0.5) * (1.0 / 4294967296.0);
  }
  if (u_out) for (int k = 0; k < 4; ++k) u_out[k] = u[k];
  double cth = 2.0 * u[0] - 1.0;
  double sth = std::sqrt(std::max(0.0, 1.0 - cth * cth));
  double phi = 2.0 * kPi * u[1], eta = 2.0 * kPi * u[2], chi = u[3];
  double rp = lev.r_plus;
  double P1m = std::sqrt(double(j) * double(j + 1)) / rp;
  y[0] = rp * sth * std::cos(phi);
  y[1] = rp * sth * std::sin(phi);
  y[2] = rp * cth;
  y[6] = P1m * (std::sin(phi) * std::cos(eta) - cth * std::cos(phi) * std::sin(eta));
  y[7] = P1m * (-std::cos(phi) * std::cos(eta) - cth * std::sin(phi) * std::sin(eta));
  y[8] = P1m * (sth * std::sin(eta));
  double P2m = std::sqrt(2.0 * M.mu123 * Ecol);
  double R = R0 + chi * P2m * lev.tau / M.mu123;
  if (!(R > b) || !(Ecol > 0)) return kStatusInvalid;
  y[3] = 0.0;
  y[4] = b;
  y[5] = -std::sqrt(R * R - b * b);
  y[9] = 0.0;
  y[10] = 0.0;
  y[11] = P2m;
  *t_scale = R / (P2m / M.mu123);
  *E0 = hamiltonian(s, y);
  return kStatusReady;
}

// Histogram record per cell (int64), identical layout to the library's
// documented reduction output: counts[8] | vt[3][64] | jt[3][256] |
// gb[3][64] (sum of W * 2^32, rounded to nearest) | w[8] | w2[8].
const int H_COUNT = 0, H_VT = 8, H_JT = 8 + 192, H_GB = 200 + 768, H_W = 968 + 192,
          H_W2 = 1160 + 8, H_STRIDE = 1176;
const int N_VT = 64, N_JT = 256;

int64_t fixed_point(double x) { return (int64_t)std::llrint(std::ldexp(x, 32)); }

}  // namespace

// ===========================================================================
// C entry points used by the Python wrapper.
// ===========================================================================
extern "C" {

int oracle_abi_version() { return 1; }

// System set-up (Sec. 3.1 inputs and Sec. 3.2 potentials).  Masses are given
// in unified atomic mass units and converted to electron masses (CODATA 2018,
// 1 u = 1822.888486209 m_e).  Spec kinds: 0 Morse {De, re, alpha};
// 1 LJ {m, n, Cm, Cn, r_scale}; 2 Buckingham {A, B, C6, r_max_guess};
// 3 LJ fitted to a well {m, n, De, re}: V'(re) = 0 and V(re) = -De give
// Cm = De n re^m / (m - n), Cn = De m re^n / (m - n);
// 4 Morse from the harmonic constant {De, re, omega_e}:
// alpha = omega_e sqrt(mu / (2 De)) with mu the pair's reduced mass.
int oracle_system_setup(const double* mass_u, const int32_t* kind, const double* spec,
                        OSystem* out) {
  const double amu = 1822.888486209;
  for (int i = 0; i < 3; ++i) out->m[i] = mass_u[i] * amu;
  const int pa[3] = {0, 1, 2}, pb[3] = {1, 2, 0};   // AB, BC, CA
  for (int k = 0; k < 3; ++k) {
    const double* q = spec + 5 * k;
    OPair& P = out->pair[k];
    std::memset(&P, 0, sizeof(P));
    double ma = out->m[pa[k]], mb = out->m[pb[k]];
    double mu = ma * mb / (ma + mb);
    switch (kind[k]) {
      case 0: P.kind = 0; P.p[0] = q[0]; P.p[1] = q[1]; P.p[2] = q[2]; break;
      case 1: P.kind = 1; for (int i = 0; i < 5; ++i) P.p[i] = q[i]; break;
      case 2: P.kind = 2; for (int i = 0; i < 4; ++i) P.p[i] = q[i]; break;
      case 3: {
        double m = q[0], n = q[1], De = q[2], re = q[3];
        if (!(m > n)) return -1;
        P.kind = 1; P.p[0] = m; P.p[1] = n;
        P.p[2] = De * n * std::pow(re, m) / (m - n);
        P.p[3] = De * m * std::pow(re, n) / (m - n);
        P.p[4] = re;
        break;
      }
      case 4: P.kind = 0; P.p[0] = q[0]; P.p[1] = q[1];
              P.p[2] = q[2] * std::sqrt(mu / (2.0 * q[0])); break;
      default: return -1;
    }
  }
  return 0;
}

void oracle_pair_potential(const OPair* q, double r, double* V, double* dV) {
  *V = pot_V(*q, r);
  *dV = pot_dV(*q, r);
}

void oracle_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  philox4x32_10(ctr, key, out);
}

void oracle_level(const OPair* q, double mu, int v, int j, OLevel* out) {
  *out = solve_level(*q, mu, v, j);
}

// Continuous v(E) for a pair with angular momentum squared L2 (Eq. for v').
double oracle_v_of_E(const OPair* q, double mu, double L2, double E) {
  Stationary st = stationary_points(*q, mu, L2);
  if (!st.has_well) return NAN;
  double rm, rp;
  return v_of_E(*q, mu, L2, E, st, st.has_top ? st.r_top : kScanHi, &rm, &rp);
}

// Stationary points and threshold of V_eff: out = {has_well, r_min, has_top,
// r_top, r_inner, threshold}.
void oracle_stationary(const OPair* q, double mu, double L2, double* out) {
  Stationary st = stationary_points(*q, mu, L2);
  out[0] = st.has_well; out[1] = st.r_min; out[2] = st.has_top; out[3] = st.r_top;
  out[4] = st.r_inner; out[5] = st.has_well ? threshold(*q, mu, L2, st) : NAN;
}

double oracle_hamiltonian(const OSystem* s, const double* y) { return hamiltonian(*s, y); }

void oracle_rhs(const OSystem* s, const double* y, double* dy) {
  rhs_jacobi(*s, masses(*s), y, dy);
}

void oracle_rhs_cartesian(const OSystem* s, const double* x, double* dx) {
  rhs_cartesian(*s, x, dx);
}

void oracle_jacobi_to_cartesian(const OSystem* s, const double* y, double* x) {
  jacobi_to_cartesian(*s, y, x);
}
void oracle_cartesian_to_jacobi(const OSystem* s, const double* x, double* y) {
  cartesian_to_jacobi(*s, x, y);
}

void oracle_dopri5_tableau(double* c, double* a, double* b, double* bs) {
  for (int i = 0; i < 7; ++i) {
    c[i] = DP_C[i]; b[i] = DP_B[i]; bs[i] = DP_BS[i];
    for (int q = 0; q < 7; ++q) a[7 * i + q] = q < 6 ? DP_A[i][q] : 0.0;
  }
}

// One Dormand-Prince step on the scalar test equation y' = lambda y.
void oracle_dopri5_linear(double lambda, double h, double y0, double* y1, double* err) {
  struct Lin { double l; void operator()(double, const double* y, double* d) { d[0] = l * y[0]; } };
  Lin f{lambda};
  double k1 = lambda * y0, kn;
  dopri5_step<1>(f, 0.0, &y0, &k1, h, y1, &kn, err);
}

// Fixed-step integration (no error control) of n lanes in place; y is
// row-major [n][12].  Step count per lane: nsteps.
void oracle_run_fixed(const OSystem* s, double* y, int64_t n, double h, int64_t nsteps) {
  JacobiRHS f{s, masses(*s)};
  double k1[12], ynew[12], knew[12], err[12];
  for (int64_t lane = 0; lane < n; ++lane) {
    double* yl = y + 12 * lane;
    f(0.0, yl, k1);
    double t = 0.0;
    for (int64_t it = 0; it < nsteps; ++it) {
      dopri5_step<12>(f, t, yl, k1, h, ynew, knew, err);
      for (int i = 0; i < 12; ++i) { yl[i] = ynew[i]; k1[i] = knew[i]; }
      t += h;
    }
  }
}

// Same, in the Cartesian form (Eq. 1); x is [18].
void oracle_run_fixed_cartesian(const OSystem* s, double* x, double h, int64_t nsteps) {
  CartRHS f{s};
  double k1[18], xnew[18], knew[18], err[18];
  f(0.0, x, k1);
  double t = 0.0;
  for (int64_t it = 0; it < nsteps; ++it) {
    dopri5_step<18>(f, t, x, k1, h, xnew, knew, err);
    for (int i = 0; i < 18; ++i) { x[i] = xnew[i]; k1[i] = knew[i]; }
    t += h;
  }
}

// Initial conditions for n lanes.  levels[n_levels] must hold the levels the
// lanes reference through lvl[n] (an index into levels).  Outputs y[n][12],
// t_scale[n], E0[n], status[n], u_out[n][4] (may be null).  u_in[n][4]
// replaces the generator when non-null.
void oracle_init(const OSystem* sys, const int32_t* sys_id, const OLevel* levels,
                 const int32_t* lvl, const double* Ecol, const double* b, const int32_t* j,
                 int64_t n, double R0, uint64_t seed, uint64_t id_offset, const double* u_in,
                 double* y, double* t_scale, double* E0, int32_t* status, double* u_out) {
  for (int64_t i = 0; i < n; ++i) {
    const OLevel& L = levels[lvl[i]];
    if (!L.ok) { status[i] = kStatusNoLevel; continue; }
    status[i] = init_lane(sys[sys_id[i]], L, Ecol[i], b[i], j[i], R0, seed, id_offset + i,
                          u_in ? u_in + 4 * i : nullptr, y + 12 * i, t_scale + i, E0 + i,
                          u_out ? u_out + 4 * i : nullptr);
  }
}

// Adaptive integration + product analysis of n lanes (y updated in place).
void oracle_run_adaptive(const OSystem* sys, const int32_t* sys_id, const OInteg* in,
                         double* y, const double* t_scale, const double* E0,
                         const int32_t* status_in, int64_t n, OResult* out) {
  for (int64_t i = 0; i < n; ++i) {
    OResult& r = out[i];
    std::memset(&r, 0, sizeof(r));
    if (status_in[i] != kStatusReady) { r.status = status_in[i]; r.cls = kClsFail; continue; }
    const OSystem& s = sys[sys_id[i]];
    r.status = integrate_adaptive(s, *in, y + 12 * i, t_scale[i], &r.t, &r.nsteps, &r.nrej);
    analyze(s, *in, y + 12 * i, E0[i], r.status, &r);
  }
}

// Product analysis alone (status given per lane).
void oracle_analyze(const OSystem* sys, const int32_t* sys_id, const OInteg* in,
                    const double* y, const double* E0, const int32_t* status, int64_t n,
                    OResult* out) {
  for (int64_t i = 0; i < n; ++i) {
    std::memset(&out[i], 0, sizeof(OResult));
    out[i].status = status[i];
    analyze(sys[sys_id[i]], *in, y + 12 * i, E0[i], status[i], &out[i]);
  }
}

// Histogram reduction (Sec. 2.3: counts N_x per (E_c, b) cell, Gaussian-binned
// v' sums, rotational bins) into hist[n_cells][H_STRIDE].  Lanes with a status
// other than DONE count as class FAIL.  isw may be null (weight 1).
void oracle_reduce(int64_t n, const int32_t* cls, const int32_t* vt, const int32_t* jt,
                   const double* gbw, const double* isw, const int32_t* cell, int32_t n_cells,
                   int64_t* hist) {
  std::memset(hist, 0, sizeof(int64_t) * H_STRIDE * (size_t)n_cells);
  for (int64_t i = 0; i < n; ++i) {
    int c = cell[i];
    if (c < 0 || c >= n_cells) continue;
    int64_t* H = hist + (int64_t)H_STRIDE * c;
    int k = cls[i];
    H[H_COUNT + k] += 1;
    H[H_COUNT + 6] += 1;
    double w = isw ? isw[i] : 1.0;
    H[H_W + k] += fixed_point(w);
    H[H_W2 + k] += fixed_point(w * w);
    if (k <= 2) {
      int v = std::min(vt[i], N_VT - 1);
      int jj = std::min(jt[i], N_JT - 1);
      H[H_VT + N_VT * k + v] += 1;
      H[H_JT + N_JT * k + jj] += 1;
      H[H_GB + N_VT * k + v] += fixed_point(gbw[i]);
    }
  }
}

// Cross sections from the histograms, Sec. 2.3 (opacity P = N_x / N with the
// binomial error delta, Eq. 16) and the cross-section integral of Sec. 4 read
// as sigma_x = 2 pi int P_x(b) b db (the printed prefactor is garbled),
// evaluated as 2 pi sum_c w_c b_c P_x(c) with caller-given quadrature
// weights w_c; the standard error is 2 pi sqrt(sum_c (w_c b_c delta_c)^2).
// N excludes FAIL.  Entries k = 0..5 are the classes, k = 6 the reactive
// total R_AC + R_BC.  Weighted mode uses P = sum w 1_x / N and its sample
// standard error.  out: per cell [7][P, delta] then per group [7][sigma, SE].
void oracle_xsec(const int64_t* hist, int32_t n_cells, const double* cell_b,
                 const double* cell_w, const int32_t* group, int32_t n_groups,
                 int32_t weighted, double* out) {
  const int NE = 7;
  double* grp = out + 2 * NE * (size_t)n_cells;
  std::memset(grp, 0, sizeof(double) * 2 * NE * (size_t)n_groups);
  double* var = new double[NE * (size_t)(n_groups > 0 ? n_groups : 1)]();
  for (int c = 0; c < n_cells; ++c) {
    const int64_t* H = hist + (int64_t)H_STRIDE * c;
    double N = 0.0;
    for (int k = 0; k < 5; ++k) N += double(H[H_COUNT + k]);
    for (int k = 0; k < NE; ++k) {
      // the reactive total: classes R_AC (1) and R_BC (2) are exclusive
      double Nx = k < 6 ? double(H[H_COUNT + k]) : double(H[H_COUNT + 1] + H[H_COUNT + 2]);
      double swf = k < 6 ? double(H[H_W + k]) : double(H[H_W + 1] + H[H_W + 2]);
      double sw2f = k < 6 ? double(H[H_W2 + k]) : double(H[H_W2 + 1] + H[H_W2 + 2]);
      double P = 0.0, d = 0.0;
      if (N > 0) {
        if (!weighted) {
          P = Nx / N;
          d = std::sqrt(Nx) / N * std::sqrt((N - Nx) / N);
        } else {
          double sw = std::ldexp(swf, -32);
          double sw2 = std::ldexp(sw2f, -32);
          P = sw / N;
          double m2 = sw2 / N;
          d = N > 1 ? std::sqrt(std::max(0.0, m2 - P * P) / (N - 1.0)) : 0.0;
        }
      }
      out[2 * NE * (size_t)c + 2 * k] = P;
      out[2 * NE * (size_t)c + 2 * k + 1] = d;
      int g = group[c];
      if (g >= 0 && g < n_groups) {
        double wb = cell_w[c] * cell_b[c];
        grp[2 * NE * (size_t)g + 2 * k] += 2.0 * kPi * wb * P;
        var[NE * (size_t)g + k] += (wb * d) * (wb * d);
      }
    }
  }
  for (int g = 0; g < n_groups; ++g)
    for (int k = 0; k < NE; ++k)
      grp[2 * NE * (size_t)g + 2 * k + 1] = 2.0 * kPi * std::sqrt(var[NE * (size_t)g + k]);
  delete[] var;
}

// Rate constant of Sec. 4 (Eq. 19): k = sigma sqrt(2 E / mu), with mu the
// atom-molecule reduced mass mu123 (reading of the unlabelled mu).
void oracle_rates(const double* sigma, const double* E, int32_t n, double mu123, double* k) {
  for (int i = 0; i < n; ++i) k[i] = sigma[i] * std::sqrt(2.0 * E[i] / mu123);
}

// Gaussian-binning product distributions, Sec. 2.3 (Eqs. 14-15): over the
// selected cells, P_c(v_t) = sum_i W_c^i(v_t) / W with the total weight
// W = sum over v_t of the reaction and quench weight sums plus N_d (each
// dissociation weighs 1).  out[3][64] for c = Q, R_AC, R_BC; returns W.
double oracle_gb_distribution(const int64_t* hist, const int32_t* cells, int32_t n_sel,
                              double* out) {
  double W = 0.0;
  for (int k = 0; k < 3 * N_VT; ++k) out[k] = 0.0;
  for (int s = 0; s < n_sel; ++s) {
    const int64_t* H = hist + (int64_t)H_STRIDE * cells[s];
    for (int c = 0; c < 3; ++c)
      for (int v = 0; v < N_VT; ++v) out[N_VT * c + v] += std::ldexp(double(H[H_GB + N_VT * c + v]), -32);
    W += double(H[H_COUNT + kClsD]);
  }
  for (int k = 0; k < 3 * N_VT; ++k) W += out[k];
  for (int k = 0; k < 3 * N_VT; ++k) out[k] /= W;
  return W;
}

}  // extern "C"
