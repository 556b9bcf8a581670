"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

None of these tests retypes an oracle formula: each checks the oracle against
a closed form, a published value, an invariant, an independent library
computation (scipy / mpmath / exact rational arithmetic), or a limit in which
the method reduces to a textbook result.  Citations name the section or
equation of Koots & Perez-Rios (PyQCAMS) that each oracle function follows.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2304_02731_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# Philox4x32-10 (random orientation / phase, Sec. 2.1): published vectors.
# ---------------------------------------------------------------------------
def test_philox_known_answers(oracle):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        ctr = [int(x, 16) for x in r[0:4]]
        key = [int(x, 16) for x in r[4:6]]
        want = [int(x, 16) for x in r[6:10]]
        assert list(oracle.philox4x32_10(ctr, key)) == want


# ---------------------------------------------------------------------------
# Potentials (Sec. 3.2 items 1-3) and set-up.
# ---------------------------------------------------------------------------
def _systems(oracle):
    return {name: oracle.system_from_spec(sp) for name, sp in
            [("morse", W.SYS_H2_CA_MORSE), ("buck", W.SYS_H2_CA_BUCK),
             ("lj12", W.SYS_H2_CA_LJ12), ("lj8", W.SYS_H2_CA_LJ8)]}


def test_potential_derivatives_match_finite_differences(oracle):
    for s in _systems(oracle).values():
        for k in range(3):
            for r in np.linspace(1.0, 20.0, 23):
                h = 1e-5 * r
                Vp, _ = oracle.pair_potential(s.pair[k], r + h)
                Vm, _ = oracle.pair_potential(s.pair[k], r - h)
                _, dV = oracle.pair_potential(s.pair[k], r)
                fd = (Vp - Vm) / (2 * h)
                # truncation O(h^2) plus the cancellation in V (~1e-16 hartree) / h
                assert abs(fd - dV) <= 1e-6 * abs(dV) + 1e-15 / h


@pytest.mark.parametrize("name", ["lj12", "lj8"])
def test_lj_fit_reproduces_well(oracle, name):
    """Generalized LJ fitted to (De, re): a minimum of depth De at re."""
    s = _systems(oracle)[name]
    V, dV = oracle.pair_potential(s.pair[2], 3.79)
    assert abs(V + 0.0630) < 1e-14
    assert abs(dV) < 1e-14
    from scipy.optimize import minimize_scalar
    res = minimize_scalar(lambda r: oracle.pair_potential(s.pair[2], r)[0],
                          bounds=(3.0, 5.0), method="bounded", options=dict(xatol=1e-10))
    assert abs(res.x - 3.79) < 1e-6


def test_morse_alpha_from_harmonic_constant(oracle):
    """Morse given by omega_e (the paper's input form): the j=0 spacing of the
    Bohr-Sommerfeld levels reproduces omega_e - 2 omega_e x_e with
    omega_e x_e = omega_e^2 / (4 De) (Morse closed form)."""
    we, De, re = 0.02005340207, 0.16456603489, 1.40104284795   # H2 input listing, Sec. 3.1
    spec = dict(mass_u=(1837.47165336 / 1822.888486209, 1837.47165336 / 1822.888486209,
                        73046.7897752 / 1822.888486209),
                pairs=(("morse_we", De, re, we), W.CAH_MORSE, W.CAH_MORSE))
    s = oracle.system_from_spec(spec)
    mu = oracle.reduced_masses(s)["mu12"]
    E0 = oracle.level(s.pair[0], mu, 0, 0).E
    E1 = oracle.level(s.pair[0], mu, 1, 0).E
    assert abs((E1 - E0) - (we - 2 * we * we / (4 * De))) < 1e-12
    assert abs(E0 - (-De + we / 2 - we * we / (16 * De))) < 1e-12


def test_buckingham_stationary_points(oracle):
    """Buckingham short-range maximum and well located by an independent
    bounded scalar optimiser on V itself."""
    from scipy.optimize import minimize_scalar
    s = _systems(oracle)["buck"]
    mu = oracle.reduced_masses(s)["mu_CA"]
    st = oracle.stationary(s.pair[2], mu, 0.0)
    V = lambda r: oracle.pair_potential(s.pair[2], r)[0]
    mx = minimize_scalar(lambda r: -V(r), bounds=(1.0, 3.5), method="bounded",
                         options=dict(xatol=1e-10))
    mn = minimize_scalar(V, bounds=(4.0, 15.0), method="bounded", options=dict(xatol=1e-10))
    assert st["has_well"]
    assert abs(st["r_inner"] - mx.x) < 1e-5
    assert abs(st["r_min"] - mn.x) < 1e-5
    assert st["threshold"] == 0.0


# ---------------------------------------------------------------------------
# Bohr-Sommerfeld levels (Sec. 2.1, tau; Sec. 2.2, v').
# ---------------------------------------------------------------------------
def _morse_closed(De, a, mu, v):
    w = a * math.sqrt(2 * De / mu)
    E = -De + w * (v + 0.5) - w * w * (v + 0.5) ** 2 / (4 * De)
    tau = 2 * math.pi / a * math.sqrt(mu / (2 * abs(E)))
    return E, tau


def test_morse_j0_levels_match_closed_form(oracle):
    """For Morse, the Bohr-Sommerfeld rule with the 1/2 is exact: levels,
    turning points and classical periods equal their closed forms."""
    s = _systems(oracle)["morse"]
    mu = oracle.reduced_masses(s)["mu12"]
    De, re, a = 0.1745, 1.40, 1.03
    nbound = 0
    for v in range(0, 20):
        L = oracle.level(s.pair[0], mu, v, 0)
        E, tau = _morse_closed(De, a, mu, v)
        if E >= 0 or (v + 0.5) > math.sqrt(2 * mu * De) / a:
            assert not L.ok
            continue
        nbound += 1
        assert L.ok
        assert abs(L.E - E) <= 1e-10 * abs(E)
        x = math.sqrt(1 + E / De)
        assert abs(L.r_plus - (re - math.log(1 - x) / a)) <= 1e-10 * L.r_plus
        assert abs(L.r_minus - (re - math.log(1 + x) / a)) <= 1e-10 * L.r_minus
        assert abs(L.tau - tau) <= 1e-9 * tau
    assert nbound == 17


def test_morse_action_closed_form(oracle):
    """v(E) = sqrt(2 mu De)/alpha (1 - sqrt(|E|/De)) - 1/2 for Morse, L = 0."""
    s = _systems(oracle)["morse"]
    mu = oracle.reduced_masses(s)["mu12"]
    De, a = 0.1745, 1.03
    for E in np.linspace(-0.17, -0.001, 17):
        want = math.sqrt(2 * mu * De) / a * (1 - math.sqrt(abs(E) / De)) - 0.5
        assert abs(oracle.v_of_E(s.pair[0], mu, 0.0, E) - want) < 1e-10


def _mp_action_and_period(V, mu, L2, E, r_lo, r_min, r_hi):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    Veff = lambda r: V(r) + mp.mpf(L2) / (2 * mu * r * r)
    rm = mp.findroot(lambda r: Veff(r) - E, (mp.mpf(r_lo), mp.mpf(r_min)), solver="anderson")
    rp = mp.findroot(lambda r: Veff(r) - E, (mp.mpf(r_min), mp.mpf(r_hi)), solver="anderson")
    c, d = (rp + rm) / 2, (rp - rm) / 2
    act = mp.quad(lambda s: mp.sqrt(max(E - Veff(c + d * mp.sin(s)), 0)) * d * mp.cos(s),
                  [-mp.pi / 2, mp.pi / 2])
    per = mp.quad(lambda r: 1 / mp.sqrt(E - Veff(r)), [rm, rp])
    return (float(-0.5 + mp.sqrt(2 * mu) / mp.pi * act), float(mp.sqrt(2 * mu) * per))


@pytest.mark.parametrize("name,pair,v,j", [("morse", 0, 3, 7), ("morse", 0, 8, 15),
                                           ("lj12", 2, 2, 5), ("lj8", 2, 1, 12),
                                           ("morse", 2, 4, 20)])
def test_levels_against_mpmath(oracle, name, pair, v, j):
    """j > 0 and non-Morse levels: an independent 30-digit mpmath computation
    (Anderson root finding for the turning points, tanh-sinh quadrature of the
    action and of the period) at the oracle's E_vj gives v and tau."""
    mp = pytest.importorskip("mpmath")
    s = _systems(oracle)[name]
    rm_ = oracle.reduced_masses(s)
    mu = rm_["mu12"] if pair == 0 else rm_["mu_CA"]
    q = s.pair[pair]
    L = oracle.level(q, mu, v, j)
    assert L.ok
    p = [q.p[i] for i in range(5)]
    if q.kind == 0:
        De, re, a = p[:3]
        V = lambda r: De * (1 - mp.exp(-a * (r - re))) ** 2 - De
    else:
        m, n, Cm, Cn = p[:4]
        V = lambda r: Cm / r ** int(m) - Cn / r ** int(n)
    L2 = j * (j + 1)
    vv, tau = _mp_action_and_period(V, mp.mpf(mu), L2, mp.mpf(L.E), L.r_minus * 0.9,
                                    L.r_min, L.r_plus * 1.05)
    assert abs(vv - v) < 1e-9
    assert abs(tau - L.tau) < 1e-8 * tau


def test_level_table_of_mixed_study(oracle):
    """H2 Morse holds 230 of the 231 (v<=10, j<=20) levels; (10, 20) is the
    missing one, and levels rise with v and with j."""
    s = _systems(oracle)["morse"]
    mu = oracle.reduced_masses(s)["mu12"]
    E = np.full((11, 21), np.nan)
    for v in range(11):
        for j in range(21):
            L = oracle.level(s.pair[0], mu, v, j)
            if L.ok:
                E[v, j] = L.E
    assert np.isnan(E).sum() == 1 and np.isnan(E[10, 20])
    assert np.all(np.diff(E[:10], axis=0) > 0)
    assert np.all(np.diff(E[:, :20], axis=1) > 0)


# ---------------------------------------------------------------------------
# Hamilton's equations (Eqs. 2-4) and the Cartesian form (Eq. 1).
# ---------------------------------------------------------------------------
def _state(oracle, name="morse", seed=3, b=2.0, E=0.1, v=1, j=3, R0=8.0):
    s = _systems(oracle)[name]
    st = oracle.init([s], [0], [E], [b], [v], [j], R0, seed)
    return s, st


def test_rhs_is_the_hamiltonian_gradient(oracle):
    for name in ["morse", "lj12", "buck"]:
        s, st = _state(oracle, name, R0=5.0, b=1.0, v=0, j=2)
        y = st["y"][0].copy()
        y[3:6] = [0.7, -1.1, -4.0]   # bring C into the interaction region
        dy = oracle.rhs(s, y)
        for i in range(12):
            h = 1e-6 * max(1.0, abs(y[i]))
            yp, ym = y.copy(), y.copy()
            yp[i] += h
            ym[i] -= h
            g = (oracle.hamiltonian(s, yp) - oracle.hamiltonian(s, ym)) / (2 * h)
            want = g if i >= 6 else -g       # d rho/dt = dH/dP ; dP/dt = -dH/drho
            idx = i - 6 if i >= 6 else i + 6
            assert abs(dy[idx] - want) <= 1e-6 * max(1e-4, abs(want))


def test_cartesian_and_jacobi_agree(oracle):
    """Runge-Kutta steps commute with the linear change of variables between
    Eq. 1 and Eq. 2, so fixed-step runs in the two forms agree to rounding;
    the Cartesian total momentum stays zero (a linear invariant)."""
    s, st = _state(oracle, R0=6.0, b=1.5, E=0.15)
    y0 = st["y"][0]
    x0 = oracle.jacobi_to_cartesian(s, y0)
    assert np.allclose(oracle.cartesian_to_jacobi(s, x0), y0, rtol=1e-14, atol=1e-14)
    P = x0[9:12] + x0[12:15] + x0[15:18]
    assert np.all(np.abs(P) < 1e-12)
    yj = oracle.run_fixed(s, y0, 0.5, 1500)[0]
    xc = oracle.run_fixed_cartesian(s, x0, 0.5, 1500)
    yc = oracle.cartesian_to_jacobi(s, xc)
    scale = np.abs(yj) + 1.0
    assert np.max(np.abs(yj - yc) / scale) < 1e-9
    P = xc[9:12] + xc[12:15] + xc[15:18]
    assert np.all(np.abs(P) < 1e-10)


# ---------------------------------------------------------------------------
# Dormand-Prince 5(4) (Sec. 3.2: SciPy solve_ivp RK45).
# ---------------------------------------------------------------------------
def _trees(order):
    """All rooted trees with `order` nodes as sorted tuples of child subtrees."""
    memo = {1: [()]}

    def trees(n):
        if n in memo:
            return memo[n]
        out = set()

        def forests(m, max_t):
            # multisets of trees with total size m, children sorted (non-increasing key)
            if m == 0:
                yield ()
                return
            for k in range(1, m + 1):
                for t in trees(k):
                    key = (k, repr(t))
                    if max_t is not None and key > max_t:
                        continue
                    for rest in forests(m - k, key):
                        yield (t,) + rest

        for f in forests(n - 1, None):
            out.add(tuple(sorted(f, key=repr)))
        memo[n] = sorted(out, key=repr)
        return memo[n]

    return trees(order)


def _size(t):
    return 1 + sum(_size(c) for c in t)


def _gamma(t):
    g = _size(t)
    for c in t:
        g *= _gamma(c)
    return g


def _phi(t, A):
    """Elementary weight vector: prod over children of A . phi(child)."""
    n = len(A)
    v = [Fraction(1)] * n
    for c in t:
        pc = _phi(c, A)
        Ac = [sum(A[i][k] * pc[k] for k in range(n)) for i in range(n)]
        v = [v[i] * Ac[i] for i in range(n)]
    return v


def _tableau_exact(oracle):
    c, a, b, bs = oracle.dopri5_tableau()
    F = lambda x: Fraction(float(x)).limit_denominator(10 ** 7)
    A = [[F(a[i, k]) for k in range(7)] for i in range(7)]
    return [F(x) for x in c], A, [F(x) for x in b], [F(x) for x in bs]


def test_dopri5_order_conditions(oracle):
    """Butcher order conditions over all rooted trees: the propagated weights
    have order 5 (17 trees), the embedded weights order 4 (8 trees) but not 5,
    and c_i is the row sum of A."""
    c, A, b, bs = _tableau_exact(oracle)
    for i in range(7):
        assert sum(A[i]) == c[i]
    counts = [len(_trees(k)) for k in range(1, 6)]
    assert counts == [1, 1, 2, 4, 9]
    for order in range(1, 6):
        for t in _trees(order):
            ph = _phi(t, A)
            assert sum(b[i] * ph[i] for i in range(7)) == Fraction(1, _gamma(t))
            if order <= 4:
                assert sum(bs[i] * ph[i] for i in range(7)) == Fraction(1, _gamma(t))
    fifth = [sum(bs[i] * p for i, p in enumerate(_phi(t, A))) == Fraction(1, _gamma(t))
             for t in _trees(5)]
    assert not all(fifth)
    # FSAL: the last stage is evaluated at the propagated solution
    assert A[6][:6] == b[:6] and b[6] == 0 and c[6] == 1


def test_dopri5_rkn_products_zero_exactly_where_the_integrators_skip(oracle):
    """The CUDA integrators use the Runge-Kutta-Nystrom products (A^2)_{sq}
    for the stage positions and (e^T A)_q for the position error (Sec. 3.2's
    Dormand-Prince step written for rho'' = a) and skip the terms they take
    to be zero: (A^2)_{sq} for q >= s - 1 and for (s, q) = (7, 2), (e^T A)_q
    for q = 2 and 7.  In exact arithmetic on the tableau those are zero,
    (A^2)_{7q} = b_q (1 - c_q), and every other product is nonzero, so the
    skipped set is exactly the zero set."""
    c, A, b, bs = _tableau_exact(oracle)
    e = [b[i] - bs[i] for i in range(7)]
    A2 = [[sum(A[s][j] * A[j][q] for j in range(7)) for q in range(7)] for s in range(7)]
    eA = [sum(e[i] * A[i][q] for i in range(7)) for q in range(7)]
    for s in range(1, 7):            # 0-based stage s + 1 = 2..7
        for q in range(s):           # 0-based q + 1 = 1..s
            skipped = q >= s - 1 or (s, q) == (6, 1)
            assert (A2[s][q] == 0) == skipped, (s + 1, q + 1, A2[s][q])
    for q in range(7):
        assert A2[6][q] == b[q] * (1 - c[q])
        assert (eA[q] == 0) == (q in (1, 6)), (q + 1, eA[q])


def test_dopri5_stability_polynomial(oracle):
    """One step on y' = lambda y multiplies y by R(z) = 1 + sum b^T A^(k-1) 1 z^k;
    for Dormand-Prince 5(4) the z^6 coefficient is 1/600."""
    c, A, b, bs = _tableau_exact(oracle)
    coef = [Fraction(1)]
    vec = [Fraction(1)] * 7
    for k in range(1, 8):
        coef.append(sum(b[i] * vec[i] for i in range(7)))
        vec = [sum(A[i][m] * vec[m] for m in range(7)) for i in range(7)]
    assert coef[:6] == [Fraction(1, math.factorial(k)) for k in range(6)]
    assert coef[6] == Fraction(1, 600) and coef[7] == 0
    for z in [-2.5, -1.0, -0.3, 0.2, 1.1]:
        y1, _ = oracle.dopri5_linear(z, 1.0)
        R = sum(float(coef[k]) * z ** k for k in range(8))
        assert abs(y1 - R) <= 1e-14 * max(1.0, abs(R))


def test_fixed_step_global_order_five(oracle):
    s, st = _state(oracle, R0=7.0, b=1.0, E=0.12, v=2, j=4)
    y0 = st["y"][0]
    T = 240.0
    ref = oracle.run_fixed(s, y0, T / 3840, 3840)[0]
    errs = []
    for n in [120, 240, 480]:
        y = oracle.run_fixed(s, y0, T / n, n)[0]
        errs.append(np.max(np.abs(y - ref)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 24 < r1 < 42 and 24 < r2 < 42, (errs, r1, r2)


def test_fixed_step_time_reversal(oracle):
    """Forward N steps, flip the momenta, N steps back: the start state returns
    up to the method's h^5 asymmetry (Dormand-Prince is not symmetric)."""
    s, st = _state(oracle, R0=12.0, b=2.0, E=0.1, v=1, j=2)
    y0 = st["y"][0]
    y = oracle.run_fixed(s, y0, 0.25, 2000)[0]
    y[6:] *= -1
    y = oracle.run_fixed(s, y, 0.25, 2000)[0]
    y[6:] *= -1
    assert np.max(np.abs(y - y0) / (np.abs(y0) + 1.0)) < 1e-8


# ---------------------------------------------------------------------------
# Initial conditions (Sec. 2.1, Eq. 5-6) and the analysis (Sec. 2.2).
# ---------------------------------------------------------------------------
def test_initial_state_invariants(oracle):
    s = _systems(oracle)["morse"]
    mu = oracle.reduced_masses(s)
    n = 64
    rng = np.random.default_rng(5)
    E = rng.uniform(0.02, 0.4, n)
    b = rng.uniform(0, 8, n)
    v = rng.integers(0, 8, n)
    j = rng.integers(0, 15, n)
    st = oracle.init([s], np.zeros(n, np.int32), E, b, v, j, 30.0, 11)
    assert np.all(st["status"] == 0)
    for i in range(n):
        y = st["y"][i]
        rho1, rho2, P1, P2 = y[0:3], y[3:6], y[6:9], y[9:12]
        L = oracle.level(s.pair[0], mu["mu12"], v[i], j[i])
        assert abs(np.dot(rho1, P1)) < 1e-12
        assert abs(np.linalg.norm(rho1) - L.r_plus) < 1e-13
        assert abs(np.linalg.norm(P1) * L.r_plus - math.sqrt(j[i] * (j[i] + 1))) < 1e-12
        P2m = math.sqrt(2 * mu["mu123"] * E[i])
        assert abs(np.linalg.norm(np.cross(rho2, P2)) - b[i] * P2m) < 1e-10
        R = np.linalg.norm(rho2)
        chi = st["u"][i, 3]
        assert abs(R - (30.0 + chi * P2m * L.tau / mu["mu123"])) < 1e-10
        assert np.dot(rho2, P2) < 0
        # E0 = E_vj + E_col + the (small) atom-molecule interaction at the start
        rAC = np.linalg.norm(rho2 + s.m[1] / (s.m[0] + s.m[1]) * rho1)
        rBC = np.linalg.norm(rho2 - s.m[0] / (s.m[0] + s.m[1]) * rho1)
        Vint = oracle.pair_potential(s.pair[2], rAC)[0] + oracle.pair_potential(s.pair[1], rBC)[0]
        assert abs(st["E0"][i] - (L.E + E[i] + Vint)) < 1e-13


def test_orientation_angles_are_uniform(oracle):
    """cos(theta), phi, eta, chi uniform (Sec. 2.3: dOmega = sin(theta) dtheta
    dphi deta dchi): Kolmogorov-Smirnov against U(0,1) for the four uniforms."""
    from scipy.stats import kstest
    s = _systems(oracle)["morse"]
    n = 4000
    st = oracle.init([s], np.zeros(n, np.int32), np.full(n, 0.1), np.zeros(n),
                     np.zeros(n, np.int32), np.zeros(n, np.int32), 30.0, 0)
    for k in range(4):
        assert kstest(st["u"][:, k], "uniform").pvalue > 1e-3
    y = st["y"]
    cth = y[:, 2] / np.linalg.norm(y[:, 0:3], axis=1)
    assert kstest((cth + 1) / 2, "uniform").pvalue > 1e-3


@pytest.mark.parametrize("v,j", [(0, 0), (1, 0), (3, 5), (6, 12), (9, 2)])
def test_init_then_analysis_round_trip(oracle, v, j):
    """A molecule prepared in (v, j) and analysed at once is a quench product
    with v' = v and j' = j (Sec. 2.1 and 2.2 use the same quantisation)."""
    s = _systems(oracle)["morse"]
    n = 8
    st = oracle.init([s], np.zeros(n, np.int32), np.full(n, 0.1), np.linspace(0, 5, n),
                     np.full(n, v, np.int32), np.full(n, j, np.int32), 30.0, 9)
    integ = oracle.make_integ()
    res = oracle.analyze([s], np.zeros(n, np.int32), integ, st["y"], st["E0"],
                         np.full(n, 2, np.int32))
    assert np.all(res["cls"] == 0)
    assert np.all(np.abs(res["vprime"] - v) < 1e-8)
    assert np.all(np.abs(res["jprime"] - j) < 1e-10)
    assert np.all(res["vt"] == v) and np.all(res["jt"] == j)
    assert np.all(np.abs(res["dE"]) < 1e-14)


def test_jprime_inverts_angular_momentum(oracle):
    s, st = _state(oracle, v=2, j=9)
    integ = oracle.make_integ()
    res = oracle.analyze([s], [0], integ, st["y"], st["E0"], [2])
    jp = res["jprime"][0]
    assert abs(jp * (jp + 1) - res["L2pair"][0, 0]) < 1e-10 * res["L2pair"][0, 0]


def test_gaussian_binning_weight_is_normal_density(oracle):
    """W(v', v_t) of Eq. 11 is the normal density N(v'; v_t, sigma)."""
    from scipy.stats import norm
    s = _systems(oracle)["morse"]
    wl = W.plain_h2_ca(per_b=3)
    integ = oracle.make_integ(**W.INTEG_FP64)
    st, res = oracle.run_lanes([s], wl.sys_id, wl.E, wl.b, wl.v, wl.j, wl.R0, wl.seed, integ)
    sig = integ.gb_sigma
    assert abs(sig * 2 * math.sqrt(2 * math.log(2)) - 0.1) < 1e-15   # FWHM 0.1
    for r in res:
        assert r["cls"] == 0
        assert abs(r["gbw"] - norm.pdf(r["vprime"], loc=r["vt"], scale=sig)) < 1e-12
        assert r["vt"] == max(0, int(round(r["vprime"])))


def test_bound_criterion_on_constructed_pairs(oracle):
    """The centrifugal barrier top r0 is a maximum of V_eff (Sec. 2.2); a pair
    below it inside r0 is bound, above it (or outside r0) is not."""
    s = _systems(oracle)["morse"]
    mu = oracle.reduced_masses(s)["mu12"]
    L2 = 12.0 * 13.0
    st = oracle.stationary(s.pair[0], mu, L2)
    assert st["has_well"] and st["has_top"]
    V = lambda r: oracle.pair_potential(s.pair[0], r)[0] + L2 / (2 * mu * r * r)
    r0 = st["r_top"]
    for d in [1e-3, 1e-2, 0.1]:
        assert V(r0) > V(r0 - d) and V(r0) > V(r0 + d)
        assert V(st["r_min"]) < V(st["r_min"] - d) and V(st["r_min"]) < V(st["r_min"] + d)
    assert st["threshold"] == pytest.approx(V(r0), rel=1e-15)
    assert oracle.stationary(s.pair[0], mu, 0.0)["threshold"] == 0.0


# ---------------------------------------------------------------------------
# Adaptive runs: conservation and the exactly known outcome of the plain study.
# ---------------------------------------------------------------------------
def _plain(oracle, t_stop):
    s = oracle.system_from_spec(W.SYS_H2_CA_MORSE)
    wl = W.plain_h2_ca(per_b=20)
    integ = oracle.make_integ(**dict(W.INTEG_FP64, t_stop=t_stop))
    st = oracle.init([s], wl.sys_id, wl.E, wl.b, wl.v, wl.j, wl.R0, wl.seed)
    y0 = st["y"].copy()
    res = oracle.run_adaptive([s], wl.sys_id, integ, st["y"], st["t_scale"], st["E0"],
                              st["status"])
    return s, wl, st, y0, res


@pytest.fixture(scope="module")
def plain_run(oracle):
    """The plain study's settings (t_stop = 15)."""
    return _plain(oracle, 15.0)


@pytest.fixture(scope="module")
def plain_run_long(oracle):
    """Same lanes with an effectively unlimited t_max, so that the few
    long-lived Ca-H2 complexes also break up before the analysis."""
    return _plain(oracle, 1000.0)


def test_adaptive_conservation(oracle, plain_run):
    s, wl, st, y0, res = plain_run
    rel = np.abs(res["dE"]) / np.maximum(np.abs(st["E0"]), wl.E)
    assert np.all(rel < 1e-8), rel.max()
    L0 = np.cross(y0[:, 0:3], y0[:, 6:9]) + np.cross(y0[:, 3:6], y0[:, 9:12])
    y = st["y"]
    L1 = np.cross(y[:, 0:3], y[:, 6:9]) + np.cross(y[:, 3:6], y[:, 9:12])
    dL = np.linalg.norm(L1 - L0, axis=1) / np.maximum(np.linalg.norm(L0, axis=1), 1.0)
    assert np.all(dL < 1e-8), dL.max()
    for i in range(0, wl.n, 25):
        x = oracle.jacobi_to_cartesian(s, y[i])
        assert np.all(np.abs(x[9:12] + x[12:15] + x[15:18]) < 1e-10)


def test_plain_study_is_all_quench(oracle, plain_run, plain_run_long):
    """E_tot = E_00 + E_col = -0.0646 hartree lies below the Ca-H well bottom
    (-0.063) and below 0: reaction and dissociation are closed, so every lane
    that separates is a quench and sigma_Q = 2 pi int_0^6 b db = 36 pi bohr^2
    exactly.  Lanes still inside a complex at t_max are never R or D."""
    s, wl, st, y0, res = plain_run
    assert np.all((res["cls"] == 0) | ((res["status"] == 3) & (res["cls"] == 4)))
    s, wl, st, y0, res = plain_run_long
    assert np.all(res["status"] == 2)
    assert np.all(res["cls"] == 0)
    hist = oracle.reduce(res["cls"], res["vt"], res["jt"], res["gbw"], wl.cell, wl.n_cells)
    cells, groups = oracle.xsec(hist, wl.cell_b, wl.cell_w, wl.cell_group, wl.n_groups)
    assert groups[0, 0, 0] == pytest.approx(36 * math.pi, rel=1e-14)
    assert groups[0, 0, 1] == 0.0
    for k in range(1, 6):
        assert groups[0, k, 0] == 0.0
    # the highest energetically open H2 level bounds v'
    mu = oracle.reduced_masses(s)["mu12"]
    Etot = oracle.level(s.pair[0], mu, 0, 0).E + 0.10
    vmax = max(v for v in range(17) if oracle.level(s.pair[0], mu, v, 0).E < Etot)
    assert res["vt"].max() <= vmax


# ---------------------------------------------------------------------------
# Reduction and cross sections (Sec. 2.3, Sec. 4).
# ---------------------------------------------------------------------------
def test_reduce_matches_brute_force(oracle):
    rng = np.random.default_rng(2)
    n, nc = 5000, 7
    cls = rng.integers(0, 6, n)
    vt = rng.integers(0, 80, n)
    jt = rng.integers(0, 300, n)
    gbw = rng.uniform(0, 9, n)
    isw = rng.uniform(0.2, 5, n)
    cell = rng.integers(0, nc, n)
    H = oracle.reduce(cls, vt, jt, gbw, cell, nc, isw)
    for c in range(nc):
        m = cell == c
        assert H[c, 6] == m.sum()
        for k in range(6):
            mk = m & (cls == k)
            assert H[c, k] == mk.sum()
            assert H[c, oracle.H_W + k] == sum(int(round(x * 2 ** 32)) for x in isw[mk])
            assert H[c, oracle.H_W2 + k] == sum(int(round(x * x * 2 ** 32)) for x in isw[mk])
            if k < 3:
                for vv in range(64):
                    sel = mk & (np.minimum(vt, 63) == vv)
                    assert H[c, oracle.H_VT + 64 * k + vv] == sel.sum()
                    assert H[c, oracle.H_GB + 64 * k + vv] == sum(
                        int(round(x * 2 ** 32)) for x in gbw[sel])
                assert H[c, oracle.H_JT + 256 * k:oracle.H_JT + 256 * (k + 1)].sum() == mk.sum()
                assert H[c, oracle.H_JT + 256 * k + 255] == (mk & (jt >= 255)).sum()


def test_xsec_binomial_error_and_linear_opacity(oracle):
    """delta is the binomial standard error sqrt(p(1-p)/N); with a constant
    opacity P the trapezoid sigma is exactly pi P b_max^2."""
    b = np.linspace(0, 6, 5)
    w = np.array([0.75, 1.5, 1.5, 1.5, 0.75])
    nc = 5
    H = np.zeros((nc, oracle.H_STRIDE), np.int64)
    N = 1000
    for c in range(nc):
        H[c, 0] = 250
        H[c, 1] = 670
        H[c, 2] = 30
        H[c, 3] = 50
        H[c, 5] = 17     # failures are excluded from N
        H[c, 6] = N + 17
    cells, groups = oracle.xsec(H, b, w, np.zeros(nc, np.int32), 1)
    # entry 6 is the reactive total R_AC + R_BC
    for k, cnt in [(0, 250), (1, 670), (2, 30), (3, 50), (6, 700)]:
        p = cnt / N
        assert cells[0, k, 0] == pytest.approx(p, rel=1e-15)
        assert cells[0, k, 1] == pytest.approx(math.sqrt(p * (1 - p) / N), rel=1e-13)
        assert groups[0, k, 0] == pytest.approx(math.pi * p * 36, rel=1e-13)
        se = 2 * math.pi * math.sqrt(sum((wi * bi) ** 2 for wi, bi in zip(w, b))) * \
            math.sqrt(p * (1 - p) / N)
        assert groups[0, k, 1] == pytest.approx(se, rel=1e-13)


def test_weighted_xsec_is_the_sample_mean_of_weighted_indicators(oracle):
    """Importance-weighted mode: P_x = mean(w 1_x) over the non-failed lanes
    and delta_x its standard error (sample variance / N), per class and for
    the reactive total; checked against the per-lane definition."""
    rng = np.random.default_rng(8)
    n = 4000
    cls = rng.choice(6, n, p=[0.6, 0.1, 0.08, 0.12, 0.05, 0.05])
    w = rng.uniform(0.2, 5.0, n)
    z = np.zeros(n, np.int32)
    H = oracle.reduce(cls, z, z, np.zeros(n), z, 1, w)
    cells, groups = oracle.xsec(H, [1.0], [50.0], [0], 1, weighted=True)
    ok = cls != 5
    N = ok.sum()
    for k, sel in [(0, cls == 0), (1, cls == 1), (2, cls == 2), (3, cls == 3),
                   (6, (cls == 1) | (cls == 2))]:
        y = (w * sel)[ok]
        assert cells[0, k, 0] == pytest.approx(y.mean(), rel=1e-9)
        assert cells[0, k, 1] == pytest.approx(y.std(ddof=1) / math.sqrt(N), rel=1e-9)
        assert groups[0, k, 0] == pytest.approx(math.pi * 100.0 * y.mean(), rel=1e-9)


def test_rate_is_sigma_times_initial_relative_speed(oracle):
    """k = sigma sqrt(2 E / mu123) equals sigma times the speed at which the
    atom approaches the molecule in the initial state (|d rho2 / dt|)."""
    s = oracle.system_from_spec(W.SYS_H2_CA_MORSE)
    mu = oracle.reduced_masses(s)["mu123"]
    E = np.array([0.02, 0.1, 0.4])
    st = oracle.init([s], np.zeros(3, np.int32), E, np.zeros(3), np.zeros(3, np.int32),
                     np.zeros(3, np.int32), 30.0, 0)
    speed = np.linalg.norm(st["y"][:, 9:12], axis=1) / mu
    k = oracle.rates(np.array([2.0, 3.0, 5.0]), E, mu)
    assert np.allclose(k, np.array([2.0, 3.0, 5.0]) * speed, rtol=1e-14)


def test_gb_distribution_normalisation_and_integer_case(oracle):
    """Eqs. 14-15: the channel distributions plus the dissociation share
    N_d / W sum to one; when every v' is an integer each lane carries the peak
    weight 1/(sigma sqrt(2 pi)), so P_c(v) = n_c(v) / (n_bound + N_d s sqrt(2 pi))."""
    rng = np.random.default_rng(4)
    n = 3000
    cls = rng.choice(6, n, p=[0.5, 0.15, 0.15, 0.1, 0.05, 0.05])
    vt = rng.integers(0, 12, n)
    sig = 0.042466
    peak = 1.0 / (sig * math.sqrt(2 * math.pi))
    gbw = np.where(cls <= 2, peak, 0.0)
    cell = rng.integers(0, 3, n)
    H = oracle.reduce(cls, vt, np.zeros(n, np.int32), gbw, cell, 3)
    P, Wt = oracle.gb_distribution(H, [0, 2])
    sel = (cell == 0) | (cell == 2)
    Nd = np.sum(sel & (cls == 3))
    assert P.sum() + Nd / Wt == pytest.approx(1.0, rel=1e-12)
    nb = np.sum(sel & (cls <= 2))
    for c in range(3):
        for v in range(12):
            ncv = np.sum(sel & (cls == c) & (vt == v))
            assert P[c, v] == pytest.approx(ncv / (nb + Nd / peak), rel=1e-9, abs=1e-15)


def test_adaptive_controller_matches_scipy_rk45(oracle):
    """The oracle's step-size control (starting step, error norm, factors,
    no growth after a rejection) restates SciPy's RK45, which the paper uses
    (Sec. 3.2): stepping scipy.integrate.RK45 itself on the oracle's
    Hamilton equations from the same initial state, with the stop rules out
    of the way (r_stop far away, t_max = 800 atomic time units), gives the
    same number of accepted steps, the same end time up to rounding-level
    step-size differences, and the same state there within the tolerance."""
    from scipy.integrate import RK45
    s = oracle.system_from_spec(W.SYS_H2_CA_MORSE)
    for E, b, v, j, rtol, atol in [(0.10, 1.5, 0, 0, 1e-10, 1e-12), (0.05, 4.0, 2, 5, 1e-8, 1e-10)]:
        st = oracle.init([s], np.zeros(1, np.int32), [E], [b], [v], [j], 30.0, 3)
        y0 = st["y"][0].copy()
        t_stop = 800.0 / st["t_scale"][0]          # t_max = 800 atomic time units
        integ = oracle.make_integ(rtol=rtol, atol=atol, r_stop=1e6, t_stop=t_stop)
        y = st["y"].copy()
        res = oracle.run_adaptive([s], np.zeros(1, np.int32), integ, y, st["t_scale"], st["E0"],
                                  st["status"])
        assert res["status"][0] == 3                  # stopped by t_max
        t_end, n_acc = res["t"][0], int(res["nsteps"][0])
        solver = RK45(lambda t, x: oracle.rhs(s, x), 0.0, y0, t_bound=1e9, rtol=rtol, atol=atol)
        n = 0
        while solver.t < 800.0:
            solver.step()
            assert solver.status == "running"
            n += 1
        assert n == n_acc, (n, n_acc)
        # the error estimate is a cancellation (5th- minus 4th-order
        # solution), so its relative rounding error is ~eps / rtol ~ 1e-6 and
        # two valid summation orders give step sizes that differ at that
        # level: the times agree to ~1e-8, and the states at the oracle's end
        # time (SciPy's dense output of its last step) to the tolerance
        dt = abs(solver.t - t_end) / t_end
        yi = solver.dense_output()(t_end)
        dy = np.max(np.abs(yi - y[0]) / (np.abs(y[0]) + 1.0))
        print(f"\nrtol {rtol:g}: {n} accepted steps both; |dt|/t {dt:.1e}, state {dy:.1e}")
        assert dt < 1e-7 and dy < 100 * rtol


# ---------------------------------------------------------------------------
# Stop rules (Sec. 3.1: r_stop, the largest distance between any two atoms;
# t_stop, a multiple of the trajectory's time scale d / v_c) and the
# Buckingham collapse (Sec. 3.2 item 3, the short-range "max").
#
# Each rule is checked against an independent integration: scipy's RK45
# (pinned to the oracle's controller above) stepped on Hamilton's equations,
# with the rule evaluated after every accepted step on CARTESIAN atom
# positions and velocities, as the paper states it.  The oracle must stop on
# exactly the same accepted step.  Plausible misreadings (no outward-motion
# condition, the atom-molecule distance instead of the largest pair distance,
# the wrong pair, the well instead of the barrier) are shown to stop on other
# steps, so each would fail.
# ---------------------------------------------------------------------------
def _T_REL(rtol):
    """Stop times of two valid RK45 implementations agree to about
    50 eps / rtol relative: the embedded error estimate is a cancellation
    whose rounding is ~eps / rtol of the norm, and the step sizes inherit
    it (the controller pin above shows the same)."""
    return 50 * 2.220446049250313e-16 / rtol


def _cartesian_view(oracle, s, y):
    m = np.array([s.m[0], s.m[1], s.m[2]])
    x = oracle.jacobi_to_cartesian(s, y)
    return x[:9].reshape(3, 3), x[9:].reshape(3, 3) / m[:, None], m


def _pair_distances(pos):
    return [float(np.linalg.norm(pos[i] - pos[k])) for i, k in ((0, 1), (1, 2), (2, 0))]


def _atom_leaving(pos, vel, m):
    """Atom C moves away from the centre of mass of A and B."""
    cm = (m[0] * pos[0] + m[1] * pos[1]) / (m[0] + m[1])
    vcm = (m[0] * vel[0] + m[1] * vel[1]) / (m[0] + m[1])
    return float(np.dot(pos[2] - cm, vel[2] - vcm)) > 0.0, float(np.linalg.norm(pos[2] - cm))


def _scipy_first_step(oracle, s, y0, rtol, atol, rule, t_end, max_steps=100_000):
    """First accepted scipy RK45 step (1-based index, time) whose end state
    satisfies rule(pos, vel, m); None if none before t_end."""
    from scipy.integrate import RK45
    solver = RK45(lambda t, x: oracle.rhs(s, x), 0.0, np.asarray(y0, float), t_bound=1e12,
                  rtol=rtol, atol=atol)
    n = 0
    while solver.t < t_end and n < max_steps:
        solver.step()
        assert solver.status == "running"
        n += 1
        pos, vel, m = _cartesian_view(oracle, s, solver.y)
        if rule(pos, vel, m):
            return n, solver.t
    return None


def _oracle_run_from(oracle, s, y0, integ, t_scale=1.0):
    y = np.asarray(y0, float)[None].copy()
    E0 = np.array([oracle.hamiltonian(s, y[0])])
    res = oracle.run_adaptive([s], np.zeros(1, np.int32), integ, y, np.array([t_scale]), E0,
                              np.zeros(1, np.int32))
    return res[0], y[0]


def test_stop_rule_against_scipy_and_cartesian_definition(oracle):
    """r_stop (Sec. 3.1): the trajectory ends after the first accepted step at
    which the largest distance between any two atoms exceeds r_stop while the
    atom leaves the molecule.  Lanes start at R0 = 40 > r_stop = 35 moving in
    (the outward condition keeps them running through the collision); the
    same states with all momenta reversed move out and stop after one step.
    The time scale t_scale of Sec. 3.1 (t_max = t_stop d / v_c) is the
    initial atom-molecule distance over the initial relative speed."""
    s = oracle.system_from_spec(W.SYS_H2_CA_MORSE)
    rtol, atol, r_stop = 1e-8, 1e-10, 35.0
    integ = oracle.make_integ(rtol=rtol, atol=atol, r_stop=r_stop, t_stop=100.0)
    E = np.array([0.10, 0.10, 0.10])
    b = np.array([0.0, 3.0, 6.0])
    v = np.array([0, 0, 1], np.int32)
    j = np.array([0, 3, 2], np.int32)
    st = oracle.init([s], np.zeros(3, np.int32), E, b, v, j, 40.0, 5)
    mu123 = oracle.reduced_masses(s)["mu123"]

    def rule_max(pos, vel, m):
        return max(_pair_distances(pos)) > r_stop and _atom_leaving(pos, vel, m)[0]

    def rule_no_outward(pos, vel, m):
        return max(_pair_distances(pos)) > r_stop

    def rule_R(pos, vel, m):
        out, R = _atom_leaving(pos, vel, m)
        return R > r_stop and out

    differs_R = 0
    for i in range(3):
        y0 = st["y"][i].copy()
        pos, vel, m = _cartesian_view(oracle, s, y0)
        leaving, R = _atom_leaving(pos, vel, m)
        assert not leaving and max(_pair_distances(pos)) > r_stop
        speed = float(np.linalg.norm(vel[2] - (m[0] * vel[0] + m[1] * vel[1]) / (m[0] + m[1])))
        assert speed == pytest.approx(math.sqrt(2 * E[i] / mu123), rel=1e-12)
        assert st["t_scale"][i] == pytest.approx(R / speed, rel=1e-12)
        r, _ = _oracle_run_from(oracle, s, y0, integ, st["t_scale"][i])
        t_end = 100.0 * st["t_scale"][i]
        ref = _scipy_first_step(oracle, s, y0, rtol, atol, rule_max, t_end)
        assert ref is not None
        print(f"\nlane {i}: oracle status {r['status']} after {r['nsteps']} accepted steps "
              f"(t = {r['t']:.6f}); scipy + Cartesian rule: step {ref[0]} (t = {ref[1]:.6f})")
        assert r["status"] == 2 and r["nsteps"] == ref[0]
        assert r["t"] == pytest.approx(ref[1], rel=_T_REL(rtol))
        # the misreadings stop elsewhere
        assert _scipy_first_step(oracle, s, y0, rtol, atol, rule_no_outward, t_end)[0] == 1
        alt = _scipy_first_step(oracle, s, y0, rtol, atol, rule_R, t_end)
        differs_R += alt[0] != ref[0]
        # reversed momenta: the atom leaves from the start, one step
        yr = y0.copy()
        yr[6:12] *= -1.0
        r, _ = _oracle_run_from(oracle, s, yr, integ, st["t_scale"][i])
        assert r["status"] == 2 and r["nsteps"] == 1
        assert _scipy_first_step(oracle, s, yr, rtol, atol, rule_max, t_end)[0] == 1
    assert differs_R >= 2


def _buck_barrier():
    """Inner barrier of the Buckingham Ca-H pair, V = A e^{-B r} - C6 / r^6
    (Sec. 3.2 item 3): the root of V'(r) below the well, by brentq."""
    from scipy.optimize import brentq
    A, B, C6 = W.CAH_BUCK[1:4]
    dV = lambda r: -A * B * math.exp(-B * r) + 6.0 * C6 / r ** 7
    return brentq(dV, 1.0, 3.5, xtol=1e-15)


def _collapse_states(oracle, s, side, speeds, gap=2.3, re=1.40):
    """Molecule AB on the x axis (rigid, both atoms at velocity u toward atom
    C, at rest): side "A" puts C at distance `gap` beyond A, side "B" beyond
    B.  Returns Jacobi states."""
    m = np.array([s.m[0], s.m[1], s.m[2]])
    out = []
    for u in speeds:
        if side == "A":
            xA, xB, xC, vv = [0, 0, 0], [-re, 0, 0], [gap, 0, 0], [u, 0, 0]
        else:
            xA, xB, xC, vv = [re, 0, 0], [0, 0, 0], [-gap, 0, 0], [-u, 0, 0]
        x = np.concatenate([xA, xB, xC, m[0] * np.array(vv), m[1] * np.array(vv),
                            np.zeros(3)]).astype(float)
        out.append(oracle.cartesian_to_jacobi(s, x))
    return out


def test_buckingham_collapse_rule_against_scipy(oracle):
    """A Buckingham pair that falls inside its short-range maximum r_b
    (Sec. 3.2 item 3, the 'max' where the potential turns over and
    collapses) ends the lane with FAIL_COLLAPSE after the first accepted step
    at which its distance is below r_b.  r_b comes from brentq on V' of the
    paper's formula; the step from scipy's RK45 with the distance test on
    Cartesian positions.  Fast approaches of atom C toward A (pair CA) and
    toward B (pair BC) collapse; a slower one turns around 0.09 bohr outside
    r_b and runs to r_stop; a pair started inside r_b collapses on the first
    step; the same approaches in a system whose BC pair is Morse collapse
    only on the CA side."""
    rb = _buck_barrier()
    rtol, atol = 1e-10, 1e-12
    integ = oracle.make_integ(rtol=rtol, atol=atol, r_stop=35.0, t_stop=3000.0)
    s = oracle.system_from_spec(W.SYS_H2_CA_BUCK)
    mu = oracle.reduced_masses(s)
    assert oracle.stationary(s.pair[2], mu["mu_CA"], 0.0)["r_inner"] == pytest.approx(rb, rel=1e-9)
    one_sided = dict(mass_u=W.MASS_H2_CA, pairs=(W.HH_MORSE, W.CAH_MORSE, W.CAH_BUCK))
    s1 = oracle.system_from_spec(one_sided)

    def collapse_in(kinds):
        def rule(pos, vel, m):
            d = _pair_distances(pos)
            return any(d[k] < rb for k in kinds)
        return rule

    def closest(sys_, y0, t_end):
        from scipy.integrate import RK45
        solver = RK45(lambda t, x: oracle.rhs(sys_, x), 0.0, y0, t_bound=1e12, rtol=rtol,
                      atol=atol)
        dmin = [math.inf] * 3
        while solver.t < t_end:
            solver.step()
            d = _pair_distances(_cartesian_view(oracle, sys_, solver.y)[0])
            dmin = [min(a, c) for a, c in zip(dmin, d)]
            if max(d) > 35.0:
                break
        return dmin

    cases = []   # (system, state, Buckingham pair indices, expect collapse)
    for side, pair in (("A", 2), ("B", 1)):
        for y0 in _collapse_states(oracle, s, side, [0.008, 0.02, 0.047]):
            cases.append((s, y0, (1, 2), True))
        cases.append((s, _collapse_states(oracle, s, side, [0.006])[0], (1, 2), False))
        cases.append((s, _collapse_states(oracle, s, side, [0.0], gap=2.0)[0], (1, 2), True))
    cases.append((s1, _collapse_states(oracle, s1, "A", [0.02])[0], (2,), True))
    cases.append((s1, _collapse_states(oracle, s1, "B", [0.02])[0], (2,), False))
    for sys_, y0, kinds, expect in cases:
        r, _ = _oracle_run_from(oracle, sys_, y0, integ)
        ref = _scipy_first_step(oracle, sys_, y0, rtol, atol, collapse_in(kinds), 3000.0)
        if expect:
            assert ref is not None
            assert r["status"] == 7 and r["cls"] == 5 and r["nsteps"] == ref[0], (r, ref)
            assert r["t"] == pytest.approx(ref[1], rel=_T_REL(rtol))
        else:
            assert ref is None
            assert r["status"] == 2, r
    # the turning point of the slow approach lies outside r_b but inside
    # the Buckingham well's minimum (a test against the well would fire)
    dmin = closest(s, _collapse_states(oracle, s, "A", [0.006])[0], 3000.0)
    r_well = oracle.stationary(s.pair[2], mu["mu_CA"], 0.0)["r_min"]
    print(f"\nr_b = {rb:.10f} bohr; slow approach turns at {dmin[2]:.4f} bohr; well at {r_well:.3f}")
    assert rb < dmin[2] < rb + 0.15 and dmin[2] < r_well
    # the Morse BC pair of the one-sided system passes inside r_b unharmed
    # while its Buckingham CA pair stays outside
    dmin = closest(s1, _collapse_states(oracle, s1, "B", [0.02])[0], 3000.0)
    assert dmin[1] < rb < dmin[2]
