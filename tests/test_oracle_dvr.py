"""The paper's DVR (Colbert-Miller particle-in-a-box basis) in the oracle:
pinned to the exact Morse spectrum for j = 0, and used to cross-check the
Bohr-Sommerfeld levels for j > 0 (quantum vs semiclassical levels differ only
by small higher-order terms)."""
import math

import numpy as np

from paper_2304_02731_gb300 import workloads as W


def test_dvr_reproduces_exact_morse_spectrum(oracle):
    from oracle import dvr
    s = oracle.system_from_spec(W.SYS_H2_CA_MORSE)
    mu = oracle.reduced_masses(s)["mu12"]
    De, a = 0.1745, 1.03
    w = a * math.sqrt(2 * De / mu)
    E = dvr.dvr_levels(s.pair[0], mu, 0, 0.3, 16.0, 800)
    for v in range(13):
        exact = -De + w * (v + 0.5) - w * w * (v + 0.5) ** 2 / (4 * De)
        assert abs(E[v] - exact) < 1e-9, (v, E[v], exact)


def test_dvr_converges_with_grid(oracle):
    from oracle import dvr
    s = oracle.system_from_spec(W.SYS_H2_CA_MORSE)
    mu = oracle.reduced_masses(s)["mu12"]
    E1 = dvr.dvr_levels(s.pair[0], mu, 7, 0.3, 14.0, 500)[:8]
    E2 = dvr.dvr_levels(s.pair[0], mu, 7, 0.3, 14.0, 900)[:8]
    assert np.max(np.abs(E1 - E2)) < 1e-10


def test_bohr_sommerfeld_levels_agree_with_dvr(oracle):
    """The semiclassical (Bohr-Sommerfeld) levels lie within 0.5 % of the
    local vibrational spacing of the quantum (DVR) ones, for j > 0 and for
    the generalized LJ pair, where the quantisation rule is not exact."""
    from oracle import dvr
    for spec, pair, a_, b_ in [(W.SYS_H2_CA_MORSE, 0, 0.3, 14.0),
                               (W.SYS_H2_CA_LJ12, 2, 2.0, 30.0)]:
        s = oracle.system_from_spec(spec)
        m = oracle.reduced_masses(s)
        mu = m["mu12"] if pair == 0 else m["mu_CA"]
        for j in (1, 5, 12, 20):
            E = dvr.dvr_levels(s.pair[pair], mu, j, a_, b_, 900)
            for v in (0, 2, 5):
                L = oracle.level(s.pair[pair], mu, v, j)
                if not L.ok:
                    continue
                spacing = E[v + 1] - E[v]
                assert abs(E[v] - L.E) < 5e-3 * spacing, (pair, v, j, E[v], L.E, spacing)
