"""C-ABI checks that need no GPU: the library builds for sm_103a, loads,
exports every function include/qcams.h declares, rejects bad arguments
before touching a device, and its host-side system set-up agrees with the
oracle's."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def Q():
    from paper_2304_02731_gb300 import build
    build.build()
    from paper_2304_02731_gb300 import qcams
    qcams.lib()
    return qcams


def _declared_functions():
    """Functions declared in every header of include/ (the path's qcams.h
    and the test-support qcams_debug.h)."""
    inc = os.path.join(ROOT, "include")
    names = set()
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            src = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, f)).read(), flags=re.S)
            names |= set(re.findall(r"\b(qcams_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(Q):
    names = _declared_functions()
    assert "qcams_init_states" in names and "qcams_run_batch" in names
    assert "qcams_reduce_xsec" in names and "qcams_debug_context_exists" in names
    L = C.CDLL(Q.library_path())
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(Q.EXPORTS)


def test_status_strings(Q):
    for code in [0, -1, -2, -3, -4, -5, -6, 17]:
        assert len(Q.lib().qcams_status_string(code)) > 0


def test_system_setup_matches_oracle(Q, oracle):
    from paper_2304_02731_gb300 import workloads as W
    for spec in [W.SYS_H2_CA_MORSE, W.SYS_H2_CA_BUCK, W.SYS_H2_CA_LJ12, W.SYS_H2_CA_LJ8]:
        a = Q.system_setup(spec)
        b = oracle.system_from_spec(spec)
        for i in range(3):
            assert a.mass[i] == pytest.approx(b.m[i], rel=1e-15)
        for k in range(3):
            assert a.pair[k].kind == b.pair[k].kind
            for i in range(5):
                assert a.pair[k].p[i] == pytest.approx(b.pair[k].p[i], rel=1e-14, abs=0)
    spec = dict(mass_u=(1.0, 1.0, 40.0),
                pairs=(("morse_we", 0.1645, 1.401, 0.02005), W.CAH_MORSE, W.CAH_MORSE))
    a, b = Q.system_setup(spec), oracle.system_from_spec(spec)
    assert a.pair[0].p[2] == pytest.approx(b.pair[0].p[2], rel=1e-15)


@pytest.mark.parametrize("bad", [
    dict(mass_u=(0.0, 1.0, 40.0), pairs=(("morse", 0.17, 1.4, 1.0),) * 3),
    dict(mass_u=(1.0, 1.0, 40.0), pairs=(("morse", -0.17, 1.4, 1.0),) * 3),
    dict(mass_u=(1.0, 1.0, 40.0), pairs=(("lj_fit", 6, 12, 0.06, 3.8),) * 3),
    dict(mass_u=(1.0, 1.0, 40.0), pairs=(("lj", 12.5, 6, 1.0, 1.0, 3.0),) * 3),
    dict(mass_u=(1.0, 1.0, 40.0), pairs=(("lj", 12, 2, 1.0, 1.0, 3.0),) * 3),
    dict(mass_u=(1.0, float("nan"), 40.0), pairs=(("morse", 0.17, 1.4, 1.0),) * 3),
    # alpha re >= 700: e^{alpha (re - r)} would overflow near r = 0
    dict(mass_u=(1.0, 1.0, 40.0), pairs=(("morse", 0.17, 1.4, 600.0),) * 3),
])
def test_system_setup_rejects_bad_parameters(Q, bad):
    with pytest.raises(Q.QcamsError) as e:
        Q.system_setup(bad)
    assert e.value.code == -1


def test_entry_points_reject_bad_arguments_without_a_device(Q):
    L = Q.lib()
    from paper_2304_02731_gb300 import workloads as W
    sysarr = Q.systems_array([W.SYS_H2_CA_MORSE])
    integ = Q.make_integ()
    b = Q.CBatch()
    b.n = 10                      # all pointers NULL
    assert L.qcams_run_batch(sysarr, 1, C.byref(integ), C.byref(b), None) == -1
    assert L.qcams_run_batch(sysarr, 0, C.byref(integ), C.byref(b), None) == -1
    # more systems than QCAMS_MAX_SYS: a size limit, rejected before any read
    assert L.qcams_run_batch(sysarr, 5, C.byref(integ), C.byref(b), None) == -4
    assert L.qcams_init_states(sysarr, 5, None, None, None, None, 30.0, 0, 0, None,
                               C.byref(b), None) == -4
    assert L.qcams_run_batch(sysarr, 1, None, C.byref(b), None) == -1
    bad = Q.make_integ(rtol=-1.0)
    assert L.qcams_run_batch(sysarr, 1, C.byref(bad), C.byref(b), None) == -1
    bad = Q.make_integ(max_steps=0)
    assert L.qcams_run_batch(sysarr, 1, C.byref(bad), C.byref(b), None) == -1
    bad = Q.make_integ(precision=16)
    assert L.qcams_run_batch(sysarr, 1, C.byref(bad), C.byref(b), None) == -1
    # launch modes 0-3 only; three or six lanes per trajectory are FP64 only
    bad = Q.make_integ(persistent=4)
    assert L.qcams_run_batch(sysarr, 1, C.byref(bad), C.byref(b), None) == -1
    bad = Q.make_integ(persistent=Q.LAUNCH_TRI, precision=32)
    assert L.qcams_run_batch(sysarr, 1, C.byref(bad), C.byref(b), None) == -1
    bad = Q.make_integ(persistent=Q.LAUNCH_TRI, fixed_step=True, h_fixed=0.1)
    assert L.qcams_run_batch(sysarr, 1, C.byref(bad), C.byref(b), None) == -1
    bad = Q.make_integ(persistent=Q.LAUNCH_HEX, precision=32)
    assert L.qcams_run_batch(sysarr, 1, C.byref(bad), C.byref(b), None) == -1
    assert L.qcams_init_states(sysarr, 1, None, None, None, None, 30.0, 0, 0, None,
                               C.byref(b), None) == -1
    b.n = -1
    assert L.qcams_analyze(sysarr, 1, C.byref(integ), C.byref(b), None) == -1
    cells = Q.Cells()
    cells.n_cells = 0
    assert L.qcams_reduce_xsec(C.byref(b), C.byref(cells), None, None, None) == -1
    cells.n_cells = 1 << 20
    b.n = 0
    assert L.qcams_reduce_xsec(C.byref(b), C.byref(cells), C.c_void_p(8), None, None) == -4
    assert L.qcams_last_run_stats(None, None) == -1
    f = C.c_double()
    assert L.qcams_fma_peak(16, C.byref(f), None) == -1
    # diagnostics: sizes and the Morse argument range are checked first
    p8 = C.c_void_p(8)
    assert L.qcams_debug_force_math(None, 1.0, 1.4, None, None, None, -1, None) == -1
    assert L.qcams_debug_force_math(p8, 1.0, 700.0, p8, p8, p8, 1, None) == -1
    assert L.qcams_debug_force_math(p8, -1.0, 1.4, p8, p8, p8, 1, None) == -1
    assert L.qcams_debug_ff_dot(p8, p8, 0, p8, p8, 1, None) == -1
    assert L.qcams_debug_ff_dot(p8, p8, 9, p8, p8, 1, None) == -1
    assert L.qcams_debug_ff_dot(None, p8, 3, p8, p8, 1, None) == -1


def test_rate_constants_match_oracle(Q, oracle):
    from paper_2304_02731_gb300 import workloads as W
    s = oracle.system_from_spec(W.SYS_H2_CA_MORSE)
    mu = oracle.reduced_masses(s)["mu123"]
    E = W.sweep_energies()
    sig = np.linspace(1.0, 30.0, E.size)
    k, kse = Q.rate_constants(sig, 0.1 * sig, E, mu)
    ko = oracle.rates(sig, E, mu)
    assert np.allclose(k, ko, rtol=1e-15) and np.allclose(kse, 0.1 * ko, rtol=1e-14)


def test_gb_distribution_matches_oracle(Q, oracle):
    rng = np.random.default_rng(6)
    n = 5000
    cls = rng.integers(0, 6, n)
    vt = rng.integers(0, 70, n)
    gbw = rng.uniform(0.0, 9.0, n)
    cell = rng.integers(0, 5, n)
    H = oracle.reduce(cls, vt, np.zeros(n, np.int32), gbw, cell, 5)
    P, Wt = Q.gb_distribution(H, [1, 3, 4])
    Po, Wo = oracle.gb_distribution(H, [1, 3, 4])
    assert Wt == pytest.approx(Wo, rel=1e-15)
    assert np.allclose(P, Po, rtol=1e-14, atol=0)
    with pytest.raises(Q.QcamsError):
        Q.gb_distribution(H, [])


def test_proposal_spec_limits_without_a_device(Q):
    """Proposal specs are validated before any device work: bad fields give
    QCAMS_E_INVALID, more than 2^22 cells QCAMS_E_CAPACITY (the pointers
    below are never dereferenced)."""
    L = Q.lib()
    fake = C.c_void_p(256)
    m = Q.CMLP()
    m.params = m.adam_m = m.adam_v = m.grad = m.params_bf16 = 256
    big = Q.proposal_spec(0.1, 0, 0, dims=(64, 64, 32, 32, 2))      # 2^23 cells
    assert L.qcams_build_proposal(C.byref(m), C.byref(big), fake, fake, fake, None) == -4
    u4 = (C.c_void_p * 4)(256, 256, 256, 256)
    assert L.qcams_sample_proposal(C.byref(big), fake, fake, 10, 0, 0, fake, u4, fake, fake,
                                   None) == -4
    bad = Q.proposal_spec(0.1, 0, 0, alpha=0.0)
    assert L.qcams_build_proposal(C.byref(m), C.byref(bad), fake, fake, fake, None) == -1
    bad = Q.proposal_spec(0.1, 0, 0, dims=(0, 8, 8, 8, 4))
    assert L.qcams_sample_proposal(C.byref(bad), fake, fake, 10, 0, 0, fake, u4, fake, fake,
                                   None) == -1
    assert L.qcams_mlp_train(C.byref(m), fake, fake, 10, 1, 0, 1e-3, 0, fake, None, None) == -1


def test_xsec_from_host_histograms_matches_oracle(Q, oracle):
    """qcams_xsec_from_hist (host, no device): the cross sections of random
    histogram records equal the oracle's (Sec. 2.3, Eqs. 13-16; Sec. 4) to
    rounding, plain and importance-weighted; a bad argument is rejected."""
    rng = np.random.default_rng(12)
    nc, ng = 40, 5
    n = 20000
    cls = rng.choice(6, n, p=[0.55, 0.1, 0.1, 0.15, 0.05, 0.05])
    cell = rng.integers(0, nc, n)
    vt, jt = rng.integers(0, 70, n), rng.integers(0, 300, n)
    gbw, isw = rng.uniform(0, 9, n), rng.uniform(0.2, 5.0, n)
    H = oracle.reduce(cls, vt, jt, gbw, cell, nc, isw)
    b, w = rng.uniform(0, 10, nc), rng.uniform(0.1, 1.0, nc)
    group = rng.integers(-1, ng, nc).astype(np.int32)
    for weighted in (False, True):
        cells, groups = Q.xsec_from_hist(H, b, w, group, ng, weighted)
        oc, og = oracle.xsec(H, b, w, group, ng, weighted)
        assert np.allclose(cells, oc, rtol=1e-14, atol=0)
        assert np.allclose(groups, og, rtol=1e-13, atol=1e-300)
    with pytest.raises(Q.QcamsError):
        Q.xsec_from_hist(H, b, w, group, 65537)
