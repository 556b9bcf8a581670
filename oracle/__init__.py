"""QCT oracle: Python access to the plain single-threaded FP64 C++ oracle.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference legs may import this package.  The
product library never imports, links or calls it, and this package imports
nothing from the product package: the two implementations share only the
seeded input generators, which hold none of the method's arithmetic.

Every function here marshals numpy arrays into ``qcams_oracle.cpp`` (Koots &
Perez-Rios, PyQCAMS, Secs. 2-4) and back; no arithmetic of the method is done
in Python.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qcams_oracle.cpp")
_SRC_IS = os.path.join(_HERE, "qcams_oracle_is.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

# lane status codes and outcome classes (same values as the library's ABI)
STATUS = dict(READY=0, RUNNING=1, DONE_RSTOP=2, DONE_TMAX=3, FAIL_MAXSTEPS=4,
              FAIL_HMIN=5, FAIL_NAN=6, FAIL_COLLAPSE=7, NO_LEVEL=8, INVALID=9)
CLS = dict(Q=0, R_AC=1, R_BC=2, D=3, AMBIG=4, FAIL=5)
H_COUNT, H_VT, H_JT, H_GB, H_W, H_W2, H_STRIDE = 0, 8, 200, 968, 1160, 1168, 1176


class OPair(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad", C.c_int32), ("p", C.c_double * 5)]


class OSystem(C.Structure):
    _fields_ = [("m", C.c_double * 3), ("pair", OPair * 3)]


class OInteg(C.Structure):
    _fields_ = [("rtol", C.c_double), ("atol", C.c_double), ("r_stop", C.c_double),
                ("t_stop", C.c_double), ("h_fixed", C.c_double), ("gb_sigma", C.c_double),
                ("max_steps", C.c_int64)]


class OLevel(C.Structure):
    _fields_ = [("ok", C.c_int32), ("pad", C.c_int32), ("E", C.c_double),
                ("r_minus", C.c_double), ("r_plus", C.c_double), ("tau", C.c_double),
                ("r_min", C.c_double), ("r_top", C.c_double), ("E_top", C.c_double)]


class OResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("cls", C.c_int32), ("vt", C.c_int32), ("jt", C.c_int32),
                ("vprime", C.c_double), ("jprime", C.c_double), ("gbw", C.c_double),
                ("dE", C.c_double), ("t", C.c_double), ("nsteps", C.c_int32),
                ("nrej", C.c_int32), ("Epair", C.c_double * 3), ("L2pair", C.c_double * 3),
                ("bound", C.c_int32 * 3), ("pad", C.c_int32)]


RESULT_DTYPE = np.dtype([("status", "<i4"), ("cls", "<i4"), ("vt", "<i4"), ("jt", "<i4"),
                         ("vprime", "<f8"), ("jprime", "<f8"), ("gbw", "<f8"), ("dE", "<f8"),
                         ("t", "<f8"), ("nsteps", "<i4"), ("nrej", "<i4"),
                         ("Epair", "<f8", 3), ("L2pair", "<f8", 3), ("bound", "<i4", 3),
                         ("pad", "<i4")])
assert RESULT_DTYPE.itemsize == C.sizeof(OResult)

_P = C.POINTER
_D = _P(C.c_double)
_I32 = _P(C.c_int32)
_I64 = _P(C.c_int64)
_U32 = _P(C.c_uint32)


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (no FMA contraction) into oracle/_build."""
    with _lock:
        os.makedirs(_BUILD, exist_ok=True)
        newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_IS))
        if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared",
               "-fPIC", _SRC, _SRC_IS, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        sig = {
            "oracle_abi_version": (C.c_int, []),
            "oracle_system_setup": (C.c_int, [_D, _I32, _D, _P(OSystem)]),
            "oracle_pair_potential": (None, [_P(OPair), C.c_double, _D, _D]),
            "oracle_philox4x32_10": (None, [_U32, _U32, _U32]),
            "oracle_level": (None, [_P(OPair), C.c_double, C.c_int, C.c_int, _P(OLevel)]),
            "oracle_v_of_E": (C.c_double, [_P(OPair), C.c_double, C.c_double, C.c_double]),
            "oracle_stationary": (None, [_P(OPair), C.c_double, C.c_double, _D]),
            "oracle_hamiltonian": (C.c_double, [_P(OSystem), _D]),
            "oracle_rhs": (None, [_P(OSystem), _D, _D]),
            "oracle_rhs_cartesian": (None, [_P(OSystem), _D, _D]),
            "oracle_jacobi_to_cartesian": (None, [_P(OSystem), _D, _D]),
            "oracle_cartesian_to_jacobi": (None, [_P(OSystem), _D, _D]),
            "oracle_dopri5_tableau": (None, [_D, _D, _D, _D]),
            "oracle_dopri5_linear": (None, [C.c_double, C.c_double, C.c_double, _D, _D]),
            "oracle_run_fixed": (None, [_P(OSystem), _D, C.c_int64, C.c_double, C.c_int64]),
            "oracle_run_fixed_cartesian": (None, [_P(OSystem), _D, C.c_double, C.c_int64]),
            "oracle_init": (None, [_P(OSystem), _I32, _P(OLevel), _I32, _D, _D, _I32, C.c_int64,
                                   C.c_double, C.c_uint64, C.c_uint64, _D, _D, _D, _D, _I32, _D]),
            "oracle_run_adaptive": (None, [_P(OSystem), _I32, _P(OInteg), _D, _D, _D, _I32,
                                           C.c_int64, C.c_void_p]),
            "oracle_analyze": (None, [_P(OSystem), _I32, _P(OInteg), _D, _D, _I32, C.c_int64,
                                      C.c_void_p]),
            "oracle_reduce": (None, [C.c_int64, _I32, _I32, _I32, _D, _D, _I32, C.c_int32, _I64]),
            "oracle_xsec": (None, [_I64, C.c_int32, _D, _D, _I32, C.c_int32, C.c_int32, _D]),
            "oracle_rates": (None, [_D, _D, C.c_int32, C.c_double, _D]),
            "oracle_gb_distribution": (C.c_double, [_I64, _I32, C.c_int32, _D]),
            "oracle_mlp_num_params": (C.c_int, []),
            "oracle_mlp_forward": (None, [_D, _D, C.c_int64, _D]),
            "oracle_mlp_loss_grad": (C.c_double, [_D, _D, _I32, C.c_int64, _D]),
            "oracle_adam_step": (None, [_D, _D, _D, _D, C.c_int64, C.c_int64, C.c_double,
                                        C.c_double, C.c_double, C.c_double]),
            "oracle_proposal": (None, [_D, _D, C.c_int64, C.c_double, C.c_double, _D]),
            "oracle_proposal_cdf": (None, [_D, C.c_int64, _I64, _I64]),
            "oracle_sample_proposal": (None, [_I32, C.c_double, _I64, _I64, C.c_int64, C.c_int64,
                                              C.c_uint64, C.c_uint64, _D, _D, _D, _I32]),
            "oracle_is_mean": (None, [_D, _D, C.c_int64, _D, _D]),
            "oracle_proposal_grid": (None, [_I32, C.c_double, C.c_double, C.c_int32, C.c_int32,
                                            _D, _D, _D]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------
def _d(a):
    return a.ctypes.data_as(_D)


def _i32(a):
    return a.ctypes.data_as(_I32)


def _arr(x, dtype):
    return np.ascontiguousarray(np.asarray(x, dtype=dtype))


def make_pair(kind: int, params) -> OPair:
    q = OPair()
    q.kind = int(kind)
    for i, v in enumerate(params):
        q.p[i] = float(v)
    return q


def make_system(sys_desc) -> OSystem:
    """sys_desc: dict(mass=(mA, mB, mC) [electron masses], pairs=[(kind, params)]*3)."""
    s = OSystem()
    for i in range(3):
        s.m[i] = float(sys_desc["mass"][i])
    for k in range(3):
        kind, params = sys_desc["pairs"][k]
        s.pair[k] = make_pair(kind, params)
    return s


SPEC_KIND = dict(morse=0, lj=1, buck=2, lj_fit=3, morse_we=4)


def system_from_spec(spec) -> OSystem:
    """spec: dict(mass_u=(mA, mB, mC), pairs=[(kind_name, *params)] * 3)."""
    mass = _arr(spec["mass_u"], np.float64)
    kinds = np.zeros(3, np.int32)
    par = np.zeros((3, 5))
    for k, pr in enumerate(spec["pairs"]):
        kinds[k] = SPEC_KIND[pr[0]]
        par[k, :len(pr) - 1] = pr[1:]
    out = OSystem()
    rc = lib().oracle_system_setup(_d(mass), _i32(kinds), _d(np.ascontiguousarray(par)),
                                   C.byref(out))
    if rc != 0:
        raise ValueError(f"invalid system spec {spec}")
    return out


def reduced_masses(sys: OSystem):
    mA, mB, mC = sys.m[0], sys.m[1], sys.m[2]
    return dict(mu12=mA * mB / (mA + mB), mu123=mC * (mA + mB) / (mA + mB + mC),
                mu_AB=mA * mB / (mA + mB), mu_BC=mB * mC / (mB + mC), mu_CA=mC * mA / (mC + mA))


def make_integ(rtol=1e-10, atol=1e-12, r_stop=35.0, t_stop=15.0, h_fixed=0.0,
               gb_sigma=0.1 / (2.0 * np.sqrt(2.0 * np.log(2.0))), max_steps=1_000_000) -> OInteg:
    return OInteg(rtol, atol, r_stop, t_stop, h_fixed, gb_sigma, int(max_steps))


def pair_potential(pair: OPair, r: float):
    V, dV = C.c_double(), C.c_double()
    lib().oracle_pair_potential(C.byref(pair), float(r), C.byref(V), C.byref(dV))
    return V.value, dV.value


def philox4x32_10(ctr, key):
    c = _arr(ctr, np.uint32)
    k = _arr(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().oracle_philox4x32_10(c.ctypes.data_as(_U32), k.ctypes.data_as(_U32),
                               out.ctypes.data_as(_U32))
    return out


def level(pair: OPair, mu: float, v: int, j: int) -> OLevel:
    out = OLevel()
    lib().oracle_level(C.byref(pair), float(mu), int(v), int(j), C.byref(out))
    return out


def v_of_E(pair: OPair, mu: float, L2: float, E: float) -> float:
    return lib().oracle_v_of_E(C.byref(pair), float(mu), float(L2), float(E))


def stationary(pair: OPair, mu: float, L2: float):
    out = np.zeros(6)
    lib().oracle_stationary(C.byref(pair), float(mu), float(L2), _d(out))
    return dict(has_well=bool(out[0]), r_min=out[1], has_top=bool(out[2]), r_top=out[3],
                r_inner=out[4], threshold=out[5])


def hamiltonian(sys: OSystem, y) -> float:
    y = _arr(y, np.float64)
    return lib().oracle_hamiltonian(C.byref(sys), _d(y))


def rhs(sys: OSystem, y):
    y = _arr(y, np.float64)
    dy = np.zeros(12)
    lib().oracle_rhs(C.byref(sys), _d(y), _d(dy))
    return dy


def rhs_cartesian(sys: OSystem, x):
    x = _arr(x, np.float64)
    dx = np.zeros(18)
    lib().oracle_rhs_cartesian(C.byref(sys), _d(x), _d(dx))
    return dx


def jacobi_to_cartesian(sys: OSystem, y):
    y = _arr(y, np.float64)
    x = np.zeros(18)
    lib().oracle_jacobi_to_cartesian(C.byref(sys), _d(y), _d(x))
    return x


def cartesian_to_jacobi(sys: OSystem, x):
    x = _arr(x, np.float64)
    y = np.zeros(12)
    lib().oracle_cartesian_to_jacobi(C.byref(sys), _d(x), _d(y))
    return y


def dopri5_tableau():
    c, a, b, bs = np.zeros(7), np.zeros(49), np.zeros(7), np.zeros(7)
    lib().oracle_dopri5_tableau(_d(c), _d(a), _d(b), _d(bs))
    return c, a.reshape(7, 7), b, bs


def dopri5_linear(lam: float, h: float, y0: float = 1.0):
    y1, err = C.c_double(), C.c_double()
    lib().oracle_dopri5_linear(float(lam), float(h), float(y0), C.byref(y1), C.byref(err))
    return y1.value, err.value


def run_fixed(sys: OSystem, y, h: float, nsteps: int):
    y = np.array(y, dtype=np.float64, order="C").reshape(-1, 12)
    lib().oracle_run_fixed(C.byref(sys), _d(y), y.shape[0], float(h), int(nsteps))
    return y


def run_fixed_cartesian(sys: OSystem, x, h: float, nsteps: int):
    x = np.array(x, dtype=np.float64, order="C").reshape(18)
    lib().oracle_run_fixed_cartesian(C.byref(sys), _d(x), float(h), int(nsteps))
    return x


def _sys_array(systems):
    arr = (OSystem * len(systems))()
    for i, s in enumerate(systems):
        arr[i] = s
    return arr


def levels_for(systems, sys_id, v, j):
    """Unique Bohr-Sommerfeld levels for the lanes: returns (levels, lvl_index)."""
    sys_id = np.asarray(sys_id, np.int32)
    v = np.asarray(v, np.int32)
    j = np.asarray(j, np.int32)
    keys = np.stack([sys_id, v, j], axis=1)
    uniq, inv = np.unique(keys, axis=0, return_inverse=True)
    levs = (OLevel * len(uniq))()
    for i, (s, vv, jj) in enumerate(uniq):
        sysd = systems[int(s)]
        mA, mB = sysd.m[0], sysd.m[1]
        mu = mA * mB / (mA + mB)
        levs[i] = level(sysd.pair[0], mu, int(vv), int(jj))
    return levs, np.ascontiguousarray(inv.reshape(-1).astype(np.int32))


def init(systems, sys_id, Ecol, b, v, j, R0, seed, id_offset=0, u_in=None):
    """Initial conditions (Sec. 2.1).  Returns dict(y, t_scale, E0, status, u)."""
    n = len(Ecol)
    levs, lvl = levels_for(systems, sys_id, v, j)
    sys_arr = _sys_array(systems)
    sid = _arr(sys_id, np.int32)
    E = _arr(Ecol, np.float64)
    bb = _arr(b, np.float64)
    jj = _arr(j, np.int32)
    y = np.zeros((n, 12))
    ts = np.zeros(n)
    E0 = np.zeros(n)
    st = np.zeros(n, np.int32)
    u = np.zeros((n, 4))
    uin = None if u_in is None else _arr(u_in, np.float64).reshape(n, 4)
    lib().oracle_init(sys_arr, _i32(sid), levs, _i32(lvl), _d(E), _d(bb), _i32(jj), n,
                      float(R0), int(seed), int(id_offset),
                      None if uin is None else _d(uin), _d(y), _d(ts), _d(E0), _i32(st), _d(u))
    return dict(y=y, t_scale=ts, E0=E0, status=st, u=u)


def run_adaptive(systems, sys_id, integ: OInteg, y, t_scale, E0, status):
    """Adaptive DOPRI5 + stop rules + product analysis; y is updated in place."""
    n = y.shape[0]
    out = np.zeros(n, RESULT_DTYPE)
    sid = _arr(sys_id, np.int32)
    ts = _arr(t_scale, np.float64)
    e0 = _arr(E0, np.float64)
    st = _arr(status, np.int32)
    assert y.flags.c_contiguous and y.dtype == np.float64
    lib().oracle_run_adaptive(_sys_array(systems), _i32(sid), C.byref(integ), _d(y), _d(ts),
                              _d(e0), _i32(st), n, out.ctypes.data)
    return out


def analyze(systems, sys_id, integ: OInteg, y, E0, status):
    y = np.ascontiguousarray(y, np.float64)
    n = y.shape[0]
    out = np.zeros(n, RESULT_DTYPE)
    lib().oracle_analyze(_sys_array(systems), _i32(_arr(sys_id, np.int32)), C.byref(integ),
                         _d(y), _d(_arr(E0, np.float64)), _i32(_arr(status, np.int32)), n,
                         out.ctypes.data)
    return out


def reduce(cls, vt, jt, gbw, cell, n_cells, isw=None):
    n = len(cls)
    hist = np.zeros(n_cells * H_STRIDE, np.int64)
    w = None if isw is None else _arr(isw, np.float64)
    lib().oracle_reduce(n, _i32(_arr(cls, np.int32)), _i32(_arr(vt, np.int32)),
                        _i32(_arr(jt, np.int32)), _d(_arr(gbw, np.float64)),
                        None if w is None else _d(w), _i32(_arr(cell, np.int32)), int(n_cells),
                        hist.ctypes.data_as(_I64))
    return hist.reshape(n_cells, H_STRIDE)


def xsec(hist, cell_b, cell_w, group, n_groups, weighted=False):
    hist = np.ascontiguousarray(hist, np.int64)
    n_cells = hist.shape[0]
    out = np.zeros(14 * n_cells + 14 * n_groups)
    lib().oracle_xsec(hist.ctypes.data_as(_I64), n_cells, _d(_arr(cell_b, np.float64)),
                      _d(_arr(cell_w, np.float64)), _i32(_arr(group, np.int32)), int(n_groups),
                      int(bool(weighted)), _d(out))
    cells = out[:14 * n_cells].reshape(n_cells, 7, 2)
    groups = out[14 * n_cells:].reshape(n_groups, 7, 2)
    return cells, groups


def run_lanes(systems, sys_id, Ecol, b, v, j, R0, seed, integ: OInteg, id_offset=0, u_in=None):
    """init + adaptive integration + analysis for a batch of lanes."""
    st = init(systems, sys_id, Ecol, b, v, j, R0, seed, id_offset, u_in)
    res = run_adaptive(systems, sys_id, integ, st["y"], st["t_scale"], st["E0"], st["status"])
    return st, res


# ---------------------------------------------------------------------------
# learned proposal (qcams_oracle_is.cpp)
# ---------------------------------------------------------------------------
MLP_NPARAMS = 9156


def mlp_forward(params, x):
    params = _arr(params, np.float64)
    x = _arr(x, np.float64).reshape(-1, 8)
    out = np.zeros((x.shape[0], 4))
    lib().oracle_mlp_forward(_d(params), _d(x), x.shape[0], _d(out))
    return out


def mlp_loss_grad(params, x, labels):
    params = _arr(params, np.float64)
    x = _arr(x, np.float64).reshape(-1, 8)
    lab = _arr(labels, np.int32)
    g = np.zeros(MLP_NPARAMS)
    loss = lib().oracle_mlp_loss_grad(_d(params), _d(x), _i32(lab), x.shape[0], _d(g))
    return loss, g


def adam_step(params, m, v, grad, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    params, m, v = (np.array(a, np.float64) for a in (params, m, v))
    g = _arr(grad, np.float64)
    lib().oracle_adam_step(_d(params), _d(m), _d(v), _d(g), params.size, int(t), float(lr),
                           float(beta1), float(beta2), float(eps))
    return params, m, v


def proposal(params, x_cells, eps, alpha):
    params = _arr(params, np.float64)
    x = _arr(x_cells, np.float64).reshape(-1, 8)
    q = np.zeros(x.shape[0])
    lib().oracle_proposal(_d(params), _d(x), x.shape[0], float(eps), float(alpha), _d(q))
    return q


def proposal_cdf(q):
    q = _arr(q, np.float64)
    qfix = np.zeros(q.size, np.int64)
    cdf = np.zeros(q.size, np.int64)
    lib().oracle_proposal_cdf(_d(q), q.size, qfix.ctypes.data_as(_I64), cdf.ctypes.data_as(_I64))
    return qfix, cdf


def sample_proposal(dims, b2_max, qfix, cdf, n, seed, id_offset=0):
    dims = _arr(dims, np.int32)
    qfix = _arr(qfix, np.int64)
    cdf = _arr(cdf, np.int64)
    b, u, w = np.zeros(n), np.zeros((n, 4)), np.zeros(n)
    cell = np.zeros(n, np.int32)
    lib().oracle_sample_proposal(_i32(dims), float(b2_max), qfix.ctypes.data_as(_I64),
                                 cdf.ctypes.data_as(_I64), qfix.size, int(n), int(seed),
                                 int(id_offset), _d(b), _d(u), _d(w), _i32(cell))
    return b, u, w, cell


def is_mean(w, f):
    w = _arr(w, np.float64)
    f = _arr(f, np.float64)
    mean, se = C.c_double(), C.c_double()
    lib().oracle_is_mean(_d(w), _d(f), w.size, C.byref(mean), C.byref(se))
    return mean.value, se.value


def proposal_grid(dims, b2_max, E, v, j, mean, std):
    dims = _arr(dims, np.int32)
    n = int(np.prod(dims))
    x = np.zeros((n, 8))
    lib().oracle_proposal_grid(_i32(dims), float(b2_max), float(E), int(v), int(j),
                               _d(_arr(mean, np.float64)), _d(_arr(std, np.float64)), _d(x))
    return x


def rates(sigma, E, mu123):
    sigma, E = _arr(sigma, np.float64), _arr(E, np.float64)
    k = np.zeros(sigma.size)
    lib().oracle_rates(_d(sigma), _d(E), sigma.size, float(mu123), _d(k))
    return k


def gb_distribution(hist, cells):
    hist = np.ascontiguousarray(hist, np.int64)
    cells = _arr(cells, np.int32)
    out = np.zeros(3 * 64)
    W = lib().oracle_gb_distribution(hist.ctypes.data_as(_I64), _i32(cells), cells.size, _d(out))
    return out.reshape(3, 64), W
