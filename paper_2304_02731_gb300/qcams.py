"""Python binding of the QCT C ABI (include/qcams.h).

Argument marshalling only: every step of the trajectory path runs in the
CUDA kernels of libqcams.so.  PyTorch provides device memory and streams.
The binding fails loudly if the library cannot be loaded; there is no CPU
fallback.

Function names follow the C ABI: ``init_states``, ``run_batch``,
``analyze``, ``reduce_xsec``, ``levels``; ``Batch`` owns the structure-of-
arrays device tensors of one batch of trajectories.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading
from dataclasses import dataclass

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "_build", "libqcams.so")
_lock = threading.Lock()
_lib = None

# status / class codes and histogram layout (include/qcams.h)
LANE = dict(READY=0, RUNNING=1, DONE_RSTOP=2, DONE_TMAX=3, FAIL_MAXSTEPS=4, FAIL_HMIN=5,
            FAIL_NAN=6, FAIL_COLLAPSE=7, NO_LEVEL=8, INVALID=9)
CLS = dict(Q=0, R_AC=1, R_BC=2, D=3, AMBIG=4, FAIL=5)
H_COUNT, H_VT, H_JT, H_GB, H_W, H_W2, H_STRIDE = 0, 8, 200, 968, 1160, 1168, 1176
SPEC_KIND = dict(morse=0, lj=1, buck=2, lj_fit=3, morse_we=4)
GB_SIGMA_DEFAULT = 0.1 / (2.0 * math.sqrt(2.0 * math.log(2.0)))

EXPORTS = ["qcams_status_string", "qcams_system_setup", "qcams_levels", "qcams_init_states",
           "qcams_run_batch", "qcams_analyze", "qcams_reduce_xsec", "qcams_last_run_stats",
           "qcams_fma_peak", "qcams_device_info", "qcams_shutdown", "qcams_run_batch_noalloc",
           "qcams_debug_exp", "qcams_debug_force_math", "qcams_debug_ff_dot",
           "qcams_debug_context_exists", "qcams_xsec_from_hist", "qcams_autotune", "qcams_mlp_init", "qcams_mlp_sync",
           "qcams_mlp_features", "qcams_mlp_fit_standardizer", "qcams_mlp_grad",
           "qcams_mlp_train_step", "qcams_mlp_train", "qcams_mlp_infer", "qcams_build_proposal",
           "qcams_sample_proposal", "qcams_rate_constants", "qcams_gb_distribution"]
MLP_NPARAMS = 9156


class QcamsError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib().qcams_status_string(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: {msg} (status {code})")
        self.code = code


class Pair(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad", C.c_int32), ("p", C.c_double * 5)]


class System(C.Structure):
    _fields_ = [("mass", C.c_double * 3), ("pair", Pair * 3)]


class Integ(C.Structure):
    _fields_ = [("rtol", C.c_double), ("atol", C.c_double), ("r_stop", C.c_double),
                ("t_stop", C.c_double), ("h_fixed", C.c_double), ("gb_sigma", C.c_double),
                ("max_steps", C.c_int64), ("fixed_step", C.c_int32), ("precision", C.c_int32),
                ("persistent", C.c_int32), ("block", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("pad", C.c_int32)]


class Level(C.Structure):
    _fields_ = [("E", C.c_double), ("r_minus", C.c_double), ("r_plus", C.c_double),
                ("tau", C.c_double), ("ok", C.c_int32), ("pad", C.c_int32)]


class CBatch(C.Structure):
    _fields_ = [("n", C.c_int64), ("sys_id", C.c_void_p), ("cell", C.c_void_p),
                ("isw", C.c_void_p), ("y", C.c_void_p * 12), ("t", C.c_void_p),
                ("h", C.c_void_p), ("t_scale", C.c_void_p), ("E0", C.c_void_p),
                ("Ecol", C.c_void_p), ("u", C.c_void_p * 4), ("status", C.c_void_p),
                ("cls", C.c_void_p), ("nsteps", C.c_void_p), ("nrej", C.c_void_p),
                ("dE", C.c_void_p), ("vprime", C.c_void_p), ("jprime", C.c_void_p),
                ("gbw", C.c_void_p), ("vt", C.c_void_p), ("jt", C.c_void_p)]


class RunStats(C.Structure):
    _fields_ = [("rhs", C.c_int64), ("steps", C.c_int64), ("integrate_ms", C.c_double),
                ("analyze_ms", C.c_double)]


class TuneResult(C.Structure):
    _fields_ = [("block", C.c_int32), ("blocks_per_sm", C.c_int32), ("regs", C.c_int32),
                ("resident_blocks", C.c_int32), ("persistent", C.c_int32), ("pad", C.c_int32),
                ("ms", C.c_double), ("lane_steps_per_s", C.c_double)]


class CMLP(C.Structure):
    _fields_ = [("params", C.c_void_p), ("adam_m", C.c_void_p), ("adam_v", C.c_void_p),
                ("grad", C.c_void_p), ("params_bf16", C.c_void_p), ("x_mean", C.c_float * 8),
                ("x_std", C.c_float * 8), ("step", C.c_int64)]


class ProposalSpec(C.Structure):
    _fields_ = [("E_col", C.c_double), ("v", C.c_int32), ("j", C.c_int32),
                ("n_b2", C.c_int32), ("n_cth", C.c_int32), ("n_phi", C.c_int32),
                ("n_eta", C.c_int32), ("n_chi", C.c_int32), ("pad", C.c_int32),
                ("b2_max", C.c_double), ("eps", C.c_double), ("alpha", C.c_double)]


class Cells(C.Structure):
    _fields_ = [("n_cells", C.c_int32), ("n_groups", C.c_int32), ("b", C.c_void_p),
                ("w", C.c_void_p), ("group", C.c_void_p), ("weighted", C.c_int32),
                ("pad", C.c_int32)]


def library_path() -> str:
    return _LIB_PATH


def lib():
    """Load libqcams.so (built by paper_2304_02731_gb300.build); raises if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise RuntimeError(
                    f"QCT CUDA library not built ({_LIB_PATH}); run "
                    "`python -c 'import __graft_entry__ as g; g.build()'` first")
            L = C.CDLL(_LIB_PATH)
            P, V, I32, I64, D = C.POINTER, C.c_void_p, C.c_int32, C.c_int64, C.c_double
            sig = {
                "qcams_status_string": (C.c_char_p, [C.c_int]),
                "qcams_system_setup": (C.c_int, [P(D), P(I32), P(D), P(System)]),
                "qcams_levels": (C.c_int, [P(System), I32, P(I32), P(I32), P(I32), I32, P(Level),
                                           V]),
                "qcams_init_states": (C.c_int, [P(System), I32, V, V, V, V, D, C.c_uint64,
                                                C.c_uint64, V, P(CBatch), V]),
                "qcams_run_batch": (C.c_int, [P(System), I32, P(Integ), P(CBatch), V]),
                "qcams_analyze": (C.c_int, [P(System), I32, P(Integ), P(CBatch), V]),
                "qcams_reduce_xsec": (C.c_int, [P(CBatch), P(Cells), V, V, V]),
                "qcams_xsec_from_hist": (C.c_int, [P(I64), P(Cells), P(D)]),
                "qcams_last_run_stats": (C.c_int, [P(RunStats), V]),
                "qcams_fma_peak": (C.c_int, [I32, P(D), V]),
                "qcams_device_info": (C.c_int, [P(I32), P(I32), P(I32)]),
                "qcams_shutdown": (C.c_int, []),
                "qcams_run_batch_noalloc": (C.c_int, [P(System), I32, P(Integ), P(CBatch), V]),
                "qcams_debug_exp": (C.c_int, [V, V, V, I64, V]),
                "qcams_debug_force_math": (C.c_int, [V, D, D, V, V, V, I64, V]),
                "qcams_debug_ff_dot": (C.c_int, [V, V, I32, V, V, I64, V]),
                "qcams_debug_context_exists": (C.c_int, [P(I32)]),
                "qcams_autotune": (C.c_int, [P(System), I32, P(Integ), P(CBatch), I64,
                                             P(TuneResult), P(I32), P(Integ), V]),
                "qcams_mlp_init": (C.c_int, [P(CMLP), C.c_uint64, V]),
                "qcams_mlp_sync": (C.c_int, [P(CMLP), V]),
                "qcams_mlp_features": (C.c_int, [P(CBatch), V, V, V, V, V, V]),
                "qcams_mlp_fit_standardizer": (C.c_int, [P(CMLP), V, I64, V]),
                "qcams_mlp_grad": (C.c_int, [P(CMLP), V, V, I64, V, V]),
                "qcams_mlp_train_step": (C.c_int, [P(CMLP), V, V, I64, C.c_float, V, V]),
                "qcams_mlp_train": (C.c_int, [P(CMLP), V, V, I64, I64, I32, C.c_float,
                                              C.c_uint64, V, V, V]),
                "qcams_mlp_infer": (C.c_int, [P(CMLP), V, I64, V, V]),
                "qcams_build_proposal": (C.c_int, [P(CMLP), P(ProposalSpec), V, V, V, V]),
                "qcams_sample_proposal": (C.c_int, [P(ProposalSpec), V, V, I64, C.c_uint64,
                                                    C.c_uint64, V, V, V, V, V]),
                "qcams_rate_constants": (C.c_int, [P(D), P(D), P(D), I32, D, P(D), P(D)]),
                "qcams_gb_distribution": (C.c_int, [P(I64), I32, P(I32), I32, P(D), P(D)]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(code: int, where: str):
    if code != 0:
        raise QcamsError(code, where)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


# ---------------------------------------------------------------------------
# systems and parameters
# ---------------------------------------------------------------------------
def system_setup(spec) -> System:
    """spec: dict(mass_u=(mA, mB, mC), pairs=[(kind_name, *params)] * 3)."""
    mass = (C.c_double * 3)(*[float(x) for x in spec["mass_u"]])
    kinds = (C.c_int32 * 3)()
    par = (C.c_double * 15)()
    for k, pr in enumerate(spec["pairs"]):
        kinds[k] = SPEC_KIND[pr[0]]
        for i, x in enumerate(pr[1:]):
            par[5 * k + i] = float(x)
    out = System()
    _check(lib().qcams_system_setup(mass, kinds, par, C.byref(out)), "qcams_system_setup")
    return out


def systems_array(systems):
    arr = (System * len(systems))()
    for i, s in enumerate(systems):
        arr[i] = s if isinstance(s, System) else system_setup(s)
    return arr


# qcams_integ.persistent = 2 / 3: three / six lanes per trajectory (FP64,
# small batches)
LAUNCH_TRI = 2
LAUNCH_HEX = 3


def make_integ(rtol=1e-10, atol=1e-12, r_stop=35.0, t_stop=15.0, h_fixed=0.0,
               gb_sigma=GB_SIGMA_DEFAULT, max_steps=1_000_000, fixed_step=False, precision=64,
               persistent=False, block=0, blocks_per_sm=0) -> Integ:
    return Integ(rtol, atol, r_stop, t_stop, h_fixed, gb_sigma, int(max_steps),
                 int(bool(fixed_step)), int(precision), int(persistent), int(block),
                 int(blocks_per_sm), 0)


# ---------------------------------------------------------------------------
# batches
# ---------------------------------------------------------------------------
_FIELDS_F64 = ["t", "h", "t_scale", "E0", "Ecol", "dE", "vprime", "jprime", "gbw"]


@dataclass
class Batch:
    """Structure-of-arrays device storage for n trajectories (qcams_batch)."""
    n: int
    device: torch.device
    y: torch.Tensor          # [12, n] float64
    f64: dict                # name -> [n] float64
    sys_id: torch.Tensor
    cell: torch.Tensor
    isw: torch.Tensor | None
    u: torch.Tensor | None   # [4, n] float64 (uniforms written by init)
    status: torch.Tensor
    cls: torch.Tensor
    nsteps: torch.Tensor
    nrej: torch.Tensor
    vt: torch.Tensor
    jt: torch.Tensor
    _c: CBatch = None

    @staticmethod
    def empty(n: int, device="cuda", sys_id=None, cell=None, isw=None, keep_u=True) -> "Batch":
        dev = torch.device(device)
        z = lambda dt: torch.zeros(n, dtype=dt, device=dev)
        sid = z(torch.int32) if sys_id is None else torch.as_tensor(
            sys_id, dtype=torch.int32).to(dev).contiguous()
        cel = z(torch.int32) if cell is None else torch.as_tensor(
            cell, dtype=torch.int32).to(dev).contiguous()
        w = None if isw is None else torch.as_tensor(isw, dtype=torch.float64).to(dev).contiguous()
        b = Batch(n=n, device=dev, y=torch.zeros(12, n, dtype=torch.float64, device=dev),
                  f64={k: z(torch.float64) for k in _FIELDS_F64}, sys_id=sid, cell=cel, isw=w,
                  u=torch.zeros(4, n, dtype=torch.float64, device=dev) if keep_u else None,
                  status=z(torch.uint8), cls=z(torch.uint8), nsteps=z(torch.int32),
                  nrej=z(torch.int32), vt=z(torch.int16), jt=z(torch.int16))
        b._build()
        return b

    def _build(self):
        c = CBatch()
        c.n = self.n
        c.sys_id = self.sys_id.data_ptr()
        c.cell = self.cell.data_ptr()
        c.isw = self.isw.data_ptr() if self.isw is not None else None
        for k in range(12):
            c.y[k] = self.y[k].data_ptr()
        for name in _FIELDS_F64:
            setattr(c, name, self.f64[name].data_ptr())
        for k in range(4):
            c.u[k] = self.u[k].data_ptr() if self.u is not None else None
        c.status = self.status.data_ptr()
        c.cls = self.cls.data_ptr()
        c.nsteps = self.nsteps.data_ptr()
        c.nrej = self.nrej.data_ptr()
        c.vt = self.vt.data_ptr()
        c.jt = self.jt.data_ptr()
        self._c = c

    @property
    def c(self) -> CBatch:
        return self._c

    def state(self) -> np.ndarray:
        """[n, 12] host copy of the phase-space state."""
        return self.y.t().contiguous().cpu().numpy()

    def set_state(self, y: np.ndarray):
        self.y.copy_(torch.as_tensor(np.ascontiguousarray(y.T), dtype=torch.float64))

    def host(self) -> dict:
        out = {k: v.cpu().numpy() for k, v in self.f64.items()}
        for k in ["status", "cls", "nsteps", "nrej", "vt", "jt"]:
            out[k] = getattr(self, k).cpu().numpy()
        out["y"] = self.state()
        if self.u is not None:
            out["u"] = self.u.t().contiguous().cpu().numpy()
        return out


def _dptr(x, dtype, device):
    """(device tensor, staged) — staged is True when a copy was made."""
    if isinstance(x, torch.Tensor) and x.device == device and x.dtype == dtype \
            and x.is_contiguous():
        return x, False
    t = torch.as_tensor(x, dtype=dtype)
    if t.device != device:
        t = t.to(device, non_blocking=True)
    return t.contiguous(), True


# ---------------------------------------------------------------------------
# entry points
# ---------------------------------------------------------------------------
def levels(systems, sys_id, v, j, stream=None):
    """qcams_levels: Bohr-Sommerfeld levels (host in / host out)."""
    arr = systems_array(systems)
    n = len(v)
    sid = np.ascontiguousarray(sys_id, np.int32)
    vv = np.ascontiguousarray(v, np.int32)
    jj = np.ascontiguousarray(j, np.int32)
    out = (Level * n)()
    P = C.POINTER(C.c_int32)
    rc = lib().qcams_levels(arr, len(systems), sid.ctypes.data_as(P), vv.ctypes.data_as(P),
                            jj.ctypes.data_as(P), n, out, _stream(stream))
    if rc not in (0, -2):
        _check(rc, "qcams_levels")
    return np.array([(L.E, L.r_minus, L.r_plus, L.tau, L.ok) for L in out],
                    dtype=[("E", "f8"), ("r_minus", "f8"), ("r_plus", "f8"), ("tau", "f8"),
                           ("ok", "i4")])


def init_states(systems, batch: Batch, E, b, v, j, R0: float, seed: int, id_offset: int = 0,
                u_in=None, stream=None):
    """qcams_init_states on `batch` (inputs may be host or device arrays)."""
    arr = systems_array(systems)
    dev = batch.device
    staged = [_dptr(E, torch.float64, dev), _dptr(b, torch.float64, dev),
              _dptr(v, torch.int32, dev), _dptr(j, torch.int32, dev)]
    tE, tb, tv, tj = [t for t, _ in staged]
    uptr = None
    if u_in is not None:
        tu, cp = _dptr(u_in, torch.float64, dev)
        tu = tu.reshape(4, batch.n)
        staged.append((tu, cp))
        uptr = (C.c_void_p * 4)(*[tu[k].data_ptr() for k in range(4)])
    keep = [t for t, cp in staged if cp]
    rc = lib().qcams_init_states(arr, len(systems), tE.data_ptr(), tb.data_ptr(), tv.data_ptr(),
                                 tj.data_ptr(), float(R0), int(seed), int(id_offset), uptr,
                                 C.byref(batch.c), _stream(stream))
    _check(rc, "qcams_init_states")
    # the staged inputs are consumed asynchronously on `stream`
    s = stream if stream is not None else torch.cuda.current_stream()
    for t in keep:
        t.record_stream(s)
    return keep


def run_batch(systems, batch: Batch, integ: Integ, stream=None):
    """qcams_run_batch: integrate (and, unless fixed-step, analyse) the batch."""
    arr = systems_array(systems)
    _check(lib().qcams_run_batch(arr, len(systems), C.byref(integ), C.byref(batch.c),
                                 _stream(stream)), "qcams_run_batch")


def run_batch_noalloc(systems, batch: Batch, integ: Integ, stream=None):
    """qcams_run_batch_noalloc: qcams_run_batch for callers that must not
    allocate device memory (scratch in a fixed static device array)."""
    arr = systems_array(systems)
    _check(lib().qcams_run_batch_noalloc(arr, len(systems), C.byref(integ), C.byref(batch.c),
                                         _stream(stream)), "qcams_run_batch_noalloc")


def analyze(systems, batch: Batch, integ: Integ, stream=None):
    arr = systems_array(systems)
    _check(lib().qcams_analyze(arr, len(systems), C.byref(integ), C.byref(batch.c),
                               _stream(stream)), "qcams_analyze")


def reduce_xsec(batch: Batch, n_cells: int, cell_b=None, cell_w=None, group=None, n_groups=0,
                weighted=False, hist_out: torch.Tensor | None = None, stream=None,
                finalize=True):
    """qcams_reduce_xsec.  Returns (hist [n_cells, H_STRIDE] device tensor,
    cells [n_cells, 7, 2] and groups [n_groups, 7, 2] host arrays or None: entries
    0..5 the classes, 6 the reactive total R_AC + R_BC)."""
    if hist_out is None:
        hist_out = torch.empty(n_cells * H_STRIDE, dtype=torch.int64, device=batch.device)
    cells = Cells()
    cells.n_cells = int(n_cells)
    cells.n_groups = int(n_groups)
    keep = []
    if finalize:
        cb = np.ascontiguousarray(cell_b, np.float64)
        cw = np.ascontiguousarray(cell_w, np.float64)
        cg = np.ascontiguousarray(group if group is not None else np.zeros(n_cells), np.int32)
        keep += [cb, cw, cg]
        cells.b = cb.ctypes.data
        cells.w = cw.ctypes.data
        cells.group = cg.ctypes.data
    cells.weighted = int(bool(weighted))
    out = np.zeros(14 * n_cells + 14 * n_groups) if finalize else None
    rc = lib().qcams_reduce_xsec(C.byref(batch.c), C.byref(cells), C.c_void_p(hist_out.data_ptr()),
                                 C.c_void_p(out.ctypes.data) if finalize else None,
                                 _stream(stream))
    _check(rc, "qcams_reduce_xsec")
    hist = hist_out.view(n_cells, H_STRIDE)
    if not finalize:
        return hist, None, None
    return (hist, out[:14 * n_cells].reshape(n_cells, 7, 2),
            out[14 * n_cells:].reshape(n_groups, 7, 2))


def xsec_from_hist(hist, cell_b, cell_w, group, n_groups, weighted=False):
    """qcams_xsec_from_hist: cross sections from host int64 histograms
    [n_cells, H_STRIDE] (e.g. the merged histograms of several shards).
    Returns (cells [n_cells, 7, 2], groups [n_groups, 7, 2])."""
    h = np.ascontiguousarray(hist, np.int64).reshape(-1, H_STRIDE)
    n_cells = h.shape[0]
    cells = Cells()
    cells.n_cells = int(n_cells)
    cells.n_groups = int(n_groups)
    cb = np.ascontiguousarray(cell_b, np.float64)
    cw = np.ascontiguousarray(cell_w, np.float64)
    cg = np.ascontiguousarray(group, np.int32)
    cells.b, cells.w, cells.group = cb.ctypes.data, cw.ctypes.data, cg.ctypes.data
    cells.weighted = int(bool(weighted))
    out = np.zeros(14 * n_cells + 14 * n_groups)
    _check(lib().qcams_xsec_from_hist(h.ctypes.data_as(C.POINTER(C.c_int64)), C.byref(cells),
                                      out.ctypes.data_as(C.POINTER(C.c_double))),
           "qcams_xsec_from_hist")
    return out[:14 * n_cells].reshape(n_cells, 7, 2), out[14 * n_cells:].reshape(n_groups, 7, 2)


def last_run_stats(stream=None) -> dict:
    """qcams_last_run_stats: work counters and kernel times of the last run."""
    st = RunStats()
    _check(lib().qcams_last_run_stats(C.byref(st), _stream(stream)), "qcams_last_run_stats")
    return dict(rhs=st.rhs, steps=st.steps, integrate_ms=st.integrate_ms,
                analyze_ms=st.analyze_ms)


def fma_peak(precision: int = 64, stream=None) -> float:
    f = C.c_double()
    _check(lib().qcams_fma_peak(int(precision), C.byref(f), _stream(stream)), "qcams_fma_peak")
    return f.value


def autotune(systems, sample: Batch, integ: Integ, max_attempts: int = 1500, stream=None):
    """qcams_autotune: measure every launch (the persistent shapes and the
    three- and six-lane groups) on an initialised sample batch; returns (best
    Integ, list of per-launch result dicts)."""
    arr = systems_array(systems)
    res = (TuneResult * 16)()
    nres = C.c_int32()
    best = Integ()
    _check(lib().qcams_autotune(arr, len(systems), C.byref(integ), C.byref(sample.c),
                                int(max_attempts), res, C.byref(nres), C.byref(best),
                                _stream(stream)), "qcams_autotune")
    out = [dict(block=r.block, blocks_per_sm=r.blocks_per_sm, persistent=r.persistent,
                regs=r.regs, resident_blocks=r.resident_blocks, ms=r.ms,
                lane_steps_per_s=r.lane_steps_per_s)
           for r in res[:nres.value]]
    return best, out


def debug_force_math(s: torch.Tensor, alpha: float, alpha_re: float, stream=None):
    """qcams_debug_force_math: (1/sqrt(s), x = alpha_re - alpha r, e^x) as the
    integrator's Morse force law forms them, for the device tensor s."""
    s = s.to(torch.float64).contiguous()
    ri, x, e = torch.empty_like(s), torch.empty_like(s), torch.empty_like(s)
    _check(lib().qcams_debug_force_math(s.data_ptr(), float(alpha), float(alpha_re),
                                        ri.data_ptr(), x.data_ptr(), e.data_ptr(), s.numel(),
                                        _stream(stream)), "qcams_debug_force_math")
    return ri, x, e


def debug_ff_dot(a: torch.Tensor, w: torch.Tensor, stream=None):
    """qcams_debug_ff_dot: (sum_q w[q] a[:, q] as the integrator's float-float
    dot product forms it, as a double and rounded to FP32) for device
    tensors a [n, m] and w [m]."""
    a = a.to(torch.float64).contiguous()
    w = w.to(device=a.device, dtype=torch.float64).contiguous()
    n, m = a.shape
    out = torch.empty(n, dtype=torch.float64, device=a.device)
    out_f = torch.empty(n, dtype=torch.float32, device=a.device)
    _check(lib().qcams_debug_ff_dot(a.data_ptr(), w.data_ptr(), m, out.data_ptr(),
                                    out_f.data_ptr(), n, _stream(stream)), "qcams_debug_ff_dot")
    return out, out_f


def debug_exp(x: torch.Tensor, stream=None):
    """qcams_debug_exp: (table-driven exp, CUDA exp) of the device tensor x."""
    x = x.to(torch.float64).contiguous()
    a, b = torch.empty_like(x), torch.empty_like(x)
    _check(lib().qcams_debug_exp(x.data_ptr(), a.data_ptr(), b.data_ptr(), x.numel(),
                                 _stream(stream)), "qcams_debug_exp")
    return a, b


def debug_context_exists() -> bool:
    """qcams_debug_context_exists: whether the library's per-device context
    (its only device allocations outside the autotuner) exists."""
    out = C.c_int32(0)
    _check(lib().qcams_debug_context_exists(C.byref(out)), "qcams_debug_context_exists")
    return bool(out.value)


def device_info():
    a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
    _check(lib().qcams_device_info(C.byref(a), C.byref(b), C.byref(c)), "qcams_device_info")
    return a.value, (b.value, c.value)


# ---------------------------------------------------------------------------
# convenience: a whole workload in one call
# ---------------------------------------------------------------------------
def run_workload(wl, integ: Integ | None = None, device="cuda", stream=None, finalize=True,
                 batch: Batch | None = None):
    """init -> run -> reduce for a workloads.Workload; returns (batch, hist, cells, groups)."""
    if integ is None:
        integ = make_integ(**wl.integ)
    if batch is None:
        batch = Batch.empty(wl.n, device, sys_id=wl.sys_id, cell=wl.cell)
    init_states(wl.systems, batch, wl.E, wl.b, wl.v, wl.j, wl.R0, wl.seed, wl.id_offset,
                stream=stream)
    run_batch(wl.systems, batch, integ, stream=stream)
    hist, cells, groups = reduce_xsec(batch, wl.n_cells, wl.cell_b, wl.cell_w, wl.cell_group,
                                      wl.n_groups, stream=stream, finalize=finalize)
    return batch, hist, cells, groups


# ---------------------------------------------------------------------------
# learned importance-sampling proposal
# ---------------------------------------------------------------------------
class MLP:
    """Device storage of the outcome MLP (qcams_mlp) and its entry points."""

    def __init__(self, device="cuda", seed: int = 0):
        dev = torch.device(device)
        f = lambda: torch.zeros(MLP_NPARAMS, dtype=torch.float32, device=dev)
        self.device = dev
        self.params, self.m, self.v, self.grad = f(), f(), f(), f()
        self.params_bf16 = torch.zeros(MLP_NPARAMS, dtype=torch.int16, device=dev)
        self.loss = torch.zeros(1, dtype=torch.float32, device=dev)
        self.c = CMLP()
        self.c.params = self.params.data_ptr()
        self.c.adam_m = self.m.data_ptr()
        self.c.adam_v = self.v.data_ptr()
        self.c.grad = self.grad.data_ptr()
        self.c.params_bf16 = self.params_bf16.data_ptr()
        _check(lib().qcams_mlp_init(C.byref(self.c), int(seed), _stream()), "qcams_mlp_init")

    def set_params(self, values):
        self.params.copy_(torch.as_tensor(values, dtype=torch.float32))
        _check(lib().qcams_mlp_sync(C.byref(self.c), _stream()), "qcams_mlp_sync")

    def set_standardizer(self, mean, std):
        for k in range(8):
            self.c.x_mean[k] = float(mean[k])
            self.c.x_std[k] = float(std[k])

    @property
    def standardizer(self):
        return np.array(list(self.c.x_mean)), np.array(list(self.c.x_std))

    @property
    def step(self) -> int:
        return self.c.step

    def features(self, batch: Batch, E, b, v, j) -> torch.Tensor:
        return mlp_features(batch, E, b, v, j)

    def fit_standardizer(self, x: torch.Tensor):
        x = x.contiguous()
        _check(lib().qcams_mlp_fit_standardizer(C.byref(self.c), x.data_ptr(), x.shape[0],
                                                _stream()), "qcams_mlp_fit_standardizer")

    def compute_grad(self, x: torch.Tensor, cls: torch.Tensor) -> float:
        x, cls = x.contiguous(), cls.to(torch.uint8).contiguous()
        _check(lib().qcams_mlp_grad(C.byref(self.c), x.data_ptr(), cls.data_ptr(), x.shape[0],
                                    self.loss.data_ptr(), _stream()), "qcams_mlp_grad")
        return self.loss

    def train_step(self, x: torch.Tensor, cls: torch.Tensor, lr: float):
        _check(lib().qcams_mlp_train_step(C.byref(self.c), x.data_ptr(), cls.data_ptr(),
                                          x.shape[0], float(lr), self.loss.data_ptr(),
                                          _stream()), "qcams_mlp_train_step")
        return self.loss

    def train(self, x: torch.Tensor, cls: torch.Tensor, steps: int, batch: int, lr: float,
              seed: int = 0):
        """qcams_mlp_train: `steps` device-side minibatch Adam steps (indices
        drawn with replacement).  Returns (losses [steps], last indices)."""
        x, cls = x.contiguous(), cls.contiguous()
        losses = torch.empty(max(int(steps), 1), dtype=torch.float32, device=x.device)
        idx = torch.empty(int(batch), dtype=torch.int64, device=x.device)
        _check(lib().qcams_mlp_train(C.byref(self.c), x.data_ptr(), cls.data_ptr(), x.shape[0],
                                     int(steps), int(batch), float(lr), int(seed),
                                     idx.data_ptr(), losses.data_ptr(), _stream()),
               "qcams_mlp_train")
        return losses[:int(steps)], idx

    def infer(self, x: torch.Tensor) -> torch.Tensor:
        x = x.contiguous()
        probs = torch.empty(x.shape[0], 4, dtype=torch.float32, device=x.device)
        _check(lib().qcams_mlp_infer(C.byref(self.c), x.data_ptr(), x.shape[0],
                                     probs.data_ptr(), _stream()), "qcams_mlp_infer")
        return probs

    def build_proposal(self, spec: ProposalSpec):
        N = spec.n_b2 * spec.n_cth * spec.n_phi * spec.n_eta * spec.n_chi
        q = torch.empty(N, dtype=torch.float64, device=self.device)
        qfix = torch.empty(N, dtype=torch.int64, device=self.device)
        cdf = torch.empty(N, dtype=torch.int64, device=self.device)
        _check(lib().qcams_build_proposal(C.byref(self.c), C.byref(spec), q.data_ptr(),
                                          qfix.data_ptr(), cdf.data_ptr(), _stream()),
               "qcams_build_proposal")
        return q, qfix, cdf


def proposal_spec(E_col, v, j, dims=(16, 8, 8, 8, 4), b2_max=100.0, eps=1e-3,
                  alpha=0.1) -> ProposalSpec:
    s = ProposalSpec()
    s.E_col, s.v, s.j = float(E_col), int(v), int(j)
    s.n_b2, s.n_cth, s.n_phi, s.n_eta, s.n_chi = (int(d) for d in dims)
    s.b2_max, s.eps, s.alpha = float(b2_max), float(eps), float(alpha)
    return s


def sample_proposal(spec: ProposalSpec, qfix: torch.Tensor, cdf: torch.Tensor, n: int,
                    seed: int, id_offset: int = 0):
    """qcams_sample_proposal: (b, u[4, n], w, cell) device tensors."""
    dev = qfix.device
    b = torch.empty(n, dtype=torch.float64, device=dev)
    u = torch.empty(4, n, dtype=torch.float64, device=dev)
    w = torch.empty(n, dtype=torch.float64, device=dev)
    cell = torch.empty(n, dtype=torch.int32, device=dev)
    uptr = (C.c_void_p * 4)(*[u[k].data_ptr() for k in range(4)])
    _check(lib().qcams_sample_proposal(C.byref(spec), qfix.data_ptr(), cdf.data_ptr(), int(n),
                                       int(seed), int(id_offset), b.data_ptr(), uptr,
                                       w.data_ptr(), cell.data_ptr(), _stream()),
           "qcams_sample_proposal")
    return b, u, w, cell


def mlp_features(batch: Batch, E, b, v, j) -> torch.Tensor:
    """qcams_mlp_features: network inputs [n, 8] of initialised lanes."""
    dev = batch.device
    tE, _ = _dptr(E, torch.float64, dev)
    tb, _ = _dptr(b, torch.float64, dev)
    tv, _ = _dptr(v, torch.int32, dev)
    tj, _ = _dptr(j, torch.int32, dev)
    x = torch.empty(batch.n, 8, dtype=torch.float32, device=dev)
    _check(lib().qcams_mlp_features(C.byref(batch.c), tE.data_ptr(), tb.data_ptr(),
                                    tv.data_ptr(), tj.data_ptr(), x.data_ptr(), _stream()),
           "qcams_mlp_features")
    torch.cuda.current_stream().synchronize()
    return x


# ---------------------------------------------------------------------------
# reports
# ---------------------------------------------------------------------------
def rate_constants(sigma, sigma_se, E_col, mu123: float):
    """qcams_rate_constants: (k, k_se) host arrays."""
    sg, se, E = (np.ascontiguousarray(a, np.float64) for a in (sigma, sigma_se, E_col))
    k, kse = np.zeros(sg.size), np.zeros(sg.size)
    P = C.POINTER(C.c_double)
    _check(lib().qcams_rate_constants(sg.ctypes.data_as(P), se.ctypes.data_as(P),
                                      E.ctypes.data_as(P), sg.size, float(mu123),
                                      k.ctypes.data_as(P), kse.ctypes.data_as(P)),
           "qcams_rate_constants")
    return k, kse


def gb_distribution(hist, cell_ids):
    """qcams_gb_distribution: ([3, 64] distribution, W) from host histograms."""
    h = np.ascontiguousarray(np.asarray(hist).reshape(-1, H_STRIDE), np.int64)
    ids = np.ascontiguousarray(cell_ids, np.int32)
    out = np.zeros(3 * 64)
    W = C.c_double()
    _check(lib().qcams_gb_distribution(h.ctypes.data_as(C.POINTER(C.c_int64)), h.shape[0],
                                       ids.ctypes.data_as(C.POINTER(C.c_int32)), ids.size,
                                       out.ctypes.data_as(C.POINTER(C.c_double)), C.byref(W)),
           "qcams_gb_distribution")
    return out.reshape(3, 64), W.value
