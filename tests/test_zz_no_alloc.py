"""qcams_run_batch_noalloc: the integrate + analyse entry point for callers
that cannot allocate device memory (it keeps its scratch in a static device
array).  Its outputs must equal those of qcams_run_batch on the same
initial states; two calls in a row check that the shared scratch (shape
table and counters) is rewritten and cleared between calls.  The same
lanes give bit-identical results, which satisfies any tolerance the other
parity tests use."""
import ctypes as C
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from paper_2304_02731_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FIELDS = ["y", "t", "h", "status", "cls", "nsteps", "nrej", "dE", "vprime", "jprime", "gbw",
          "vt", "jt"]


@pytest.fixture(scope="module")
def Q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_02731_gb300 import build
    build.build()
    from paper_2304_02731_gb300 import qcams
    qcams.lib()
    return qcams


def _run(Q, wl, entry, persistent, **integ_kw):
    import torch
    integ = Q.make_integ(**dict(wl.integ, **integ_kw), persistent=persistent)
    batch = Q.Batch.empty(wl.n, "cuda", sys_id=wl.sys_id, cell=wl.cell)
    Q.init_states(wl.systems, batch, wl.E, wl.b, wl.v, wl.j, wl.R0, wl.seed, wl.id_offset)
    arr = Q.systems_array(wl.systems)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    fn = getattr(Q.lib(), entry)
    rc = fn(arr, len(wl.systems), C.byref(integ), C.byref(batch.c), stream)
    assert rc == 0, Q.lib().qcams_status_string(rc)
    torch.cuda.synchronize()
    return batch.host()


def test_noalloc_matches_run_batch_on_two_calls(Q):
    # call 1: all-Morse plain study lanes (persistent launch);
    # call 2: mixed Buckingham / LJ systems (one thread per lane);
    # calls 3, 4: three lanes per trajectory; call 5: six lanes
    cases = [(W.plain_h2_ca(per_b=12), True), (W.mixed_ca_h(n=120, seed=5), False),
             (W.plain_h2_ca(per_b=12), Q.LAUNCH_TRI), (W.mixed_ca_h(n=121, seed=5), Q.LAUNCH_TRI),
             (W.mixed_ca_h(n=61, seed=5), Q.LAUNCH_HEX)]
    for wl, persistent in cases:
        ref = _run(Q, wl, "qcams_run_batch", persistent)
        got = _run(Q, wl, "qcams_run_batch_noalloc", persistent)
        assert np.all(np.isin(got["status"], [2, 3, 8])), got["status"]
        for k in FIELDS:
            assert np.array_equal(got[k], ref[k]), k


def test_noalloc_fp32_and_fixed_step(Q):
    """The FP32 integrator (its own refill-queue head in the shared scratch;
    persistent and one thread per lane, Morse and mixed systems) and the
    fixed-step mode (no analysis) give the same bits as qcams_run_batch."""
    plain, mixed = W.plain_h2_ca(per_b=12), W.mixed_ca_h(n=120, seed=6)
    cases = [(plain, True, dict(W.INTEG_FP32, precision=32)),
             (mixed, True, dict(W.INTEG_FP32, precision=32)),
             (plain, False, dict(W.INTEG_FP32, precision=32)),
             (plain, False, dict(fixed_step=True, h_fixed=0.5, max_steps=300)),
             (mixed, False, dict(fixed_step=True, h_fixed=0.5, max_steps=300))]
    for wl, persistent, kw in cases:
        ref = _run(Q, wl, "qcams_run_batch", persistent, **kw)
        got = _run(Q, wl, "qcams_run_batch_noalloc", persistent, **kw)
        if kw.get("fixed_step"):
            assert np.all(np.isin(got["status"], [1, 8])), got["status"]
        else:
            assert np.all(np.isin(got["status"], [2, 3, 8])), got["status"]
        for k in FIELDS:
            assert np.array_equal(got[k], ref[k]), (k, kw, persistent)


def test_noalloc_rejects_too_many_systems(Q):
    import torch
    wl = W.plain_h2_ca(per_b=1)
    arr = Q.systems_array(wl.systems * 5)
    batch = Q.Batch.empty(wl.n, "cuda")
    integ = Q.make_integ()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert Q.lib().qcams_run_batch_noalloc(arr, 5, C.byref(integ), C.byref(batch.c), stream) == -4


_CHILD = textwrap.dedent("""
    import ctypes as C, sys
    import numpy as np, torch
    sys.path.insert(0, sys.argv[1])
    from paper_2304_02731_gb300 import qcams as Q
    from paper_2304_02731_gb300 import workloads as W
    src = np.load(sys.argv[2])
    wl = W.plain_h2_ca(per_b=12)
    batch = Q.Batch.empty(wl.n, "cuda", sys_id=wl.sys_id, cell=wl.cell)
    batch.y.copy_(torch.as_tensor(src["y0"]))
    for k in Q._FIELDS_F64:
        batch.f64[k].copy_(torch.as_tensor(src["f0_" + k]))
    batch.status.copy_(torch.as_tensor(src["status0"]))
    integ = Q.make_integ(**wl.integ, persistent=True)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    rc = Q.lib().qcams_run_batch_noalloc(Q.systems_array(wl.systems), len(wl.systems),
                                         C.byref(integ), C.byref(batch.c), stream)
    assert rc == 0, rc
    torch.cuda.synchronize()
    # the library's per-device context (its cudaMalloc'd scratch) was never created
    assert not Q.debug_context_exists()
    out = batch.host()
    # a second call on the same lanes (now finished) allocates nothing either
    free0 = torch.cuda.mem_get_info()[0]
    rc = Q.lib().qcams_run_batch_noalloc(Q.systems_array(wl.systems), len(wl.systems),
                                         C.byref(integ), C.byref(batch.c), stream)
    assert rc == 0, rc
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert not Q.debug_context_exists()
    np.savez(sys.argv[3], **out)
""")


def test_noalloc_as_the_first_call_of_a_process(Q, tmp_path):
    """In a fresh process whose only library calls are
    qcams_run_batch_noalloc, the results equal qcams_run_batch's on the
    same initial states, and the library's per-device context (the scratch
    qcams_run_batch allocates with cudaMalloc) is never created."""
    import torch
    wl = W.plain_h2_ca(per_b=12)
    batch = Q.Batch.empty(wl.n, "cuda", sys_id=wl.sys_id, cell=wl.cell)
    Q.init_states(wl.systems, batch, wl.E, wl.b, wl.v, wl.j, wl.R0, wl.seed, wl.id_offset)
    torch.cuda.synchronize()
    init = {"y0": batch.y.cpu().numpy(), "status0": batch.status.cpu().numpy()}
    init.update({"f0_" + k: v.cpu().numpy() for k, v in batch.f64.items()})
    np.savez(tmp_path / "init.npz", **init)
    Q.run_batch(wl.systems, batch, Q.make_integ(**wl.integ, persistent=True))
    torch.cuda.synchronize()
    ref = batch.host()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    subprocess.run([sys.executable, "-c", _CHILD, root, str(tmp_path / "init.npz"),
                    str(tmp_path / "out.npz")], check=True, timeout=600)
    got = np.load(tmp_path / "out.npz")
    assert np.all(np.isin(got["status"], [2, 3])), got["status"]
    for k in FIELDS:
        assert np.array_equal(got[k], ref[k]), k
