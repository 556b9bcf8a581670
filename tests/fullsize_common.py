"""Shared pieces of the full-size GPU tests: a workload run in the launch
configuration bench.py times (autotuned persistent refill-queue kernel, the
init -> integrate -> reduce step captured in one CUDA graph), the oracle run
lane by lane on host cores (spawned processes), and the comparison of cross
sections within combined binomial standard errors."""
import math
import os

import numpy as np

from paper_2304_02731_gb300 import workloads as W


def run_bench_config(wl, precision=64, integ_kw=None):
    """Run workload `wl` once as the benchmark does; returns (per-lane host
    outputs, histograms [n_cells][stride], per-cell and per-group xsec)."""
    import torch
    from paper_2304_02731_gb300 import build
    build.build()
    from paper_2304_02731_gb300 import qcams as Q
    dev = torch.device("cuda")
    integ = Q.make_integ(**(integ_kw or wl.integ), persistent=True, precision=precision)
    if precision == 64:
        sw = wl.take(W.stratified(wl, max(1, min(64, wl.n // wl.n_cells))))
        sb = Q.Batch.empty(sw.n, dev, sys_id=sw.sys_id, cell=sw.cell, keep_u=False)
        Q.init_states(sw.systems, sb, sw.E, sw.b, sw.v, sw.j, sw.R0, sw.seed)
        integ, _ = Q.autotune(sw.systems, sb, integ, max_attempts=500)
        del sb
    batch = Q.Batch.empty(wl.n, dev, sys_id=wl.sys_id, cell=wl.cell, keep_u=False)
    E, b = torch.as_tensor(wl.E, device=dev), torch.as_tensor(wl.b, device=dev)
    v, j = torch.as_tensor(wl.v, device=dev), torch.as_tensor(wl.j, device=dev)
    hist = torch.empty(wl.n_cells * Q.H_STRIDE, dtype=torch.int64, device=dev)
    g = torch.cuda.CUDAGraph()
    Q.init_states(wl.systems, batch, E, b, v, j, wl.R0, wl.seed)   # context before capture
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        Q.init_states(wl.systems, batch, E, b, v, j, wl.R0, wl.seed)
        Q.run_batch(wl.systems, batch, integ)
        Q.reduce_xsec(batch, wl.n_cells, hist_out=hist, finalize=False)
    g.replay()
    torch.cuda.synchronize()
    stats = Q.last_run_stats()
    _, cells, groups = Q.reduce_xsec(batch, wl.n_cells, wl.cell_b, wl.cell_w, wl.cell_group,
                                     wl.n_groups, hist_out=hist)
    out = dict(status=batch.status.cpu().numpy(), cls=batch.cls.cpu().numpy(),
               vt=batch.vt.cpu().numpy(), jt=batch.jt.cpu().numpy(),
               gbw=batch.f64["gbw"].cpu().numpy(), dE=batch.f64["dE"].cpu().numpy(),
               E0=batch.f64["E0"].cpu().numpy(), nsteps=batch.nsteps.cpu().numpy(),
               stats=stats)
    del batch, g
    return out, hist.cpu().numpy().reshape(wl.n_cells, -1), cells, groups


LANE_DTYPE = np.dtype([("cls", "i4"), ("vt", "i4"), ("jt", "i4"), ("status", "i4"),
                       ("nsteps", "i4"), ("dE", "f8"), ("E0", "f8")])


def _oracle_chunk(payload):
    import oracle as O
    specs, sid, E, b, v, j, R0, seed, ids, integ_kw = payload
    systems = [O.system_from_spec(sp) for sp in specs]
    integ = O.make_integ(**integ_kw)
    out = np.zeros(len(E), LANE_DTYPE)
    for k in range(len(E)):
        st, res = O.run_lanes(systems, sid[k:k + 1], E[k:k + 1], b[k:k + 1], v[k:k + 1],
                              j[k:k + 1], R0, seed, integ, id_offset=int(ids[k]))
        out[k] = (res["cls"][0], res["vt"][0], res["jt"][0], res["status"][0],
                  res["nsteps"][0], res["dE"][0], st["E0"][0])
    return out


def oracle_lanes(wl, idx, integ_kw=None):
    """The oracle's outcomes (LANE_DTYPE: cls, v_t, j_t, status, accepted
    steps, energy error, initial energy) for lanes idx of
    wl, each run from its own (seed, id), one oracle process per host core
    (spawned, so that no process inherits the parent's CUDA context)."""
    import multiprocessing as mp
    idx = np.asarray(idx)
    cores = max(1, min(os.cpu_count() or 1, 64))
    parts = [c for c in np.array_split(np.arange(len(idx)), cores) if len(c)]
    payloads = [(wl.systems, wl.sys_id[idx[c]], wl.E[idx[c]], wl.b[idx[c]], wl.v[idx[c]],
                 wl.j[idx[c]], wl.R0, wl.seed, wl.id_offset + idx[c],
                 dict(integ_kw or wl.integ)) for c in parts]
    with mp.get_context("spawn").Pool(len(payloads)) as pool:
        return np.concatenate(pool.map(_oracle_chunk, payloads))


def sigma_deviations(wl, groups, idx, res, oracle, classes=(0, 1, 2, 3)):
    """|sigma_gpu - sigma_oracle| / SE for every group and class, with the
    oracle's estimate from the sampled lanes idx (outcomes res) and SE the
    two estimates' standard errors combined.  A count of 0 or N has a zero
    binomial error; the sample's error is bounded with the count clipped to
    [1, N - 1].  Returns (deviations [n_groups][len(classes)], the median
    ratio of the oracle sample's SE to the GPU's over the non-degenerate
    entries)."""
    cls_o = res["cls"]
    zeros = np.zeros(len(idx), np.int32)
    h_o = oracle.reduce(cls_o, zeros, zeros, np.zeros(len(idx)), wl.cell[idx], wl.n_cells)
    _, g_o = oracle.xsec(h_o, wl.cell_b, wl.cell_w, wl.cell_group, wl.n_groups)
    N = h_o[:, :5].sum(axis=1).astype(float)
    wb = wl.cell_w * wl.cell_b
    dev = np.zeros((wl.n_groups, len(classes)))
    ratios = []
    for g in range(wl.n_groups):
        cg = (wl.cell_group == g) & (N > 0)
        for col, k in enumerate(classes):
            p = np.clip(h_o[cg, k], 1, N[cg] - 1) / N[cg]
            se_o = 2 * math.pi * math.sqrt(np.sum(wb[cg] ** 2 * p * (1 - p) / N[cg]))
            se_o = max(g_o[g, k, 1], se_o)
            se = math.hypot(groups[g, k, 1], se_o)
            dev[g, col] = abs(groups[g, k, 0] - g_o[g, k, 0]) / se if se > 0 else 0.0
            if groups[g, k, 1] > 0 and g_o[g, k, 1] > 0:
                ratios.append(g_o[g, k, 1] / groups[g, k, 1])
    return dev, float(np.median(ratios)) if ratios else float("nan")
