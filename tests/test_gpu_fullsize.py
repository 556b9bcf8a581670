"""Full-size parity: the 3,145,728-trajectory H2 + Ca sweep (16 energies x
24 impact parameters x 8,192) in the launch configuration bench.py times
(autotuned persistent refill-queue kernel, step captured in a CUDA graph),
checked on lanes sampled across every energy and the oracle run one by one,
and on properties that hold at any size."""
import math

import numpy as np
import pytest

from paper_2304_02731_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full_run():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_02731_gb300 import build
    build.build()
    from paper_2304_02731_gb300 import qcams as Q
    dev = torch.device("cuda")
    wl = W.sweep_h2_ca()
    integ = Q.make_integ(**wl.integ, persistent=True)
    sw = wl.take(W.stratified(wl, 64))
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
    _, cells, groups = Q.reduce_xsec(batch, wl.n_cells, wl.cell_b, wl.cell_w, wl.cell_group,
                                     wl.n_groups, hist_out=hist)
    out = dict(status=batch.status.cpu().numpy(), cls=batch.cls.cpu().numpy(),
               vt=batch.vt.cpu().numpy(), jt=batch.jt.cpu().numpy(),
               gbw=batch.f64["gbw"].cpu().numpy(), dE=batch.f64["dE"].cpu().numpy(),
               E0=batch.f64["E0"].cpu().numpy(), nsteps=batch.nsteps.cpu().numpy())
    return wl, out, hist.cpu().numpy().reshape(wl.n_cells, -1), cells, groups


def test_full_size_sampled_lanes_match_oracle(full_run, oracle):
    """200 lanes drawn across the whole sweep, each re-run by the oracle from
    the same (seed, id).  Outcome classes of lanes that reached a product
    (both sides stopped by r_stop) agree for >= 99 %; lanes still inside a
    complex at t_max are a snapshot of a chaotic orbit and are reported
    separately.  Energy conservation matches the oracle's lane by lane."""
    wl, out, hist, cells, groups = full_run
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(wl.n, 200, replace=False))
    systems = [oracle.system_from_spec(s) for s in wl.systems]
    integ = oracle.make_integ(**wl.integ)
    rows = []
    for i in idx:
        st, res = oracle.run_lanes(systems, wl.sys_id[i:i + 1], wl.E[i:i + 1], wl.b[i:i + 1],
                                   wl.v[i:i + 1], wl.j[i:i + 1], wl.R0, wl.seed, integ,
                                   id_offset=int(i))
        r = res[0]
        rows.append((i, wl.E[i], wl.b[i], out["status"][i], out["cls"][i], out["nsteps"][i],
                     r["status"], r["cls"], r["nsteps"], out["dE"][i], r["dE"], st["E0"][0]))
    rows = np.array(rows, dtype=object)
    done = np.array([(r[3] == 2 and r[6] == 2) for r in rows])
    agree = np.array([r[4] == r[7] for r in rows])
    for r in rows[~agree]:
        print("mismatch lane %d E=%.4f b=%.2f gpu(st=%d cls=%d n=%d) oracle(st=%d cls=%d n=%d)"
              % tuple(r[:9]))
    print(f"\nsampled: {agree.mean():.3f} agree overall; {agree[done].mean():.4f} of "
          f"{done.sum()} lanes that reached a product; {(~done).sum()} at t_max")
    assert agree[done].mean() >= 0.99
    # energy conservation: the same order as the oracle's on every lane
    e_g = np.array([abs(r[9]) for r in rows]) / np.array([max(abs(r[11]), r[1]) for r in rows])
    e_o = np.array([abs(r[10]) for r in rows]) / np.array([max(abs(r[11]), r[1]) for r in rows])
    assert np.all(e_g <= np.maximum(10 * e_o, 1e-9))
    assert np.median(e_g) < 1e-8


def test_full_size_invariants(full_run, oracle):
    wl, out, hist, cells, groups = full_run
    n = wl.n
    assert np.all(np.isin(out["status"], [2, 3]))              # no failed lane
    sep = out["status"] == 2
    rel = np.abs(out["dE"][sep]) / np.maximum(np.abs(out["E0"][sep]), wl.E[sep])
    print(f"\n|dE|/max(|E0|,Ecol) over {sep.sum()} separated lanes: median {np.median(rel):.2e}"
          f", 99% {np.quantile(rel, 0.99):.2e}, max {rel.max():.2e}")
    # the drift grows with trajectory length (the oracle's does too, lane by
    # lane: see the sampled test); the 1e-8 bar is pinned on the plain study
    assert np.median(rel) < 1e-8 and rel.max() < 1e-6
    assert hist[:, 6].sum() == n and hist[:, :6].sum() == n
    # histograms are those of the per-lane outcomes (bit-exact)
    ho = oracle.reduce(out["cls"], out["vt"], out["jt"], out["gbw"], wl.cell, wl.n_cells)
    assert np.array_equal(hist, ho)
    # A = B (H2): the two reactive arrangements have equal cross sections
    for g in range(wl.n_groups):
        s1, e1 = groups[g, 1]
        s2, e2 = groups[g, 2]
        assert abs(s1 - s2) <= 4.0 * math.hypot(e1, e2) + 1e-12, (g, s1, s2, e1, e2)


def _oracle_chunk(payload):
    import oracle as O
    specs, sid, E, b, v, j, R0, seed, ids, integ_kw = payload
    systems = [O.system_from_spec(sp) for sp in specs]
    integ = O.make_integ(**integ_kw)
    out = np.zeros((len(E), 5), np.int32)    # cls, v_t, j_t, status, accepted steps
    for k in range(len(E)):
        _, res = O.run_lanes(systems, sid[k:k + 1], E[k:k + 1], b[k:k + 1], v[k:k + 1],
                             j[k:k + 1], R0, seed, integ, id_offset=int(ids[k]))
        out[k] = (res["cls"][0], res["vt"][0], res["jt"][0], res["status"][0],
                  res["nsteps"][0])
    return out


@pytest.fixture(scope="module")
def oracle_sample(full_run, oracle):
    """The oracle's outcomes (class, v_t, j_t, status, steps) for 16 lanes per
    (E, b) cell of the sweep (6,144 trajectories run one by one, one oracle
    process per host core)."""
    import multiprocessing as mp
    import os
    wl = full_run[0]
    idx = W.stratified(wl, 16)
    cores = max(1, min(os.cpu_count() or 1, 32))
    parts = [c for c in np.array_split(np.arange(len(idx)), cores) if len(c)]
    payloads = [(wl.systems, wl.sys_id[idx[c]], wl.E[idx[c]], wl.b[idx[c]], wl.v[idx[c]],
                 wl.j[idx[c]], wl.R0, wl.seed, idx[c], dict(wl.integ)) for c in parts]
    with mp.get_context("spawn").Pool(len(payloads)) as pool:
        res = np.concatenate(pool.map(_oracle_chunk, payloads))
    return idx, res


def _within_3se(wl, groups, idx, res, oracle):
    cls_o = res[:, 0]
    zeros = np.zeros(len(idx), np.int32)
    h_o = oracle.reduce(cls_o, zeros, zeros, np.zeros(len(idx)), wl.cell[idx], wl.n_cells)
    _, g_o = oracle.xsec(h_o, wl.cell_b, wl.cell_w, wl.cell_group, wl.n_groups)
    # a count of 0 or N has a zero binomial error; bound the sample's error
    # with the count clipped to [1, N - 1]
    N = h_o[:, :5].sum(axis=1).astype(float)
    wb = wl.cell_w * wl.cell_b
    worst = 0.0
    for g in range(wl.n_groups):
        cg = wl.cell_group == g
        for k in range(4):            # Q, R_AC, R_BC, D
            p = np.clip(h_o[cg, k], 1, N[cg] - 1) / N[cg]
            se_o = 2 * math.pi * math.sqrt(np.sum(wb[cg] ** 2 * p * (1 - p) / N[cg]))
            d = abs(groups[g, k, 0] - g_o[g, k, 0])
            se = math.hypot(groups[g, k, 1], max(g_o[g, k, 1], se_o))
            worst = max(worst, d / se)
            assert d <= 3.0 * se, (g, k, groups[g, k], g_o[g, k])
    return worst


def test_full_size_cross_sections_within_3se_of_oracle(full_run, oracle_sample, oracle):
    """Every cross section of the full GPU sweep lies within 3 combined
    standard errors of the oracle's estimate from the sampled lanes."""
    wl, out, hist, cells, groups = full_run
    worst = _within_3se(wl, groups, *oracle_sample, oracle)
    print(f"\nlargest |sigma_gpu - sigma_oracle| / SE over 16 energies x 4 channels: {worst:.2f}")


def test_full_size_product_states_match_oracle(full_run, oracle_sample):
    """Product analysis at full size (v' from the action integral, j' from
    L^2).  Lane by lane on the 6,144 oracle lanes that reached the same
    product by r_stop on both sides: where the two trajectories stayed
    together (accepted step counts within 2 %), the integer bins (v_t, j_t)
    agree for >= 99.5 % (a bin flips only when v' or j' lies within the
    rounding-level difference of a half-integer); over all of them, which
    include chaotic complexes that separate long before the end, for
    >= 95 %.  As distributions: in each quarter of the energy range, the
    oracle sample's quench v_t and j_t histograms are consistent
    (chi-square, p > 1e-4) with the full GPU sweep's."""
    from scipy import stats
    wl, out, hist, cells, groups = full_run
    idx, res = oracle_sample
    cls_o, vt_o, jt_o, st_o, ns_o = res.T
    same = (out["status"][idx] == 2) & (st_o == 2) & (out["cls"][idx] == cls_o) & (cls_o <= 2)
    bins = (out["vt"][idx] == vt_o) & (out["jt"][idx] == jt_o)
    ns_g = out["nsteps"][idx].astype(float)
    close = same & (np.abs(ns_g - ns_o) <= 0.02 * ns_o)
    agree_all, agree_close = np.mean(bins[same]), np.mean(bins[close])
    print(f"\n(v_t, j_t) agreement: {agree_close:.4f} on {close.sum()} lanes whose trajectories "
          f"stayed together, {agree_all:.4f} on all {same.sum()} product lanes")
    assert same.sum() > 4500 and close.sum() > 0.8 * same.sum()
    assert agree_close >= 0.995 and agree_all >= 0.95
    e_idx = wl.cell // 24                       # energy index of each lane (24 b per energy)
    worst = 1.0
    for band in range(4):
        g_sel = (e_idx // 4 == band) & (out["cls"] == 0) & (out["status"] == 2)
        o_sel = (e_idx[idx] // 4 == band) & (cls_o == 0) & (st_o == 2)
        for gv, ov in ((out["vt"][g_sel], vt_o[o_sel]), (out["jt"][g_sel], jt_o[o_sel])):
            top = int(max(gv.max(), ov.max())) + 1
            pg = np.bincount(gv, minlength=top) / len(gv)
            co = np.bincount(ov, minlength=top).astype(float)
            exp = pg * len(ov)
            keep = exp >= 5                     # pool the sparse bins into one
            obs_b = np.r_[co[keep], co[~keep].sum()]
            exp_b = np.r_[exp[keep], exp[~keep].sum()]
            if exp_b[-1] < 5:
                obs_b, exp_b = obs_b[:-1], exp_b[:-1]
                exp_b *= obs_b.sum() / exp_b.sum()
            chi2 = np.sum((obs_b - exp_b) ** 2 / exp_b)
            p = stats.chi2.sf(chi2, len(obs_b) - 1)
            worst = min(worst, p)
            assert p > 1e-4, (band, chi2, len(obs_b))
    print(f"smallest chi-square p-value over 4 energy bands x (v_t, j_t): {worst:.3g}")


def test_fp32_full_size_against_fp64_oracle(full_run, oracle_sample, oracle):
    """The FP32 integrator with compensated updates (tolerances 1e-6 / 1e-8)
    on the same 3,145,728 trajectories: every cross section within 3 combined
    standard errors of the FP64 oracle's; energy drift and class agreement
    with the FP64 run are reported."""
    import torch
    from paper_2304_02731_gb300 import qcams as Q
    wl = full_run[0]
    integ = Q.make_integ(**W.INTEG_FP32, persistent=True, precision=32)
    b32, hist32, cells32, groups32 = Q.run_workload(wl, integ)
    torch.cuda.synchronize()
    st = Q.last_run_stats()
    worst = _within_3se(wl, groups32, *oracle_sample, oracle)
    cls32, status32 = b32.cls.cpu().numpy(), b32.status.cpu().numpy()
    dE, E0 = b32.f64["dE"].cpu().numpy(), b32.f64["E0"].cpu().numpy()
    sep = status32 == 2
    rel = np.abs(dE[sep]) / np.maximum(np.abs(E0[sep]), wl.E[sep])
    out64 = full_run[1]
    done = sep & (out64["status"] == 2)
    agree = np.mean(cls32[done] == out64["cls"][done])
    print(f"\nFP32: worst sigma deviation {worst:.2f} SE; |dE/E| median {np.median(rel):.2e} "
          f"99% {np.quantile(rel, .99):.2e}; class agreement with FP64 {agree:.4f} over "
          f"{done.sum()} lanes; integrator {st['integrate_ms']:.1f} ms")
    assert np.all(np.isin(status32, [2, 3]))
    assert agree > 0.99 and np.median(rel) < 1e-5
