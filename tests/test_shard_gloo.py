"""Sharding over ranks (CPU, gloo): the same global trajectory ids split over
1, 2 or 4 ranks give bit-identical merged histograms (per-cell records in
the library's layout, QCAMS_H_STRIDE int64 per cell) and, through the
library's host entry point qcams_xsec_from_hist, bit-identical cross
sections; a rank that dies before the merge makes the survivors' collective
fail within the timeout instead of hanging."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2304_02731_gb300 import workloads as W
from paper_2304_02731_gb300.shard import shard_range


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, per_b, out_q, die_rank):
    import torch
    import oracle as O
    from paper_2304_02731_gb300 import shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    shard.init_process_group("gloo", timeout_s=8.0)
    wl = W.plain_h2_ca(per_b=per_b)
    lo, hi = shard.shard_range(wl.n, rank, world)
    part = wl.slice(lo, hi)
    s = O.system_from_spec(wl.systems[0])
    integ = O.make_integ(**dict(wl.integ, t_stop=1000.0))
    st, res = O.run_lanes([s], part.sys_id, part.E, part.b, part.v, part.j, part.R0, part.seed,
                          integ, id_offset=part.id_offset)
    h = O.reduce(res["cls"], res["vt"], res["jt"], res["gbw"], part.cell, wl.n_cells)
    t = torch.from_numpy(h.reshape(-1).copy())
    if rank == die_rank:
        os._exit(3)                      # this rank dies before the merge
    try:
        shard.merge_histograms(t)
        from paper_2304_02731_gb300 import qcams as Q
        assert O.H_STRIDE == Q.H_STRIDE
        cells, groups = Q.xsec_from_hist(t.numpy(), wl.cell_b, wl.cell_w, wl.cell_group,
                                         wl.n_groups)
        out_q.put((rank, "ok", (t.numpy().copy(), cells.copy(), groups.copy())))
    except Exception as e:              # the collective reports the dead peer
        out_q.put((rank, "error", type(e).__name__))
    finally:
        try:
            torch.distributed.destroy_process_group()
        except Exception:
            pass


def _run(world, per_b, die_rank=-1, timeout=120):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, per_b, q, die_rank))
             for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    expect = world - (1 if die_rank >= 0 else 0)
    for _ in range(expect):
        r, status, payload = q.get(timeout=timeout)
        out[r] = (status, payload)
    for p in procs:
        p.join(timeout=30)
        if p.is_alive():
            p.kill()
    return out


def test_shard_range_partitions():
    for n in (0, 1, 7, 1000, 1001):
        for world in (1, 2, 3, 4, 8):
            parts = [shard_range(n, r, world) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[k][1] == parts[k + 1][0] for k in range(world - 1))
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)


@pytest.mark.parametrize("world", [2, 4])
def test_sharded_histograms_are_bit_identical(oracle, world):
    per_b = 4
    ref = _run(1, per_b)[0]
    got = _run(world, per_b)
    assert ref[0] == "ok"
    for r in range(world):
        assert got[r][0] == "ok"
        for a, b in zip(got[r][1], ref[1]):      # histograms, per-cell and per-group xsec
            assert np.array_equal(a, b)
    # sigma_Q of the plain study: every separated lane is a quench
    assert ref[1][2][0, 0, 0] > 0


def test_dead_rank_fails_the_merge_instead_of_hanging(oracle):
    got = _run(2, 2, die_rank=1, timeout=90)
    assert got[0][0] == "error"
