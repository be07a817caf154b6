"""Column sharding across ranks (no data-path collective).

Host logic of the multi-GPU path: the partition itself, and a world-size-2
gloo run in which every rank solves only its shard of a mixed-class grid with
the FP64 oracle; the shards gathered on rank 0 must equal the single-process
solve bit for bit, since columns are independent (Sec. 3, Sec. 4.3).
"""

import os
import socket

import numpy as np
import pytest

import hevi_inputs
from paper_2311_11425_gb300.shard import column_shards, column_work, shard_of


def test_uniform_shards_cover_and_balance():
    for ncols in (0, 1, 7, 32, 86402):
        for world in (1, 2, 3, 8):
            sh = column_shards(ncols, world)
            assert len(sh) == world
            assert sh[0][0] == 0 and sh[-1][1] == ncols
            for (a, b), (c, _) in zip(sh, sh[1:]):
                assert b == c and a <= b
            lens = [b - a for a, b in sh]
            assert max(lens) - min(lens) <= 1


def test_weighted_shards_bound():
    g = hevi_inputs.rng(11)
    classes = [(8, 4), (10, 4), (16, 3), (24, 4)]
    cls = g.integers(0, len(classes), 5000)
    w = column_work(cls, classes)
    for world in (2, 3, 4, 8):
        sh = column_shards(len(w), world, w)
        assert sh[0][0] == 0 and sh[-1][1] == len(w)
        tot = w.sum()
        for a, b in sh:
            assert w[a:b].sum() < tot / world + w.max()
        # the greedy bound is not vacuous: the shards are close to even
        loads = np.array([w[a:b].sum() for a, b in sh])
        assert loads.max() / loads.mean() < 1.01


def test_column_work_is_band_size():
    # (10, 4): n = 123, k = 14, ldab = 43
    assert column_work([0], [(10, 4)])[0] == 43 * 123
    # (16, 3): n = 147, k = 11, ldab = 34
    assert column_work([0], [(16, 3)])[0] == 34 * 147


def test_shard_edge_cases():
    assert column_shards(3, 5) == [(0, 0), (0, 1), (1, 1), (1, 2), (2, 3)]
    assert column_shards(4, 2, np.zeros(4)) == [(0, 2), (2, 4)]
    with pytest.raises(ValueError):
        column_shards(4, 0)
    with pytest.raises(ValueError):
        column_shards(4, 2, [1.0, 2.0])
    with pytest.raises(ValueError):
        column_shards(2, 2, [1.0, -1.0])
    with pytest.raises(ValueError):
        shard_of(4, 2, 2)


# ---------------------------------------------------------------------------
# world-size-2 gloo run
# ---------------------------------------------------------------------------

CLASSES = [(2, 4), (3, 3), (4, 2)]
LAM = 87.868


def _problem():
    g = hevi_inputs.rng(21)
    ncols = 37
    cls = g.integers(0, len(CLASSES), ncols)
    ztop = g.uniform(20e3, 60e3, ncols)
    bs = []
    for c in range(ncols):
        nez, N = CLASSES[cls[c]]
        n = 3 * (nez * N + 1)
        bs.append(g.standard_normal(n))
    return cls, ztop, bs


def _solve_columns(cols, cls, ztop, bs):
    import oracle
    out = {}
    for c_id, (nez, N) in enumerate(CLASSES):
        idx = [c for c in cols if cls[c] == c_id]
        if not idx:
            continue
        q0 = oracle.reference_q(nez, N, ztop[idx], len(idx))
        b = np.stack([bs[c] for c in idx])
        x, info = oracle.stage_solve(nez, N, ztop[idx], LAM, q0, b)
        assert (info == 0).all()
        for k, c in enumerate(idx):
            out[c] = x[k]
    return out


def _rank_main(rank, world, port):
    import time
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cls, ztop, bs = _problem()
        w = column_work(cls, CLASSES)
        a, b = shard_of(len(cls), rank, world, w)
        t0 = time.perf_counter()
        mine = _solve_columns(range(a, b), cls, ztop, bs)
        el = time.perf_counter() - t0
        gathered = [None] * world
        dist.all_gather_object(gathered, (a, b, mine))
        t = torch.tensor([el], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        els = [None] * world
        dist.all_gather_object(els, el)
        if rank == 0:
            assert t.item() == max(els)
            # shards tile [0, ncols) and every column is solved exactly once
            spans = sorted((s, e) for s, e, _ in gathered)
            assert spans[0][0] == 0 and spans[-1][1] == len(cls)
            assert all(e0 == s1 for (_, e0), (s1, _) in zip(spans, spans[1:]))
            merged = {}
            for _, _, part in gathered:
                assert not set(part) & set(merged)
                merged.update(part)
            serial = _solve_columns(range(len(cls)), cls, ztop, bs)
            assert sorted(merged) == sorted(serial)
            for c in serial:
                np.testing.assert_array_equal(merged[c], serial[c])
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_gloo_two_ranks_shard_solve_matches_serial():
    import oracle
    import torch.multiprocessing as mp
    oracle.build()  # once, before the ranks start
    mp.spawn(_rank_main, args=(2, _free_port()), nprocs=2, join=True)
