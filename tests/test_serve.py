"""Serving loop: admission under an HBM budget, concurrency, and results that
do not depend on what a request is served with.

The CPU tests cover the host side (the library's byte estimate, budget
accounting); the GPU tests run the scheduler on small requests."""

import numpy as np
import pytest

import hevi_inputs
import oracle
from oracle import tableaux


def _requests(count=6, seed=5, cols=(40, 160), steps=(1, 3)):
    from paper_2311_11425_gb300.serve import Request
    raw = hevi_inputs.serve_requests(seed=seed, count=count, rate=200.0, cols_range=cols,
                                     steps_range=steps)
    return [Request(**r) for r in raw]


def test_estimate_bytes_host_only():
    import paper_2311_11425_gb300 as hv
    base = hv.hevi_estimate_bytes([(10, 4)], ncols=1000)
    more = hv.hevi_estimate_bytes([(10, 4)], ncols=2000)
    assert 0 < base < more
    lh = hv.hevi_estimate_bytes([(10, 4)], ncols=1000, kind=hv.LHEVI, stages=4)
    nh = hv.hevi_estimate_bytes([(10, 4)], ncols=1000, kind=hv.NHEVI, stages=4)
    n = 1000 * 123
    assert lh - base == 9 * n * 8          # 2s + 1 vectors: stages, tendencies, rhs
    assert nh - base > 6 * n * 8           # s + 2 vectors, the linearisation, U scratch
    fp64 = hv.hevi_estimate_bytes([(10, 4)], ncols=1000, precision=hv.FP64)
    assert fp64 > base                     # FP64 factors are twice as large
    mixed = hv.hevi_estimate_bytes([(8, 4), (16, 3)], class_of_col=[0, 1, 1, 0], ncols=4)
    assert mixed > 0
    with pytest.raises(hv.HeviError):
        hv.hevi_estimate_bytes([(10, 9)], ncols=10)
    with pytest.raises(hv.HeviError):
        hv.hevi_estimate_bytes([(10, 4)], ncols=10, kind=3)
    with pytest.raises(hv.HeviError):
        hv.hevi_estimate_bytes([(10, 4), (8, 4)], class_of_col=[0, 2], ncols=2)


def test_granule_allocator_matches_a_bitmap_model():
    """First fit over random alloc / release sequences, against a plain
    bitmap of the granules."""
    from paper_2311_11425_gb300.serve import GranuleAllocator
    g = np.random.default_rng(11)
    count = 64
    a = GranuleAllocator(count)
    used = np.zeros(count, bool)
    live = []
    for _ in range(3000):
        if live and g.random() < 0.45:
            s, n = live.pop(int(g.integers(len(live))))
            a.release(s, n)
            assert used[s:s + n].all()
            used[s:s + n] = False
        else:
            n = int(g.integers(1, 12))
            s = a.alloc(n)
            # the model: the lowest start of n free granules in a row
            runs = [k for k in range(count - n + 1) if not used[k:k + n].any()]
            assert s == (runs[0] if runs else None)
            if s is not None:
                used[s:s + n] = True
                live.append((s, n))
        assert a.free_granules == int((~used).sum())
        # free runs are disjoint, sorted and merged
        for (s0, n0), (s1, n1) in zip(a.free, a.free[1:]):
            assert s0 + n0 < s1
    with pytest.raises(AssertionError):
        a.release(*a.free[0])  # a free run cannot be released again
    # split allocation: the lowest free granules, in runs, or nothing
    b = GranuleAllocator(16)
    x, y, z = b.alloc(4), b.alloc(4), b.alloc(4)
    b.release(x, 4)
    b.release(z, 4)
    assert b.alloc_split(9) == [(0, 4), (8, 5)]  # (8, 4) merged with the free tail
    assert b.alloc_split(4) is None and b.free == [(13, 3)]


def test_pool_bytes_and_budget_check():
    from paper_2311_11425_gb300.serve import GRANULE, Server, pool_bytes
    import paper_2311_11425_gb300 as hv
    classes = [(8, 4), (16, 3)]
    pb = pool_bytes(classes, [40, 70], "LHEVI", hv.FP32_IR, 4)
    cap = [64, 96]  # rounded up to granules of 32
    assert all(c % GRANULE == 0 for c in cap)
    cls = np.repeat([0, 1], cap).astype(np.int32)
    n = cap[0] * 99 + cap[1] * 147
    assert pb == hv.hevi_estimate_bytes(classes, cls, sum(cap), hv.FP32_IR, hv.LHEVI, 4) + 3 * n * 8
    assert pool_bytes(classes, 64, "NHEVI") > pool_bytes(classes, 64, "LHEVI") - 1
    # the pools must fit the budget: checked before anything touches the device
    with pytest.raises(ValueError):
        Server(classes, slots_per_class=1 << 20, hbm_budget=1 << 30)


def test_request_blocks_regroup_columns_by_class():
    from paper_2311_11425_gb300.serve import Request
    classes = [(2, 1), (2, 2)]  # n = 9 and 15
    cls = np.array([1, 0, 1, 1, 0], np.int32)
    n_of = np.array([9, 15])[cls]
    H = np.arange(n_of.sum(), dtype=float)
    dq = -H
    r = Request(rid=0, classes=classes, class_of_col=cls, ztop=np.arange(5) + 30e3, steps=1,
                variant="NHEVI", H=H, dq=dq)
    blocks = r.as_blocks()
    assert [tuple(b.cls) for b, _ in blocks] == classes
    (b0, c0), (b1, c1) = blocks
    assert list(c0) == [1, 4] and list(c1) == [0, 2, 3]
    off = np.concatenate([[0], np.cumsum(n_of)])
    assert np.array_equal(b0.H, np.concatenate([H[off[1]:off[2]], H[off[4]:off[5]]]))
    assert np.array_equal(b1.dq, -np.concatenate([H[off[0]:off[1]], H[off[2]:off[4]]]))
    assert np.array_equal(b1.ztop, [30e3, 30e3 + 2, 30e3 + 3])
    assert r.ncols == 5


# ---------------------------------------------------------------------------
# GPU
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def hv():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2311_11425_gb300 as hv
    hv.load(build=True)
    return hv


@pytest.mark.gpu
def test_estimate_equals_device_bytes(hv):
    import torch
    classes = hevi_inputs.SIZE_CLASSES
    g = np.random.default_rng(3)
    cls = g.integers(0, 4, 300).astype(np.int32)
    zt = g.uniform(30e3, 100e3, 300)
    for prec, kind in ((hv.FP32_IR, hv.LHEVI), (hv.FP64, hv.LHEVI), (hv.FP32_IR, hv.NHEVI)):
        ctx = hv.Context(classes, zt, class_of_col=cls, precision=prec)
        assert ctx.device_bytes == hv.hevi_estimate_bytes(classes, cls, 300, prec, 0, 3)
        q = ctx.hevi_reference_state()
        H = torch.zeros_like(q)
        if kind == hv.LHEVI:
            ctx.hevi_lhevi_step(hv.tableau("ARK3"), 300.0, q, H)
        else:
            ctx.hevi_nhevi_step(hv.tableau("ARK3"), 300.0, q, H)
        ctx.hevi_sync()
        assert ctx.device_bytes == hv.hevi_estimate_bytes(classes, cls, 300, prec, kind, 4)
        ctx.close()


def _alone(hv, r, tab, dt=300.0, rtol=1e-10, max_iter=20):
    """The request's columns stepped in a context of their own."""
    import torch
    ctx = hv.Context(r.classes, r.ztop, class_of_col=r.class_of_col, precision=hv.FP32_IR)
    q = ctx.hevi_reference_state()
    if r.dq is not None:
        q += torch.from_numpy(np.asarray(r.dq, dtype=np.float64)).cuda()
    H = torch.from_numpy(np.asarray(r.H, dtype=np.float64)).cuda()
    b = ctx.empty()
    for _ in range(r.steps):
        if r.variant == "LHEVI":
            ctx.hevi_lhevi_step(tab, dt, q, H, b)
        else:
            ctx.hevi_nhevi_step(tab, dt, q, H, b, rtol=rtol, max_iter=max_iter)
        q, b = b, q
    ctx.hevi_sync()
    out = q.cpu().numpy()
    ctx.close()
    return out


@pytest.mark.gpu
def test_same_result_alone_and_in_mix(hv):
    """Small pools (3 granules per class) force queueing, slot reuse and
    runs at different positions; every request matches its own columns run
    alone, bit for bit."""
    from paper_2311_11425_gb300.serve import Server
    reqs = _requests(count=8, cols=(20, 90), steps=(1, 3))
    assert {r.variant for r in reqs} == {"LHEVI", "NHEVI"}
    server = Server(hevi_inputs.SIZE_CLASSES, slots_per_class=96, hbm_budget=40 << 30)
    mix = server.run(reqs, realtime=False)
    assert all(r.error is None for r in mix), [(r.rid, r.error) for r in mix]
    assert all(p.ticks > 0 for p in server.pools.values())
    tab = hv.tableau("ARK3")
    for r, m in zip(reqs, mix):
        np.testing.assert_array_equal(_alone(hv, r, tab), m.q)
    # every slot is back at rest with zero tendency (idle slots step from
    # rest to rest up to the rounding of the refined solves)
    import torch
    for p in server.pools.values():
        assert not p.placed and all(a.free_granules == a.count for a in p.alloc)
        assert float(p.H.abs().max()) == 0.0
        ref = p.ctx.hevi_reference_state()
        assert torch.allclose(p.q[p.cur], ref, rtol=1e-9, atol=1e-9)
    server.close()


@pytest.mark.gpu
def test_admission_rejection_and_time_limit(hv):
    from paper_2311_11425_gb300.serve import Request, Server
    reqs = _requests(count=6, seed=6, cols=(30, 60), steps=(1, 2))
    server = Server(hevi_inputs.SIZE_CLASSES, slots_per_class=64, hbm_budget=40 << 30,
                    variants=("LHEVI", "NHEVI"))
    # a class the pools do not hold, and more columns of a class than a pool holds
    bad = [Request(rid=100, classes=[(5, 2)], ztop=np.full(4, 30e3), steps=1, variant="LHEVI",
                   H=np.zeros(4 * 33)),
           Request(rid=101, classes=[(8, 4)], ztop=np.full(70, 30e3), steps=1, variant="LHEVI",
                   H=np.zeros(70 * 99))]
    res = server.run(reqs + bad, realtime=False)
    assert all(r.error is None for r in res[:6]), [(r.rid, r.error) for r in res]
    assert "not served" in res[6].error and "more columns" in res[7].error
    # admission in arrival order within a variant
    for v in ("LHEVI", "NHEVI"):
        sub = sorted((r for r in res[:6] if r.variant == v), key=lambda r: r.arrival)
        assert [r.admitted for r in sub] == sorted(r.admitted for r in sub)
    # a time limit reports what was not admitted and finishes the rest
    res2 = server.run(reqs, realtime=True, time_limit=0.0)
    assert all(r.error in (None, "not admitted within the time limit") for r in res2)
    server.close()


@pytest.mark.gpu
def test_served_lhevi_matches_oracle(hv):
    from paper_2311_11425_gb300.serve import Request, Server
    nez, N, ncols = 8, 4, 30
    inp = hevi_inputs.lhevi_ark3(seed=2, ncols=ncols, nez=nez, N=N)
    r = Request(rid=0, classes=[(nez, N)], class_of_col=None,
                ztop=np.broadcast_to(np.asarray(inp["ztop"], dtype=float), (ncols,)).copy(),
                steps=2, variant="LHEVI", H=inp["H"].reshape(-1))
    server = Server([(nez, N)], slots_per_class=64, hbm_budget=8 << 30, variants=("LHEVI",))
    res = server.run([r], realtime=False)[0]
    server.close()
    assert res.error is None
    q = oracle.reference_q(nez, N, inp["ztop"], ncols)
    q0 = q.copy()
    for _ in range(2):
        q, info = oracle.lhevi_step(nez, N, inp["ztop"], tableaux.ALL["ARK3"], inp["dt"], q,
                                    inp["H"], lin=0)
        assert (info == 0).all()
    got = res.q.reshape(ncols, -1)
    # the state at 1e-10; the increment (from rest, ~1e-4 of the state) at
    # 1e-10 times the acoustic Courant number c_s dt / dz_min, the factor by
    # which the explicit S(Q_i) = H + V(Q_i) carries stage-value errors into it
    err_state = np.linalg.norm(got - q, axis=1) / np.linalg.norm(q, axis=1)
    assert err_state.max() < 1e-10, err_state.max()
    cs = np.sqrt(1004.67 / (1004.67 - 287.17) * 287.17 * 300.0)
    zt0 = float(np.atleast_1d(inp["ztop"])[0])
    courant = cs * inp["dt"] / np.diff(oracle.column_grid(nez, N, zt0)[0]).min()
    err = np.linalg.norm(got - q, axis=1) / np.linalg.norm(q - q0, axis=1)
    assert err.max() < 1e-10 * courant, (err.max(), courant)


@pytest.mark.gpu
def test_realtime_latency_stats(hv):
    from paper_2311_11425_gb300.serve import Server, latency_stats
    reqs = _requests(count=8, seed=7)
    server = Server(hevi_inputs.SIZE_CLASSES, slots_per_class=256, hbm_budget=40 << 30,
                    keep_state=False)
    res = server.run(reqs, realtime=True)
    st = latency_stats(res)
    assert st["served"] == 8 and st["not_served"] == 0
    assert 0 < st["p50_s"] <= st["p99_s"] <= st["max_s"]
    for r in res:
        assert r.done >= r.admitted >= r.arrival - 1e-9 and r.q is None
    s = server.stats
    assert 0.0 < s["gpu_busy_fraction"] <= 1.0
    assert sum(v["request_column_steps"] for v in s["variants"].values()) == \
        sum(r.ncols * r.steps for r in reqs)
    server.close()


def test_serve_stream_per_request_seeds_and_bank_windows():
    """The long stream draws each request from its own seed: a request does not
    depend on how many requests the stream has, and its class windows stay
    inside the banks; the arrivals are a Poisson process of the given rate."""
    s1 = hevi_inputs.serve_stream(seed=5, count=40, rate=50.0, bank_cols=32768)
    s2 = hevi_inputs.serve_stream(seed=5, count=400, rate=50.0, bank_cols=32768)
    for a, b in zip(s1, s2):
        assert a == b
    gaps = np.diff([0.0] + [r["arrival"] for r in s2])
    assert abs(gaps.mean() - 1 / 50.0) < 0.2 / 50.0  # mean inter-arrival 1 / rate
    for r in s2:
        total = sum(m for _, _, m in r["parts"])
        assert 2000 <= total <= 86402 and 1 <= r["steps"] <= 20
        assert r["variant"] in ("LHEVI", "NHEVI")
        for c, start, m in r["parts"]:
            assert 0 <= c < 4 and 0 <= start and start + m <= 32768
    bank = hevi_inputs.serve_bank(seed=6, cols_per_class=64)
    for b, (nez, N) in zip(bank, hevi_inputs.SIZE_CLASSES):
        n = 3 * (nez * N + 1)
        assert b["H"].shape == (64, n) and b["dq"].shape == (64, n) and b["ztop"].shape == (64,)
        assert (b["ztop"] >= 30e3).all() and (b["ztop"] <= 100e3).all()
