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


def test_request_bytes_counts_state_buffers():
    from paper_2311_11425_gb300.serve import Server
    import paper_2311_11425_gb300 as hv
    s = Server(hbm_budget=1 << 30)
    r = _requests(count=1)[0]
    kind = hv.LHEVI if r.variant == "LHEVI" else hv.NHEVI
    lib = hv.hevi_estimate_bytes(r.classes, r.class_of_col, r.ncols, hv.FP32_IR, kind, 4)
    assert s.request_bytes(r) == lib + 3 * r.H.size * 8


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


@pytest.mark.gpu
def test_same_result_alone_and_in_mix(hv):
    from paper_2311_11425_gb300.serve import Server
    reqs = _requests(count=6)
    assert {r.variant for r in reqs} == {"LHEVI", "NHEVI"}
    server = Server(hbm_budget=40 << 30)
    mix = server.run(reqs, realtime=False)
    assert all(r.error is None for r in mix), [(r.rid, r.error) for r in mix]
    for k in (1, 4):
        alone = Server(hbm_budget=40 << 30).run([reqs[k]], realtime=False)[0]
        assert alone.error is None
        np.testing.assert_array_equal(alone.q, mix[k].q)


@pytest.mark.gpu
def test_budget_admission_and_rejection(hv):
    from paper_2311_11425_gb300.serve import Server
    reqs = _requests(count=5, seed=6)
    s0 = Server(hbm_budget=1 << 40)
    sizes = [s0.request_bytes(r) for r in reqs]
    # room for the largest request alone: requests are served one after another
    server = Server(hbm_budget=max(sizes))
    res = server.run(reqs, realtime=False)
    assert all(r.error is None for r in res), [(r.rid, r.error) for r in res]
    assert server.peak_bytes <= max(sizes)
    # admission is first come, first served
    order = sorted(range(len(reqs)), key=lambda i: reqs[i].arrival)
    adm = [res[i].admitted for i in order]
    assert adm == sorted(adm)
    # a budget below one request rejects that request and serves the rest
    small = sorted(sizes)[1]
    res2 = Server(hbm_budget=small).run(reqs, realtime=False)
    for r, b in zip(res2, sizes):
        assert (r.error is None) == (b <= small), (r.rid, r.error, b, small)


@pytest.mark.gpu
def test_served_lhevi_matches_oracle(hv):
    from paper_2311_11425_gb300.serve import Request, Server
    nez, N, ncols = 8, 4, 30
    inp = hevi_inputs.lhevi_ark3(seed=2, ncols=ncols, nez=nez, N=N)
    r = Request(rid=0, classes=[(nez, N)], class_of_col=None,
                ztop=np.broadcast_to(np.asarray(inp["ztop"], dtype=float), (ncols,)).copy(),
                steps=2, variant="LHEVI", H=inp["H"].reshape(-1))
    res = Server(hbm_budget=8 << 30).run([r], realtime=False)[0]
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
    res = Server(hbm_budget=40 << 30).run(reqs, realtime=True)
    st = latency_stats(res)
    assert st["served"] == 8 and st["rejected"] == 0
    assert 0 < st["p50_s"] <= st["p99_s"] <= st["max_s"]
    for r in res:
        assert r.done >= r.admitted >= r.arrival - 1e-9
