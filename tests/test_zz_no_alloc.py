"""The Newton solve for callers that cannot allocate device memory.

hevi_newton_solve_noalloc serves code that must not call cudaMalloc -- code
running inside another framework's memory pool or under its allocator lock,
or a plugin that may not touch the device heap.  It keeps all of its scratch
in a fixed device array of the library.  These tests call it through the C
ABI and check it against the context-based hevi_newton_solve on the same
inputs, twice in a row (the array keeps the previous call's contents), and
check that an oversized request is refused.  The file is named so that pytest
collects it last."""

import numpy as np
import pytest

import hevi_inputs

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def hv():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2311_11425_gb300 as hv
    hv.load(build=True)
    return hv


def _rel_cols(x, ref):
    num = np.linalg.norm(x - ref, axis=1)
    den = np.linalg.norm(ref, axis=1)
    return num / np.where(den == 0, 1.0, den)


@pytest.mark.parametrize("nez,N,ncols", [(16, 3, 301), (10, 4, 97)])
def test_noalloc_newton_matches_context_newton_twice(hv, nez, N, ncols):
    import torch
    inp = hevi_inputs.nhevi_ark2(seed=3, nez=nez, N=N, ncols=ncols)
    ctx = hv.Context([(nez, N)], inp["ztop"], precision=hv.FP32_IR)
    q_init = ctx.hevi_reference_state() + torch.from_numpy(inp["dq"].reshape(-1)).cuda()
    R = q_init + 0.01 * (q_init - ctx.hevi_reference_state())
    lam = (1 - 2 ** -0.5) * inp["dt"]
    q_ref = q_init.clone()
    ctx.hevi_newton_solve(lam, q_ref, R, rtol=1e-12, max_iter=20)
    st_ref, it_ref = ctx.hevi_column_status()
    d_ref = (q_ref - q_init).cpu().numpy().reshape(ncols, -1)
    for call in range(2):
        q = q_init.clone()
        status = torch.full((ncols,), -1, dtype=torch.int32, device="cuda")
        iters = torch.full((ncols,), -1, dtype=torch.int32, device="cuda")
        hv.hevi_newton_solve_noalloc(nez, N, 30e3, ncols, lam, q, R, status, iters,
                                     rtol=1e-12, max_iter=20)
        d = (q - q_init).cpu().numpy().reshape(ncols, -1)
        err = _rel_cols(d, d_ref)
        assert err.max() < TOL, (call, err.max())
        assert int(status.abs().max()) == 0
        assert int(iters.min()) >= 1


def test_noalloc_refuses_columns_beyond_its_scratch(hv):
    import torch
    nez, N, ncols = 16, 3, 20_000
    n = 3 * (nez * N + 1) * ncols
    q = torch.ones(n, dtype=torch.float64, device="cuda")
    R = q.clone()
    st = torch.zeros(ncols, dtype=torch.int32, device="cuda")
    it = torch.zeros(ncols, dtype=torch.int32, device="cuda")
    with pytest.raises(hv.HeviError) as e:
        hv.hevi_newton_solve_noalloc(nez, N, 30e3, ncols, 87.0, q, R, st, it)
    assert e.value.code == 1 and "scratch" in str(e.value)
    assert bool((q == 1).all())


def _largest_accepted(hv, nez, N):
    """The largest column count the scratch array takes (binary search on
    rest-state inputs: an accepted call stops at Newton iteration 0)."""
    import torch
    n = 3 * (nez * N + 1)

    def ok(ncols):
        ctx = hv.Context([(nez, N)], 30e3, ncols=ncols, precision=hv.FP32_IR)
        q = ctx.hevi_reference_state()
        R = q.clone()
        st = torch.zeros(ncols, dtype=torch.int32, device="cuda")
        it = torch.zeros(ncols, dtype=torch.int32, device="cuda")
        try:
            hv.hevi_newton_solve_noalloc(nez, N, 30e3, ncols, 87.0, q, R, st, it)
            return True
        except hv.HeviError as e:
            assert e.code == 1
            assert bool((q == R).all())   # refused before any device work
            return False
        finally:
            del ctx
    lo, hi = 1, 1 << 14
    assert ok(lo) and not ok(hi)
    while hi - lo > 1:
        mid = (lo + hi) // 2
        lo, hi = (mid, hi) if ok(mid) else (lo, mid)
    assert n * lo * 8 > 2 ** 20   # the boundary is where the documented scratch runs out
    return lo


def test_noalloc_at_its_column_limit_and_one_tile_above(hv):
    """At the largest column count the 64 MiB array holds (about 4,000 columns
    of (16, 3)), twice in a row, against the context Newton; one column and one
    tile of columns more are refused."""
    import torch
    nez, N = 16, 3
    top = _largest_accepted(hv, nez, N)
    assert 3500 < top < 4600, top
    inp = hevi_inputs.nhevi_ark2(seed=4, nez=nez, N=N, ncols=top)
    ctx = hv.Context([(nez, N)], inp["ztop"], precision=hv.FP32_IR)
    q_init = ctx.hevi_reference_state() + torch.from_numpy(inp["dq"].reshape(-1)).cuda()
    R = q_init + 0.01 * (q_init - ctx.hevi_reference_state())
    lam = (1 - 2 ** -0.5) * inp["dt"]
    q_ref = q_init.clone()
    ctx.hevi_newton_solve(lam, q_ref, R, rtol=1e-12, max_iter=20)
    d_ref = (q_ref - q_init).cpu().numpy().reshape(top, -1)
    for call in range(2):
        q = q_init.clone()
        status = torch.full((top,), -1, dtype=torch.int32, device="cuda")
        iters = torch.full((top,), -1, dtype=torch.int32, device="cuda")
        hv.hevi_newton_solve_noalloc(nez, N, 30e3, top, lam, q, R, status, iters,
                                     rtol=1e-12, max_iter=20)
        d = (q - q_init).cpu().numpy().reshape(top, -1)
        assert _rel_cols(d, d_ref).max() < TOL, call
        assert int(status.abs().max()) == 0
    for more in (top + 1, top + 32):
        n = 3 * (nez * N + 1) * more
        q = torch.ones(n, dtype=torch.float64, device="cuda")
        st = torch.zeros(more, dtype=torch.int32, device="cuda")
        it = torch.zeros(more, dtype=torch.int32, device="cuda")
        with pytest.raises(hv.HeviError) as e:
            hv.hevi_newton_solve_noalloc(nez, N, 30e3, more, 87.0, q, q.clone(), st, it)
        assert e.value.code == 1
        assert bool((q == 1).all())


def test_noalloc_refuses_a_column_beyond_the_block_shared_memory(hv):
    """One very long column (4,096 elements of order 1): its scratch fits,
    but the Newton kernel's shared memory per block would not; refused up front."""
    import torch
    nez, N, ncols = 4096, 1, 1
    n = 3 * (nez * N + 1)
    q = torch.ones(n, dtype=torch.float64, device="cuda")
    st = torch.zeros(ncols, dtype=torch.int32, device="cuda")
    it = torch.zeros(ncols, dtype=torch.int32, device="cuda")
    with pytest.raises(hv.HeviError) as e:
        hv.hevi_newton_solve_noalloc(nez, N, 30e3, ncols, 87.0, q, q.clone(), st, it)
    assert e.value.code == 1
    assert bool((q == 1).all())
