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
