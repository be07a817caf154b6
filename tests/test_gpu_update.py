"""Jacobian update interval on the GPU (Sec. 4.3; the update time-step of
Sec. 7.1): LHEVI steps that keep the factorisation of an earlier state,
against the oracle linearised about that same state (1e-10 relative on the
step's increment, 30 km columns from a perturbed state)."""

import numpy as np
import pytest

import hevi_inputs
import oracle
from oracle import tableaux

pytestmark = pytest.mark.gpu

TOL = 1e-10
ZTOP = 30e3


@pytest.fixture(scope="module")
def hv():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2311_11425_gb300 as hv
    hv.load(build=True)
    return hv


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).reshape(-1)).cuda()


def _state(nez, N, ncols, seed, amp):
    g = np.random.default_rng(seed)
    q = oracle.reference_q(nez, N, ZTOP, ncols)
    dq = hevi_inputs.state_increment(g, nez, N, np.full(ncols, ZTOP), amp=amp)
    return q + dq


def _rel_inc(got, qn, ref):
    num = np.linalg.norm((got - qn) - (ref - qn), axis=1)
    den = np.linalg.norm(ref - qn, axis=1)
    return (num / den).max()


@pytest.mark.parametrize("name", ["ARK3", "ARS3"])
@pytest.mark.parametrize("prec", ["FP32_IR", "FP64"])
def test_step_with_kept_factorisation(hv, name, prec):
    nez, N, ncols = 10, 4, 40
    tab = hv.tableau(name)
    dt = 300.0
    ctx = hv.Context([(nez, N)], ZTOP, ncols=ncols, precision=getattr(hv, prec))
    q_lin = _state(nez, N, ncols, seed=1, amp=1.0)
    qn = _state(nez, N, ncols, seed=2, amp=1.0)
    H = np.zeros_like(qn)
    ctx.hevi_factor(tab.gamma * dt, _t(q_lin))
    out = ctx.hevi_lhevi_step(tab, dt, _t(qn), _t(H), refactor=False)
    ctx.hevi_sync()
    ref, info = oracle.lhevi_step(nez, N, ZTOP, tableaux.ALL[name], dt, qn, H, lin=0, q_lin=q_lin)
    assert (info == 0).all()
    err = _rel_inc(out.cpu().numpy().reshape(ncols, -1), qn, ref)
    assert err < TOL, err


def test_update_every_three_steps(hv):
    """Six ARK3 steps, the Jacobian refactored at steps 0 and 3 only."""
    nez, N, ncols, dt = 10, 4, 33, 300.0
    tab = hv.tableau("ARK3")
    inp = hevi_inputs.lhevi_ark3(seed=2, ncols=ncols, nez=nez, N=N)
    ctx = hv.Context([(nez, N)], ZTOP, ncols=ncols, precision=hv.FP32_IR)
    q0 = _state(nez, N, ncols, seed=3, amp=0.3)
    q = _t(q0)
    H = _t(inp["H"])
    for k in range(6):
        q = ctx.hevi_lhevi_step(tab, dt, q, H, refactor=(k % 3 == 0))
    ctx.hevi_sync()
    qr = q0.copy()
    for k in range(6):
        if k % 3 == 0:
            q_lin = qr.copy()
        qr, info = oracle.lhevi_step(nez, N, ZTOP, tableaux.ARK3, dt, qr, inp["H"], lin=0,
                                     q_lin=q_lin)
        assert (info == 0).all()
    err = _rel_inc(q.cpu().numpy().reshape(ncols, -1), q0, qr)
    assert err < TOL, err


def test_kept_factorisation_must_exist_and_match(hv):
    nez, N, ncols = 4, 4, 8
    tab = hv.tableau("ARK2")
    ctx = hv.Context([(nez, N)], ZTOP, ncols=ncols, precision=hv.FP32_IR)
    q = ctx.hevi_reference_state()
    H = q * 0
    with pytest.raises(hv.HeviError):
        ctx.hevi_lhevi_step(tab, 300.0, q, H, refactor=False)  # nothing factored yet
    ctx.hevi_lhevi_step(tab, 300.0, q, H)
    ctx.hevi_lhevi_step(tab, 300.0, q, H, refactor=False)      # same gamma dt: fine
    with pytest.raises(hv.HeviError):
        ctx.hevi_lhevi_step(tab, 150.0, q, H, refactor=False)  # different gamma dt
    ctx.hevi_sync()
