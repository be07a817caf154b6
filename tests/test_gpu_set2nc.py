"""Equation set 2NC (unknowns rho, w, theta: the advective set of Sec. 2.1) on
the GPU's FP64 path against the FP64 oracle in the same set: reference state,
operator applies, stage solves, LHEVI steps and NHEVI-LU Newton solves, at the
same 1e-10 relative bar as sets 2C and 3C; and the refusals (FP32 contexts,
NHEVI-GMRES)."""

import numpy as np
import pytest

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


def _np(t, ncols):
    return t.cpu().numpy().reshape(ncols, -1)


def _rel_cols(x, ref):
    num = np.linalg.norm(x - ref, axis=1)
    den = np.linalg.norm(ref, axis=1)
    return num / np.where(den == 0, 1.0, den)


def _ctx(hv, nez, N, ncols):
    ctx = hv.Context([(nez, N)], ZTOP, ncols=ncols, precision=hv.FP64)
    ctx.hevi_set_equation_set(hv.SET_2NC)
    return ctx


def _state(nez, N, ncols, seed, amp_w=5.0, amp_t=2.0):
    """Rest density times 1 +- 1%, w uniform (0 at both ends), theta =
    theta_bar +- amp_t."""
    g = np.random.default_rng(seed)
    with oracle.equation_set(oracle.SET_2NC):
        qr = oracle.reference_q(nez, N, ZTOP, 1)[0].reshape(-1, 3)
    nz = qr.shape[0]
    rho = qr[:, 0] * (1 + 0.01 * g.uniform(-1, 1, (ncols, nz)))
    w = g.uniform(-amp_w, amp_w, (ncols, nz))
    w[:, 0] = w[:, -1] = 0.0
    th = qr[:, 2] + g.uniform(-amp_t, amp_t, (ncols, nz))
    return np.stack([rho, w, th], -1).reshape(ncols, -1)


def _small(nez, N, ncols, seed, amp=1e-2):
    with oracle.equation_set(oracle.SET_2NC):
        s = oracle.scales(oracle.column_grid(nez, N, ZTOP)[0])
    b = np.random.default_rng(seed).standard_normal((ncols, s.size)) * s * amp
    b[:, 1] = b[:, -2] = 0.0
    return b


def test_set2nc_reference_state_and_rest(hv):
    nez, N, ncols = 8, 4, 37
    ctx = _ctx(hv, nez, N, ncols)
    q = ctx.hevi_reference_state()
    with oracle.equation_set(oracle.SET_2NC):
        ref = oracle.reference_q(nez, N, ZTOP, ncols)
    assert _rel_cols(_np(q, ncols), ref).max() < 1e-14
    v = ctx.empty()
    ctx.hevi_apply_Lv(q, v, nonlinear=True)
    assert float(v.abs().max()) == 0.0


@pytest.mark.parametrize("nez,N", [(3, 2), (8, 4), (16, 3), (2, 5)])
def test_set2nc_operators_match_oracle(hv, nez, N):
    ncols = 35
    ctx = _ctx(hv, nez, N, ncols)
    q = _state(nez, N, ncols, seed=51)
    x = _small(nez, N, ncols, seed=52, amp=1.0)
    v = ctx.empty()
    ctx.hevi_apply_Lv(_t(q), v, nonlinear=True)
    ctx.hevi_factor(0.0, _t(q))  # the linearisation about q
    y = ctx.empty()
    ctx.hevi_apply_Lv(_t(x), y, nonlinear=False)
    with oracle.equation_set(oracle.SET_2NC):
        vr = oracle.apply_V(nez, N, ZTOP, q)
        yr = oracle.apply_L(nez, N, ZTOP, q, x)
    assert _rel_cols(_np(v, ncols), vr).max() < 1e-12
    assert _rel_cols(_np(y, ncols), yr).max() < 1e-12


@pytest.mark.parametrize("rhs", ["increment", "state"])
@pytest.mark.parametrize("nez,N,ncols", [(4, 3, 35), (8, 4, 70), (24, 4, 33), (1, 1, 3)])
def test_set2nc_stage_solve_matches_oracle(hv, nez, N, ncols, rhs):
    lam = 87.868
    ctx = _ctx(hv, nez, N, ncols)
    q0 = _state(nez, N, ncols, seed=53)
    b = _small(nez, N, ncols, seed=54)
    if rhs == "state":
        b = q0 + b
    ctx.hevi_factor(lam, _t(q0))
    x = _np(ctx.hevi_stage_solve(_t(b)), ncols)
    with oracle.equation_set(oracle.SET_2NC):
        xr, info = oracle.stage_solve(nez, N, ZTOP, lam, q0, b)
    assert (info == 0).all()
    err = _rel_cols(x, xr)
    assert err.max() < TOL, err.max()
    st, _ = ctx.hevi_column_status()
    assert int(st.abs().max()) == 0


@pytest.mark.parametrize("name", ["ARK2", "ARK3"])
def test_set2nc_lhevi_step_matches_oracle(hv, name):
    """One LHEVI-PS step from a perturbed set-2NC state under a small explicit
    tendency: the increment q^{n+1} - q^n at 1e-10 relative."""
    nez, N, ncols, dt = 10, 4, 45, 300.0
    ctx = _ctx(hv, nez, N, ncols)
    q_in = _state(nez, N, ncols, seed=55, amp_w=1.0, amp_t=0.5)
    H = _small(nez, N, ncols, seed=56, amp=1e-7)
    q_out = ctx.hevi_lhevi_step(hv.tableau(name), dt, _t(q_in), _t(H))
    ctx.hevi_sync()
    with oracle.equation_set(oracle.SET_2NC):
        q_ref, info = oracle.lhevi_step(nez, N, ZTOP, tableaux.ALL[name], dt, q_in, H, lin=0)
    assert (info == 0).all()
    err = _rel_cols(_np(q_out, ncols) - q_in, q_ref - q_in)
    assert err.max() < TOL, err.max()


@pytest.mark.parametrize("nez,N,ncols", [(16, 3, 40), (8, 4, 33)])
def test_set2nc_newton_matches_oracle(hv, nez, N, ncols):
    """NHEVI-LU in set 2NC at rtol 1e-10: the Newton update against the
    oracle's solve at the same tolerance and against its root."""
    lam = 87.868
    ctx = _ctx(hv, nez, N, ncols)
    q_init = _state(nez, N, ncols, seed=57, amp_w=2.0, amp_t=1.0)
    R = q_init + _small(nez, N, ncols, seed=58)
    with oracle.equation_set(oracle.SET_2NC):
        q_ref, _, st_ref = oracle.newton(nez, N, ZTOP, lam, R, q_init, rtol=1e-10)
        q_root, _, _ = oracle.newton(nez, N, ZTOP, lam, R, q_init, rtol=0.0, max_iter=30)
    assert (st_ref == 0).all()
    q = _t(q_init)
    ctx.hevi_newton_solve(lam, q, _t(R), rtol=1e-10)
    d = _np(q, ncols) - q_init
    assert _rel_cols(d, q_ref - q_init).max() < TOL
    assert _rel_cols(d, q_root - q_init).max() < TOL
    st, _ = ctx.hevi_column_status()
    assert int(st.abs().max()) == 0


def test_set2nc_refusals(hv):
    ctx32 = hv.Context([(8, 4)], ZTOP, ncols=8, precision=hv.FP32_IR)
    with pytest.raises(hv.HeviError):
        ctx32.hevi_set_equation_set(hv.SET_2NC)
    ctx = _ctx(hv, 8, 4, 8)
    q = ctx.hevi_reference_state()
    with pytest.raises(hv.HeviError):
        ctx.hevi_newton_gmres_solve(87.0, q, q.clone())
    ctx.hevi_set_equation_set(hv.SET_2C)  # back to set 2C on the same context
    q2 = ctx.hevi_reference_state()
    ref = oracle.reference_q(8, 4, ZTOP, 8)
    assert _rel_cols(_np(q2, 8), ref).max() < 1e-14
