"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on
the same seeded inputs.  Bar: relative L2 error per column <= 1e-10 for FP64
and for FP32 factors with FP64 refinement."""

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


def _np(t, ncols):
    return t.cpu().numpy().reshape(ncols, -1)


def _rel_cols(x, ref):
    num = np.linalg.norm(x - ref, axis=1)
    den = np.linalg.norm(ref, axis=1)
    den = np.where(den == 0, 1.0, den)
    return num / den


def _perturbed(nez, N, ncols, seed, ztop=ZTOP, amp_w=5.0, amp_th=2.0):
    g = np.random.default_rng(seed)
    q = oracle.reference_q(nez, N, ztop, ncols).reshape(ncols, -1, 3)
    nz = q.shape[1]
    w = g.uniform(-amp_w, amp_w, (ncols, nz))
    w[:, 0] = w[:, -1] = 0.0
    th = g.uniform(-amp_th, amp_th, (ncols, nz))
    rho = q[:, :, 0] * (1 + 0.01 * g.uniform(-1, 1, (ncols, nz)))
    Theta = q[:, :, 2] / q[:, :, 0] * rho + rho * th
    return np.stack([rho, rho * w, Theta], -1).reshape(ncols, -1)


def _rhs(nez, N, ncols, seed, ztop=ZTOP):
    s = oracle.scales(oracle.column_grid(nez, N, ztop)[0])
    b = np.random.default_rng(seed).standard_normal((ncols, s.size)) * s * 1e-2
    b[:, 1] = b[:, -2] = 0.0
    return b


# ---------------------------------------------------------------------------
# reference state, operator applies
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("nez,N", [(1, 1), (3, 2), (8, 4), (16, 3), (24, 4), (2, 5)])
def test_reference_state(hv, nez, N):
    ncols = 37
    ctx = hv.Context([(nez, N)], ZTOP, ncols=ncols)
    q = _np(ctx.hevi_reference_state(), ncols)
    ref = oracle.reference_q(nez, N, ZTOP, ncols)
    assert _rel_cols(q, ref).max() < 1e-14


@pytest.mark.parametrize("nez,N", [(1, 1), (3, 2), (8, 4), (16, 3), (24, 4), (2, 5)])
def test_rest_state_exact_on_gpu(hv, nez, N):
    ncols = 40
    ctx = hv.Context([(nez, N)], ZTOP, ncols=ncols)
    q = ctx.hevi_reference_state()
    v = ctx.hevi_apply_Lv(q, nonlinear=True)
    assert float(v.abs().max()) == 0.0


@pytest.mark.parametrize("nez,N,ncols", [(2, 1, 5), (3, 2, 33), (8, 4, 70), (16, 3, 65), (2, 5, 31)])
def test_apply_parity(hv, nez, N, ncols):
    ctx = hv.Context([(nez, N)], ZTOP, ncols=ncols, precision=hv.FP64)
    q = _perturbed(nez, N, ncols, seed=1)
    x = _rhs(nez, N, ncols, seed=2)
    v_gpu = _np(ctx.hevi_apply_Lv(_t(q), nonlinear=True), ncols)
    v_ref = oracle.apply_V(nez, N, ZTOP, q)
    assert _rel_cols(v_gpu, v_ref).max() < 1e-12
    ctx.hevi_factor(50.0, _t(q))
    l_gpu = _np(ctx.hevi_apply_Lv(_t(x), nonlinear=False), ncols)
    l_ref = oracle.apply_L(nez, N, ZTOP, q, x)
    assert _rel_cols(l_gpu, l_ref).max() < 1e-12


# ---------------------------------------------------------------------------
# stage solve: FP64 band LU and FP32 LU + FP64 refinement
# ---------------------------------------------------------------------------

SOLVE_CASES = [(1, 1, 3), (2, 2, 33), (3, 3, 40), (8, 4, 97), (10, 4, 70), (16, 3, 64),
               (24, 4, 35), (2, 5, 33)]


@pytest.mark.parametrize("prec", ["FP64", "FP32_IR"])
@pytest.mark.parametrize("nez,N,ncols", SOLVE_CASES)
def test_stage_solve_parity(hv, prec, nez, N, ncols):
    lam = 87.868
    ctx = hv.Context([(nez, N)], ZTOP, ncols=ncols, precision=getattr(hv, prec))
    q0 = _perturbed(nez, N, ncols, seed=3 + N)
    b = _rhs(nez, N, ncols, seed=4 + nez)
    ctx.hevi_factor(lam, _t(q0))
    x = _np(ctx.hevi_stage_solve(_t(b)), ncols)
    x_ref, info = oracle.stage_solve(nez, N, ZTOP, lam, q0, b)
    assert (info == 0).all()
    err = _rel_cols(x, x_ref)
    assert err.max() < TOL, err.max()
    st, it = ctx.hevi_column_status()
    assert int(st.abs().max()) == 0
    if prec == "FP32_IR":
        its = it.cpu().numpy()
        assert its.min() >= 2 and its.max() <= 4


@pytest.mark.parametrize("ncols,tol,sweeps", [
    (5, 1e-11, 10),     # one partial tile: every sweep by the whole warp, one column at a time
    (40, 1e-11, 10),    # a full tile (shared-memory record ring) and a partial one
    (40, 1e-15, 6),     # every column refines past the contraction limit: ring for all sweeps
    (70, 1e-13, 10),    # mixed: ring sweeps, then a few lanes per warp continue
    (64, 1.0, 10),      # one sweep (the first FP32 solve) is accepted
])
def test_stage_solve_refinement_paths(hv, ncols, tol, sweeps):
    """The FP32 + refinement solve takes three code paths per warp (all 32
    lanes through the record ring, a few lanes by the whole warp, otherwise
    one lane per column); each must give the oracle's solution."""
    nez, N, lam = 10, 4, 87.868
    ctx = hv.Context([(nez, N)], ZTOP, ncols=ncols, precision=hv.FP32_IR)
    ctx.hevi_set_refinement(tol, sweeps)
    q0 = _perturbed(nez, N, ncols, seed=21)
    b = _rhs(nez, N, ncols, seed=22)
    ctx.hevi_factor(lam, _t(q0))
    x = ctx.empty()
    try:
        ctx.hevi_stage_solve(_t(b), x)
    except hv.HeviError as e:
        assert tol < 1e-14 and e.code == 5, e   # the contraction stop reports NOT_CONVERGED
    x = _np(x, ncols)
    x_ref, info = oracle.stage_solve(nez, N, ZTOP, lam, q0, b)
    assert (info == 0).all()
    err = _rel_cols(x, x_ref)
    st, it = ctx.hevi_column_status()
    its = it.cpu().numpy()
    if tol >= 1.0:
        assert (its == 1).all()
        assert err.max() < 1e-3, err.max()  # FP32 factors alone
    else:
        assert err.max() < TOL, err.max()
        assert its.min() >= 2 and its.max() <= sweeps


def test_record_copy_wait_runs_out(hv):
    """A record copy that never arrives: the ring's bounded wait runs out, the
    tiles' columns end WAIT_TIMEOUT with x = NaN, nothing is left in flight,
    and the same context then solves normally."""
    nez, N, ncols, lam = 10, 4, 64, 87.868
    ctx = hv.Context([(nez, N)], ZTOP, ncols=ncols, precision=hv.FP32_IR)
    q0 = _perturbed(nez, N, ncols, seed=23)
    b = _rhs(nez, N, ncols, seed=24)
    ctx.hevi_factor(lam, _t(q0))
    ctx.hevi_test_drop_record_copy(5)
    x = ctx.empty()
    with pytest.raises(hv.HeviError) as e:
        ctx.hevi_stage_solve(_t(b), x)
    assert e.value.code == 7
    st, _ = ctx.hevi_column_status()
    assert bool((st == 7).all())
    assert bool(x.isnan().all())
    ctx.hevi_test_drop_record_copy(-1)
    x = _np(ctx.hevi_stage_solve(_t(b)), ncols)
    x_ref, info = oracle.stage_solve(nez, N, ZTOP, lam, q0, b)
    assert _rel_cols(x, x_ref).max() < TOL


@pytest.mark.parametrize("prec", ["FP64", "FP32_IR"])
def test_stage_solve_lhevi_stage_workload(hv, prec):
    """1,538 columns, Nez=8, N=4, 30 km, about the rest state (all columns)."""
    inp = hevi_inputs.lhevi_stage(seed=1)
    nez, N, ncols = inp["nez"], inp["N"], inp["ncols"]
    ctx = hv.Context([(nez, N)], inp["ztop"], precision=getattr(hv, prec))
    ctx.hevi_factor(inp["lam"], None)
    x = _np(ctx.hevi_stage_solve(_t(inp["b"])), ncols)
    q0 = oracle.reference_q(nez, N, ZTOP, ncols)
    x_ref, info = oracle.stage_solve(nez, N, inp["ztop"], inp["lam"], q0, inp["b"])
    assert _rel_cols(x, x_ref).max() < TOL


@pytest.mark.parametrize("prec", ["FP64", "FP32_IR"])
def test_stage_solve_full_size_sampled(hv, prec):
    """86,402 columns of (10, 4): the launch the benchmark times; sampled
    columns against the oracle one by one."""
    ne, nez, N = 30, 10, 4
    ncols = 6 * (ne * 4) ** 2 + 2
    ctx = hv.Context([(nez, N)], ZTOP, ncols=ncols, precision=getattr(hv, prec))
    g = np.random.default_rng(5)
    sample = np.sort(g.choice(ncols, 48, replace=False))
    sample[-1] = ncols - 1
    q0 = _perturbed(nez, N, ncols, seed=6, amp_w=1.0, amp_th=1.0)
    b = _rhs(nez, N, ncols, seed=7)
    lam = 87.868
    ctx.hevi_factor(lam, _t(q0))
    x = _np(ctx.hevi_stage_solve(_t(b)), ncols)
    x_ref, _ = oracle.stage_solve(nez, N, ZTOP, lam, q0[sample], b[sample])
    assert _rel_cols(x[sample], x_ref).max() < TOL
    assert np.isfinite(x).all()


def test_stage_solve_lambda_zero_is_identity(hv):
    nez, N, ncols = 8, 4, 33
    ctx = hv.Context([(nez, N)], ZTOP, ncols=ncols, precision=hv.FP32_IR)
    b = _rhs(nez, N, ncols, seed=8)
    ctx.hevi_factor(0.0, None)
    x = _np(ctx.hevi_stage_solve(_t(b)), ncols)
    # the last refinement correction is scaled back in FP32 (relative 6e-8 of a
    # correction of ~1e-7 |x|), so the identity is exact to ~1e-14
    assert _rel_cols(x, b).max() < 1e-13


def test_stage_solve_zero_rhs(hv):
    nez, N, ncols = 8, 4, 33
    for prec in (hv.FP64, hv.FP32_IR):
        ctx = hv.Context([(nez, N)], ZTOP, ncols=ncols, precision=prec)
        ctx.hevi_factor(87.0, None)
        x = ctx.hevi_stage_solve(ctx.hevi_reference_state() * 0)
        assert float(x.abs().max()) == 0.0


def test_mixed_classes_and_tops(hv):
    """Uneven columns (4 size classes, tops 30-100 km) in one context."""
    classes = hevi_inputs.SIZE_CLASSES
    g = np.random.default_rng(9)
    ncols = 150
    cls = g.integers(0, 4, ncols).astype(np.int32)
    zt = g.uniform(30e3, 100e3, ncols)
    for prec in ("FP64", "FP32_IR"):
        ctx = hv.Context(classes, zt, class_of_col=cls, precision=getattr(hv, prec))
        off = ctx.offsets()
        q0 = np.zeros(ctx.n)
        b = np.zeros(ctx.n)
        for i, (nez, N) in enumerate(classes):
            idx = np.nonzero(cls == i)[0]
            qi = _perturbed(nez, N, 1, seed=10 + i, ztop=50e3)  # shape only
            for c in idx:
                qq = oracle.reference_q(nez, N, zt[c])[0]
                qq = qq * (1 + 0.001 * np.random.default_rng(c).standard_normal(qq.size))
                qq[1::3] = 0.0
                q0[off[c]:off[c + 1]] = qq
                bb = _rhs(nez, N, 1, seed=100 + c, ztop=zt[c])[0]
                b[off[c]:off[c + 1]] = bb
            del qi
        ctx.hevi_factor(60.0, _t(q0))
        x = ctx.hevi_stage_solve(_t(b)).cpu().numpy()
        worst = 0.0
        for c in range(ncols):
            nez, N = classes[cls[c]]
            xr, info = oracle.stage_solve(nez, N, zt[c], 60.0, q0[None, off[c]:off[c + 1]],
                                          b[None, off[c]:off[c + 1]])
            worst = max(worst, _rel_cols(x[None, off[c]:off[c + 1]], xr).max())
        assert worst < TOL, (prec, worst)


def test_bad_input_reported(hv):
    nez, N, ncols = 4, 3, 40
    ctx = hv.Context([(nez, N)], ZTOP, ncols=ncols, precision=hv.FP32_IR)
    q0 = oracle.reference_q(nez, N, ZTOP, ncols)
    q0[7, 3] = -1.0       # negative density in column 7
    ctx.hevi_factor(50.0, _t(q0))
    with pytest.raises(hv.HeviError) as e:
        ctx.hevi_stage_solve(_t(_rhs(nez, N, ncols, 1)))
    assert e.value.code == 6
    st, _ = ctx.hevi_column_status()
    st = st.cpu().numpy()
    assert st[7] == hv.COL_BAD_INPUT and (np.delete(st, 7) == 0).all()


# ---------------------------------------------------------------------------
# NHEVI-LU Newton
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("nez,N,ncols", [(2, 1, 5), (4, 2, 33), (16, 3, 70), (8, 4, 40)])
def test_newton_parity(hv, nez, N, ncols):
    # Both sides converge to rtol 1e-12: two Newton iterations that stop at the
    # same residual tolerance may differ by about that tolerance times the
    # conditioning (the FP32-factored GPU Newton converges linearly, the FP64
    # oracle quadratically), so parity at 1e-10 is checked 100x inside it.
    lam = 87.868
    ctx = hv.Context([(nez, N)], ZTOP, ncols=ncols, precision=hv.FP32_IR)
    q_init = _perturbed(nez, N, ncols, seed=11, amp_w=2.0, amp_th=1.0)
    R = q_init + _rhs(nez, N, ncols, seed=12)
    q_ref, it_ref, st_ref = oracle.newton(nez, N, ZTOP, lam, R, q_init, rtol=1e-12, max_iter=20)
    assert (st_ref == 0).all()
    q = _t(q_init)
    ctx.hevi_newton_solve(lam, q, _t(R), rtol=1e-12, max_iter=20)
    q = _np(q, ncols)
    # compare the Newton update q - q_init, stricter than the full state
    err = _rel_cols(q - q_init, q_ref - q_init)
    assert err.max() < TOL, err.max()
    st, it = ctx.hevi_column_status()
    assert int(st.abs().max()) == 0
    assert int(it.max()) <= 8


@pytest.mark.parametrize("nez,N,ncols", [(16, 3, 40), (8, 4, 37), (4, 2, 33)])
def test_newton_parity_at_config_tolerance(hv, nez, N, ncols):
    """At the configuration's rtol = 1e-10 the GPU Newton solve matches the
    oracle's solve at the same tolerance, and the root (the oracle iterated to
    its rounding floor), to 1e-10 in the Newton update."""
    lam = 87.868
    ctx = hv.Context([(nez, N)], ZTOP, ncols=ncols, precision=hv.FP32_IR)
    q_init = _perturbed(nez, N, ncols, seed=11, amp_w=2.0, amp_th=1.0)
    R = q_init + _rhs(nez, N, ncols, seed=12)
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


def test_newton_rest_state_no_update(hv):
    nez, N, ncols = 16, 3, 33
    ctx = hv.Context([(nez, N)], ZTOP, ncols=ncols, precision=hv.FP32_IR)
    q = ctx.hevi_reference_state()
    q0 = q.clone()
    ctx.hevi_newton_solve(87.0, q, q0.clone())
    assert bool((q == q0).all())
    _, it = ctx.hevi_column_status()
    assert int(it.max()) == 0


def test_newton_full_size_sampled(hv):
    """86,402 columns of (16, 3), the NHEVI workload's state and Lambda of ARK2
    at 300 s, Newton to the configuration's rtol 1e-10: sampled columns
    against the oracle at the same tolerance."""
    inp = hevi_inputs.nhevi_ark2(seed=3)
    nez, N, ncols = inp["nez"], inp["N"], inp["ncols"]
    ctx = hv.Context([(nez, N)], inp["ztop"], precision=hv.FP32_IR)
    q0 = ctx.hevi_reference_state() + _t(inp["dq"])
    lam = tableaux.ARK2.gamma * inp["dt"]
    R = q0.clone()
    q = q0.clone()
    # a stage-like problem: R = q0, guess q0
    ctx.hevi_newton_solve(lam, q, R, rtol=1e-10)
    sample = np.sort(np.random.default_rng(13).choice(ncols, 24, replace=False))
    sample[-1] = ncols - 1
    qn = _np(q, ncols)
    q0n = _np(q0, ncols)
    q_ref, _, st = oracle.newton(nez, N, inp["ztop"][sample], lam, q0n[sample], q0n[sample],
                                 rtol=1e-10)
    assert (st == 0).all()
    assert _rel_cols(qn[sample] - q0n[sample], q_ref - q0n[sample]).max() < TOL
    assert np.isfinite(qn).all()


# ---------------------------------------------------------------------------
# whole ARK steps
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["ARK2", "ARK3", "ARS3", "ARK4"])
@pytest.mark.parametrize("prec", ["FP64", "FP32_IR"])
def test_lhevi_step_parity(hv, name, prec):
    nez, N, ncols = 10, 4, 45
    inp = hevi_inputs.lhevi_ark3(seed=2, ncols=ncols, nez=nez, N=N)
    ctx = hv.Context([(nez, N)], inp["ztop"], precision=getattr(hv, prec))
    tab = hv.tableau(name)
    q_in = ctx.hevi_reference_state()
    q_in += _t(_perturbed(nez, N, ncols, seed=14, amp_w=1.0, amp_th=0.5)) - q_in  # perturbed start
    H = _t(inp["H"])
    q_out = ctx.hevi_lhevi_step(tab, inp["dt"], q_in, H)
    ctx.hevi_sync()
    qi = _np(q_in, ncols)
    q_ref, info = oracle.lhevi_step(nez, N, inp["ztop"], tableaux.ALL[name], inp["dt"], qi,
                                    inp["H"], lin=0)
    assert (info == 0).all()
    err = _rel_cols(_np(q_out, ncols) - qi, q_ref - qi)
    assert err.max() < TOL, err.max()


@pytest.mark.parametrize("name", ["ARK2", "ARK3"])
def test_nhevi_step_parity(hv, name):
    nez, N, ncols = 16, 3, 40
    inp = hevi_inputs.nhevi_ark2(seed=3, ncols=ncols)
    ctx = hv.Context([(nez, N)], inp["ztop"], precision=hv.FP32_IR)
    q_in = ctx.hevi_reference_state() + _t(inp["dq"])
    H = _t(_rhs(nez, N, ncols, seed=15) * 1e-3)
    q_out = ctx.hevi_nhevi_step(hv.tableau(name), inp["dt"], q_in, H, rtol=1e-12)
    ctx.hevi_sync()
    qi = _np(q_in, ncols)
    q_ref, it, st = oracle.nhevi_step(nez, N, inp["ztop"], tableaux.ALL[name], inp["dt"], qi,
                                      H.cpu().numpy().reshape(ncols, -1), rtol=1e-12)
    assert (st == 0).all()
    err = _rel_cols(_np(q_out, ncols) - qi, q_ref - qi)
    assert err.max() < TOL, err.max()
