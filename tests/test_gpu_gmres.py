"""NHEVI-GMRES on the GPU (Sec. 4.2.1): Jacobian-free Newton-Krylov column
solves against the FP64 oracle's same algorithm and against Newton-LU.

At tight settings (small Frechet perturbation, tolerances 1e-12) both sides
reach the root of F to rounding, so the increments agree to 1e-10.  At the
paper's settings (eps = 0.05, Newton 1e-5, GMRES 1e-9) the iteration stops
early and the root is held to the Newton tolerance."""

import numpy as np
import pytest

import hevi_inputs
import oracle
from oracle import tableaux

pytestmark = pytest.mark.gpu

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


def _case(classes, ncols, seed):
    g = np.random.default_rng(seed)
    cls = g.integers(0, len(classes), ncols).astype(np.int32)
    qs, ns = [], []
    for c in range(ncols):
        nez, N = classes[cls[c]]
        q = oracle.reference_q(nez, N, ZTOP, 1)[0]
        q = q + hevi_inputs.state_increment(g, nez, N, np.array([ZTOP]))[0]
        qs.append(q)
    return cls, qs


def _pack(qs):
    return np.concatenate(qs)


@pytest.mark.parametrize("classes", [[(16, 3)], [(16, 3), (10, 4)]])
def test_gmres_matches_oracle_tight(hv, classes):
    import torch
    ncols = 40
    lam = tableaux.ARK2.gamma * 300.0
    cls, qs = _case(classes, ncols, seed=51)
    ctx = hv.Context(classes, ZTOP, class_of_col=cls if len(classes) > 1 else None, ncols=ncols,
                     precision=hv.FP32_IR)
    off = ctx.offsets()
    q0 = _pack(qs)
    q = _t(q0)
    R = _t(q0)
    kry = torch.zeros(ncols, dtype=torch.int32, device="cuda")
    ctx.hevi_newton_gmres_solve(lam, q, R, eps=1e-7, rtol=1e-12, gtol=1e-12, krylov=kry)
    qg = q.cpu().numpy()
    st, it = ctx.hevi_column_status()
    assert bool((st == 0).all())
    kry = kry.cpu().numpy()
    worst = 0.0
    for c in range(ncols):
        nez, N = classes[cls[c]]
        a, b = off[c], off[c + 1]
        qr, itr, kitr, str_ = oracle.newton_gmres(nez, N, ZTOP, lam, q0[None, a:b], q0[None, a:b],
                                                  eps=1e-7, rtol=1e-12, gtol=1e-12)
        assert str_[0] == 0
        s = oracle.scales(oracle.column_grid(nez, N, ZTOP)[0])
        d = np.linalg.norm((qg[a:b] - qr[0]) / s) / np.linalg.norm((qr[0] - q0[a:b]) / s)
        worst = max(worst, d)
        n = b - a
        assert 1 <= kry[c] <= it[c].item() * n
    assert worst < 1e-10, worst


def test_gmres_paper_settings(hv):
    import torch
    classes = [(16, 3)]
    ncols = 64
    lam = tableaux.ARK2.gamma * 300.0
    cls, qs = _case(classes, ncols, seed=52)
    ctx = hv.Context(classes, ZTOP, ncols=ncols, precision=hv.FP32_IR)
    q0 = _pack(qs)
    q, R = _t(q0), _t(q0)
    kry = torch.zeros(ncols, dtype=torch.int32, device="cuda")
    ctx.hevi_newton_gmres_solve(lam, q, R, krylov=kry)
    st, it = ctx.hevi_column_status()
    assert bool((st == 0).all())
    qg = q.cpu().numpy().reshape(ncols, -1)
    q0r = q0.reshape(ncols, -1)
    qr, _, _ = oracle.newton(16, 3, ZTOP, lam, q0r, q0r, rtol=1e-12)
    _, ito, kito, sto = oracle.newton_gmres(16, 3, ZTOP, lam, q0r, q0r)
    assert (sto == 0).all()
    s = oracle.scales(oracle.column_grid(16, 3, ZTOP)[0])
    rel = np.linalg.norm((qg - qr) / s, axis=1) / np.linalg.norm((qr - q0r) / s, axis=1)
    assert rel.max() < 1e-3, rel.max()
    # the same algorithm: the same Newton count and nearly the same Krylov count
    assert np.array_equal(it.cpu().numpy(), ito)
    assert np.abs(kry.cpu().numpy() - kito).max() <= 3 * ito.max()


def test_gmres_and_lu_find_the_same_root(hv):
    classes = [(10, 4)]
    ncols = 32
    lam = tableaux.ARK2.gamma * 300.0
    cls, qs = _case(classes, ncols, seed=53)
    ctx = hv.Context(classes, ZTOP, ncols=ncols, precision=hv.FP32_IR)
    q0 = _pack(qs)
    qa, qb, R = _t(q0), _t(q0), _t(q0)
    ctx.hevi_newton_gmres_solve(lam, qa, R, eps=1e-7, rtol=1e-12, gtol=1e-12)
    ctx.hevi_newton_solve(lam, qb, R, rtol=1e-12)
    a = qa.cpu().numpy().reshape(ncols, -1)
    b = qb.cpu().numpy().reshape(ncols, -1)
    q0r = q0.reshape(ncols, -1)
    s = oracle.scales(oracle.column_grid(10, 4, ZTOP)[0])
    rel = np.linalg.norm((a - b) / s, axis=1) / np.linalg.norm((b - q0r) / s, axis=1)
    assert rel.max() < 1e-9, rel.max()
