"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics
(closed forms, invariants, brute force, library routines), none of them a
restatement of the oracle's own formulas.  CPU only."""

import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
from scipy.linalg import lapack

import oracle
from oracle import tableaux

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ZTOP = 30e3


def _rest(nez, N, ztop=ZTOP, ncols=1):
    return oracle.reference_q(nez, N, ztop, ncols)


def _perturbed_state(nez, N, seed=0, ztop=ZTOP, amp_w=5.0, amp_th=2.0):
    """A non-rest state: rest + random w (0 at both ends) and theta'."""
    g = np.random.default_rng(seed)
    q = _rest(nez, N, ztop)[0].reshape(-1, 3)
    nz = q.shape[0]
    w = g.uniform(-amp_w, amp_w, nz)
    w[0] = w[-1] = 0.0
    th = g.uniform(-amp_th, amp_th, nz)
    rho = q[:, 0] * (1 + 0.01 * g.uniform(-1, 1, nz))
    Theta = q[:, 2] / q[:, 0] * rho + rho * th
    return np.stack([rho, rho * w, Theta], 1).reshape(-1)


# --------------------------------------------------------------------------
# Sec. 3: LGL nodes, weights, differentiation matrix
# --------------------------------------------------------------------------

def test_lgl_order4_closed_form():
    xi, w = oracle.lgl(4)
    r = math.sqrt(3.0 / 7.0)
    np.testing.assert_allclose(xi, [-1, -r, 0, r, 1], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10], rtol=1e-15)


@pytest.mark.parametrize("N", range(1, 11))
def test_lgl_nodes_are_roots_of_dPN_and_quadrature_exact(N):
    xi, w = oracle.lgl(N)
    # interior nodes are the roots of P_N' (numpy's Legendre series)
    dP = np.polynomial.legendre.Legendre.basis(N).deriv()
    np.testing.assert_allclose(np.sort(dP.roots().real), xi[1:-1], atol=1e-13)
    # Lobatto quadrature with N+1 points is exact to degree 2N-1
    for p in range(2 * N):
        exact = 0.0 if p % 2 else 2.0 / (p + 1)
        assert abs(np.dot(w, xi**p) - exact) < 1e-13
    # ... and not exact at degree 2N (the inexact mass matrix of Sec. 3)
    assert abs(np.dot(w, xi ** (2 * N)) - 2.0 / (2 * N + 1)) > 1e-6


@pytest.mark.parametrize("N", range(1, 11))
def test_dmatrix_exact_rowsum_sbp(N):
    xi, w = oracle.lgl(N)
    D = oracle.dmatrix(N)
    # row-sum property (Sec. 3): derivative of a constant is zero
    np.testing.assert_allclose(D.sum(1), 0.0, atol=1e-12 * N * N)
    # exact on polynomials of degree <= N
    for p in range(N + 1):
        np.testing.assert_allclose(D @ xi**p, p * xi ** max(p - 1, 0) if p else 0 * xi,
                                   atol=1e-12 * N * N)
    # summation by parts: W D + D^T W = diag(-1, 0, ..., 0, 1)
    W = np.diag(w)
    B = np.zeros((N + 1, N + 1))
    B[0, 0], B[-1, -1] = -1.0, 1.0
    np.testing.assert_allclose(W @ D + D.T @ W, B, atol=1e-12 * N * N)


def test_dmatrix_matches_lgl_closed_form():
    # classical closed form for LGL points: D_kj = P_N(x_k) / (P_N(x_j)(x_k - x_j)),
    # D_00 = -N(N+1)/4, D_NN = N(N+1)/4, other diagonal entries 0
    for N in (2, 3, 4, 7):
        xi, _ = oracle.lgl(N)
        PN = np.polynomial.legendre.Legendre.basis(N)(xi)
        ref = np.zeros((N + 1, N + 1))
        for k in range(N + 1):
            for j in range(N + 1):
                if k != j:
                    ref[k, j] = PN[k] / (PN[j] * (xi[k] - xi[j]))
        ref[0, 0], ref[N, N] = -N * (N + 1) / 4, N * (N + 1) / 4
        np.testing.assert_allclose(oracle.dmatrix(N), ref, atol=1e-12)


@pytest.mark.parametrize("nez,N", [(1, 1), (3, 2), (8, 4), (10, 4), (16, 3), (24, 4)])
def test_grid_mass(nez, N):
    z, M = oracle.column_grid(nez, N, ZTOP)
    assert z.size == nez * N + 1
    assert np.all(np.diff(z) > 0) and z[0] == 0.0 and z[-1] == ZTOP
    assert abs(M.sum() - ZTOP) < 1e-10 * ZTOP
    # mass integrates polynomials in z of degree <= 2N-1 exactly on each element
    for p in range(2 * N):
        assert abs(np.dot(M, (z / ZTOP) ** p) - ZTOP / (p + 1)) < 1e-11 * ZTOP


# --------------------------------------------------------------------------
# Band structure of Sec. 4.2.3 (golden values of the paper's formulas)
# --------------------------------------------------------------------------

def test_band_structure_golden():
    with open(os.path.join(GOLDEN, "band_structure.json")) as f:
        gold = json.load(f)
    for row in gold["rows"]:
        nvar, N = row["n_var"], row["N"]
        assert nvar * (N + 1) - 1 == row["k_l"] == row["k_u"]
        assert 3 * nvar * (N + 1) - 2 == row["ldab"]
        if nvar == 3:
            # the assembled Jacobian lies inside the band and reaches k_l below
            # the diagonal (Theta-row, rho-column); above it reaches k_u - 1,
            # since the rho-row couples to m only
            nez = 3
            q = _perturbed_state(nez, N, seed=1)
            ab = oracle.assemble_band(nez, N, ZTOP, 50.0, q[None])[0]
            A = oracle.band_to_dense(ab, row["k_l"], row["k_u"])
            i, j = np.nonzero(A)
            assert (i - j).max() == row["k_l"] and (j - i).max() == row["k_u"] - 1


# --------------------------------------------------------------------------
# Reference state and operator invariants
# --------------------------------------------------------------------------

def test_reference_state_isothermal_closed_form():
    z, _ = oracle.column_grid(10, 4, ZTOP)
    rho, theta, Theta, P = oracle.reference_state(z)
    R, T0, p0, g = 287.17, 300.0, 1e5, 9.80616
    p_exact = p0 * np.exp(-g * z / (R * T0))
    np.testing.assert_allclose(P, p_exact, rtol=1e-12)       # EOS(Theta_bar) = p_bar
    np.testing.assert_allclose(rho * R * T0, p_exact, rtol=1e-14)
    # theta = T (p0/p)^(R/cp)
    np.testing.assert_allclose(theta, T0 * (p0 / p_exact) ** (R / 1004.67), rtol=1e-13)


@pytest.mark.parametrize("nez,N", [(1, 1), (2, 3), (8, 4), (16, 3), (24, 4)])
def test_rest_state_is_exact_equilibrium(nez, N):
    q = _rest(nez, N)
    assert np.array_equal(oracle.apply_V(nez, N, ZTOP, q), np.zeros_like(q))


@pytest.mark.parametrize("nez,N", [(2, 2), (8, 4), (16, 3)])
def test_column_mass_and_theta_conserved(nez, N):
    """Sec. 2.2 / 3: the divergence form conserves the column integrals of rho
    and Theta under LGL quadrature when m = 0 at both ends."""
    _, M = oracle.column_grid(nez, N, ZTOP)
    q = _perturbed_state(nez, N, seed=2)
    v = oracle.apply_V(nez, N, ZTOP, q)[0].reshape(-1, 3)
    scale_r = np.abs(M * q.reshape(-1, 3)[:, 0]).sum() / ZTOP
    assert abs(np.dot(M, v[:, 0])) < 1e-13 * scale_r * ZTOP
    assert abs(np.dot(M, v[:, 2])) < 1e-13 * scale_r * 300 * ZTOP
    g = np.random.default_rng(3)
    x = g.standard_normal(q.size).reshape(-1, 3)
    x[0, 1] = x[-1, 1] = 0.0
    y = oracle.apply_L(nez, N, ZTOP, q[None], x.reshape(1, -1))[0].reshape(-1, 3)
    assert abs(np.dot(M, y[:, 0])) < 1e-12 * np.abs(M[:, None] * y).sum()
    assert abs(np.dot(M, y[:, 2])) < 1e-12 * np.abs(M[:, None] * y).sum()


@pytest.mark.parametrize("nez,N", [(2, 2), (4, 4), (16, 3)])
def test_linear_operator_is_the_frechet_derivative(nez, N):
    """L(q0) x against central differences of the nonlinear V (pins every
    entry of the flux Jacobian, its signs and the gravity coupling)."""
    q0 = _perturbed_state(nez, N, seed=4)
    g = np.random.default_rng(5)
    s = oracle.scales(oracle.column_grid(nez, N, ZTOP)[0])
    x = s * g.standard_normal(q0.size)
    x[1] = x[-2] = 0.0
    L = oracle.apply_L(nez, N, ZTOP, q0[None], x[None])[0]
    eps = 1e-5
    fd = (oracle.apply_V(nez, N, ZTOP, (q0 + eps * x)[None])[0]
          - oracle.apply_V(nez, N, ZTOP, (q0 - eps * x)[None])[0]) / (2 * eps)
    assert np.linalg.norm(L - fd) <= 1e-7 * np.linalg.norm(L)


def test_operator_differentiates_polynomial_flux_exactly():
    """With rho = const and a polynomial momentum of degree <= N on each
    element, V_rho = -dm/dz exactly at every point (continuous derivative)."""
    nez, N = 3, 4
    z, _ = oracle.column_grid(nez, N, ZTOP)
    q = _rest(nez, N)[0].reshape(-1, 3)
    m = (z / ZTOP) * (1 - z / ZTOP) * 2.0        # degree 2, zero at both ends
    q[:, 1] = m
    v = oracle.apply_V(nez, N, ZTOP, q.reshape(1, -1))[0].reshape(-1, 3)
    dm = 2.0 * (1 - 2 * z / ZTOP) / ZTOP
    np.testing.assert_allclose(-v[:, 0], dm, atol=1e-14 * 2.0 / ZTOP * 100)


def test_assembly_matches_operator_columns():
    """Band column j of A equals e_j - Lambda L(q0) e_j (App. A.3 vs Sec. 4.3.1)."""
    nez, N, lam = 3, 4, 87.0
    q0 = _perturbed_state(nez, N, seed=6)
    _, n, k = oracle.sizes(nez, N)
    A = oracle.band_to_dense(oracle.assemble_band(nez, N, ZTOP, lam, q0[None])[0], k, k)
    E = np.eye(n)
    L = np.stack([oracle.apply_L(nez, N, ZTOP, q0[None], E[j][None])[0] for j in range(n)], 1)
    ref = np.eye(n) - lam * L
    # the boundary m-rows are identity rows (reading R3)
    for I in (0, n // 3 - 1):
        ref[3 * I + 1, :] = 0.0
        ref[3 * I + 1, 3 * I + 1] = 1.0
    np.testing.assert_allclose(A, ref, atol=1e-13 * np.abs(ref).max())


# --------------------------------------------------------------------------
# Band LU (Sec. 4.2.3) against LAPACK and dense brute force
# --------------------------------------------------------------------------

CASES = [(1, 1), (2, 1), (3, 2), (1, 4), (2, 4), (3, 3), (8, 4), (10, 4), (16, 3)]


@pytest.mark.parametrize("nez,N", CASES)
def test_band_lu_matches_lapack_and_dense(nez, N):
    _, n, k = oracle.sizes(nez, N)
    q0 = _perturbed_state(nez, N, seed=7 + nez)
    lam = 87.868
    ab = oracle.assemble_band(nez, N, ZTOP, lam, q0[None])[0].copy()
    ab_orig = ab.copy()
    A = oracle.band_to_dense(ab, k, k)
    lu_ref, piv_ref, info_ref = lapack.dgbtrf(np.asfortranarray(ab.T), k, k)
    info, piv = oracle.gbtrf(ab, k, k)
    assert info == info_ref == 0
    np.testing.assert_array_equal(piv, piv_ref)           # pivot sequence: reading R6
    np.testing.assert_allclose(ab.T, lu_ref, atol=1e-12 * np.abs(lu_ref).max())
    g = np.random.default_rng(8)
    b = g.standard_normal(n) * oracle.scales(oracle.column_grid(nez, N, ZTOP)[0])
    x = oracle.gbtrs(ab, k, k, piv, b)
    x_dense = np.linalg.solve(A, b)
    x_band = sla.solve_banded((k, k), ab_orig.T[k:, :], b)
    kappa = np.linalg.cond(A)
    assert np.linalg.norm(x - x_dense) <= 1e-15 * kappa * np.linalg.norm(x_dense) * 10
    assert np.linalg.norm(x - x_band) <= 1e-15 * kappa * np.linalg.norm(x_band) * 10
    assert np.linalg.norm(b - A @ x) <= 1e-14 * np.linalg.norm(b) * max(1.0, np.abs(A).max())


def test_band_lu_tie_break_first_maximum():
    """Equal-magnitude candidates: the first row wins, as LAPACK's i_amax."""
    n, kl, ku = 4, 1, 1
    A = np.array([[1.0, 2.0, 0, 0], [-1.0, 1.0, 3.0, 0], [0, 2.0, -2.0, 1.0], [0, 0, 2.0, 1.0]])
    ab = np.zeros((n, 2 * kl + ku + 1))
    for j in range(n):
        for i in range(max(0, j - ku), min(n, j + kl + 1)):
            ab[j, kl + ku + i - j] = A[i, j]
    _, piv_ref, _ = lapack.dgbtrf(np.asfortranarray(ab.T), kl, ku)
    info, piv = oracle.gbtrf(ab.copy(), kl, ku)
    np.testing.assert_array_equal(piv, piv_ref)
    assert piv[0] == 0


def test_band_lu_reports_singular_pivot():
    n, kl, ku = 3, 1, 1
    A = np.array([[1.0, 2.0, 0], [1.0, 2.0, 0.0], [0, 0, 1.0]])
    ab = np.zeros((n, 4))
    for j in range(n):
        for i in range(max(0, j - ku), min(n, j + kl + 1)):
            ab[j, kl + ku + i - j] = A[i, j]
    _, _, info_ref = lapack.dgbtrf(np.asfortranarray(ab.T), kl, ku)
    info, _ = oracle.gbtrf(ab.copy(), kl, ku)
    assert info == info_ref == 2


def test_stage_solve_identity_when_lambda_zero():
    nez, N = 8, 4
    q0 = _rest(nez, N)
    b = np.random.default_rng(9).standard_normal(q0.shape)
    x, info = oracle.stage_solve(nez, N, ZTOP, 0.0, q0, b)
    assert info[0] == 0
    np.testing.assert_array_equal(x, b)


def test_stage_solve_rest_zero_rhs_gives_zero():
    nez, N = 8, 4
    q0 = _rest(nez, N)
    x, _ = oracle.stage_solve(nez, N, ZTOP, 87.868, q0, np.zeros_like(q0))
    assert np.array_equal(x, np.zeros_like(q0))


def test_stage_solve_conserves_column_mass():
    import hevi_inputs
    inp = hevi_inputs.lhevi_stage(seed=11, ncols=4)
    nez, N = inp["nez"], inp["N"]
    q0 = _rest(nez, N, ZTOP, 4)
    x, info = oracle.stage_solve(nez, N, inp["ztop"], inp["lam"], q0, inp["b"])
    assert (info == 0).all()
    _, M = oracle.column_grid(nez, N, ZTOP)
    for c in range(4):
        xb, bb = x[c].reshape(-1, 3), inp["b"][c].reshape(-1, 3)
        tot = np.abs(M * bb[:, 2]).sum()
        assert abs(np.dot(M, xb[:, 0]) - np.dot(M, bb[:, 0])) < 1e-13 * tot
        assert abs(np.dot(M, xb[:, 2]) - np.dot(M, bb[:, 2])) < 1e-13 * tot
        # identity m-rows at both ends; pivoting may reorder them, so zero to rounding
        assert abs(xb[0, 1]) < 1e-15 * np.abs(xb[:, 1]).max()
        assert abs(xb[-1, 1]) < 1e-15 * np.abs(xb[:, 1]).max()


# --------------------------------------------------------------------------
# Newton (Sec. 4.2.3) and its relation to LHEVI (Sec. 4.3)
# --------------------------------------------------------------------------

def test_newton_at_rest_takes_no_step():
    nez, N = 16, 3
    q = _rest(nez, N)
    out, it, st = oracle.newton(nez, N, ZTOP, 87.0, q, q)
    assert it[0] == 0 and st[0] == 0 and np.array_equal(out, q)


def test_one_newton_iteration_is_the_lhevi_solve():
    """Sec. 4.3: LHEVI-PS is NHEVI-LU with one Newton iteration: from q0,
    (I - Lambda L(q0)) q1 = R + Lambda (V(q0) - L(q0) q0)."""
    nez, N, lam = 8, 4, 87.868
    q0 = _perturbed_state(nez, N, seed=12)[None]
    R = q0 + 0.01 * oracle.scales(oracle.column_grid(nez, N, ZTOP)[0])[None] * \
        np.random.default_rng(13).standard_normal(q0.shape)
    R[0, 1] = R[0, -2] = 0.0
    q1, it, st = oracle.newton(nez, N, ZTOP, lam, R, q0, rtol=0.0, max_iter=1)
    assert it[0] == 1
    b = R + lam * (oracle.apply_V(nez, N, ZTOP, q0) - oracle.apply_L(nez, N, ZTOP, q0, q0))
    x, _ = oracle.stage_solve(nez, N, ZTOP, lam, q0, b)
    np.testing.assert_allclose(q1, x, rtol=1e-12, atol=1e-12 * np.abs(q0).max())


def test_newton_converges_quadratically():
    nez, N, lam = 8, 4, 87.868
    q0 = _perturbed_state(nez, N, seed=14, amp_w=20.0, amp_th=5.0)[None]
    s = oracle.scales(oracle.column_grid(nez, N, ZTOP)[0])
    R = q0.copy()

    def fnorm(q):
        F = q - lam * oracle.apply_V(nez, N, ZTOP, q) - R
        return np.linalg.norm(F / s)
    norms = [fnorm(q0)]
    for m in range(1, 5):
        q, it, st = oracle.newton(nez, N, ZTOP, lam, R, q0, rtol=0.0, max_iter=m)
        norms.append(fnorm(q))
    norms = np.array(norms) / norms[0]
    # quadratic: e_{m+1} <= C e_m^2 with a bounded C, down to the rounding floor
    for m in range(3):
        assert norms[m + 1] <= 10.0 * norms[m] ** 2, norms
    assert norms[4] < 1e-13, norms


def test_newton_restart_from_root_stops_at_rounding_floor():
    """Reading R7: restarted from its own root, Newton has |F(q_0)| at the
    rounding level of the FP64 residual, where the relative test
    |F(q_m)| <= rtol |F(q_0)| cannot be met; the rounding floor
    |S^-1 F| <= 512 eps |S^-1 q| stops it at once, converged.  Stiffest
    class of the workloads (Nez = 24, N = 4, 30 km top: acoustic Courant
    number ~480 at dt = 300 s)."""
    nez, N, lam = 24, 4, 87.868
    q0 = _perturbed_state(nez, N, seed=16, amp_w=1.0, amp_th=0.5)[None]
    R = q0.copy()
    root, it, st = oracle.newton(nez, N, ZTOP, lam, R, q0, rtol=1e-10, max_iter=20)
    assert st[0] == 0 and 1 <= it[0] <= 8
    s = oracle.scales(oracle.column_grid(nez, N, ZTOP)[0])
    F = root - lam * oracle.apply_V(nez, N, ZTOP, root) - R
    assert np.linalg.norm(F / s) <= 512 * np.finfo(float).eps * np.linalg.norm(root / s)
    again, it2, st2 = oracle.newton(nez, N, ZTOP, lam, R, root, rtol=1e-10, max_iter=20)
    assert st2[0] == 0 and it2[0] == 0 and np.array_equal(again, root)
    # with the relative test alone (floor below rounding) it would not stop:
    # one more update moves the root by no more than rounding
    moved, it3, _ = oracle.newton(nez, N, ZTOP, lam, R, root, rtol=0.0, max_iter=1)
    assert it3[0] == 0 or np.linalg.norm((moved - root) / s) < 1e-12


# --------------------------------------------------------------------------
# NHEVI-GMRES (Sec. 4.2.1): Jacobian-free Newton-Krylov
# --------------------------------------------------------------------------

@pytest.mark.parametrize("nez,N", [(16, 3), (10, 4)])
def test_newton_gmres_reaches_the_lu_root(nez, N):
    """With a small Frechet perturbation and tight tolerances JFNK-GMRES and
    Newton-LU find the same root of F; GMRES needs at most n iterations per
    Newton step (unrestarted GMRES is exact after n)."""
    lam = tableaux.ARK2.gamma * 300.0
    q0 = _perturbed_state(nez, N, seed=41, amp_w=1.0, amp_th=0.5)[None]
    R = q0.copy()
    n = q0.shape[1]
    q, it, kit, st = oracle.newton_gmres(nez, N, ZTOP, lam, R, q0, eps=1e-7, rtol=1e-12,
                                         gtol=1e-12)
    qr, _, str_ = oracle.newton(nez, N, ZTOP, lam, R, q0, rtol=1e-12)
    assert st[0] == 0 and str_[0] == 0
    s = oracle.scales(oracle.column_grid(nez, N, ZTOP)[0])
    assert np.linalg.norm((q - qr)[0] / s) < 1e-10 * np.linalg.norm((qr - q0)[0] / s)
    assert 1 <= it[0] <= 6 and it[0] <= kit[0] <= it[0] * n


def test_one_gmres_newton_step_is_one_lu_newton_step():
    """One Newton update with a tiny perturbation and a tight GMRES tolerance
    solves the same linear system as one Newton-LU update: the two agree to
    the Frechet difference error (Eq. Frechet-derivative)."""
    nez, N = 8, 4
    lam = 87.868
    q0 = _perturbed_state(nez, N, seed=42, amp_w=2.0, amp_th=1.0)[None]
    R = q0 + 1e-3 * oracle.scales(oracle.column_grid(nez, N, ZTOP)[0])[None]
    R[0, 1] = R[0, -2] = 0.0
    q1, it, kit, st = oracle.newton_gmres(nez, N, ZTOP, lam, R, q0, eps=1e-8, rtol=0.0,
                                          gtol=1e-13, max_newton=1)
    ql, itl, _ = oracle.newton(nez, N, ZTOP, lam, R, q0, rtol=0.0, max_iter=1)
    assert it[0] == 1 and itl[0] == 1
    d_lu = np.linalg.norm(ql - q0)
    assert np.linalg.norm(q1 - ql) < 1e-6 * d_lu


def test_newton_gmres_paper_settings_converge():
    """The configuration of the paper's timing table (eps = 0.05, Newton
    tolerance 1e-5, GMRES tolerance 1e-9): converged, with the residual
    reduced 1e5-fold and the root within that tolerance of the LU root."""
    nez, N = 16, 3
    lam = tableaux.ARK2.gamma * 300.0
    q0 = _perturbed_state(nez, N, seed=43, amp_w=1.0, amp_th=0.5)[None]
    R = q0.copy()
    q, it, kit, st = oracle.newton_gmres(nez, N, ZTOP, lam, R, q0)
    assert st[0] == 0
    s = oracle.scales(oracle.column_grid(nez, N, ZTOP)[0])
    F0 = q0 - lam * oracle.apply_V(nez, N, ZTOP, q0) - R
    F = q - lam * oracle.apply_V(nez, N, ZTOP, q) - R
    assert np.linalg.norm(F[0] / s) <= 1e-5 * np.linalg.norm(F0[0] / s)
    qr, _, _ = oracle.newton(nez, N, ZTOP, lam, R, q0, rtol=1e-12)
    assert np.linalg.norm((q - qr)[0] / s) < 1e-3 * np.linalg.norm((qr - q0)[0] / s)


def test_newton_linear_problem_one_iteration():
    """Sec. 4.3: LHEVI is NHEVI-LU with one Newton iteration.  For the linear
    problem V := L_RS (q - q_bar), F(q) = q - Lambda V(q) - R is affine with
    the constant Jacobian J = I - Lambda L_RS, so one Newton step from any
    guess lands on the root, and the root is the LHEVI solve about the rest
    state: q = q_bar + (I - Lambda L_RS)^-1 (R - q_bar).  The step is built
    from apply_L (the matrix-free operator) and the solve with the assembled,
    LU-factored band, two independent code paths."""
    nez, N, lam = 4, 4, 87.868
    q_bar = _rest(nez, N).reshape(-1)
    s = oracle.scales(oracle.column_grid(nez, N, ZTOP)[0])
    g = np.random.default_rng(15)
    R = q_bar + 1e-3 * s * g.standard_normal(q_bar.size)
    R[1] = R[-2] = 0.0
    guess = q_bar + 1e-2 * s * g.standard_normal(q_bar.size)
    guess[1] = guess[-2] = 0.0

    def F(q):
        return q - lam * oracle.apply_L(nez, N, ZTOP, q_bar, (q - q_bar)[None])[0] - R

    delta, info = oracle.stage_solve(nez, N, ZTOP, lam, q_bar, -F(guess)[None])
    assert info[0] == 0
    q1 = guess + delta[0]
    x, _ = oracle.stage_solve(nez, N, ZTOP, lam, q_bar, (R - q_bar)[None])
    q_lhevi = q_bar + x[0]
    # rounding of O(1) scaled states (~1e-14); a wrong operator entry is O(1e-3)
    assert np.linalg.norm((q1 - q_lhevi) / s) < 1e-10 * np.linalg.norm((q_lhevi - q_bar) / s)
    # the step lands on the root: the residual is at rounding level
    assert np.linalg.norm(F(q1) / s) < 1e-10 * np.linalg.norm(F(guess) / s)


def _hydrostatic_perturbation(nez, N, eps=0.01):
    """A discretely smooth hydrostatic perturbation of the rest state: Theta' =
    eps Theta_bar sin(pi z / z_top), P' = EOS(Theta_bar + Theta') - P_bar (App.
    A.1), and rho' = -(1/g) dP'/dz from the analytic derivative; m = 0."""
    T0, p0, Rg, cp, g = 300.0, 1e5, 287.17, 1004.67, 9.80616
    gam = cp / (cp - Rg)
    Hs = Rg * T0 / g
    z = oracle.column_grid(nez, N, ZTOP)[0]
    q = _rest(nez, N).reshape(-1, 3)
    rb, Tb = q[:, 0], q[:, 2]
    Pb = p0 * (Rg * Tb / p0) ** gam
    x = eps * np.sin(np.pi * z / ZTOP)
    dx = eps * np.pi / ZTOP * np.cos(np.pi * z / ZTOP)
    dTb = Tb * (-1.0 / Hs + g / (cp * T0))
    dPb = gam * Pb / Tb * dTb
    dPp = dPb * ((1 + x) ** gam - 1) + Pb * gam * (1 + x) ** (gam - 1) * dx
    rp = -dPp / g
    return np.stack([rb + rp, 0 * rb, Tb * (1 + x)], -1).reshape(-1), rp, g


def test_gravity_balances_pressure_gradient_at_spectral_rate():
    """The gravity term of the m equation (App. A.2, reference subtracted):
    for a hydrostatic perturbation (dP'/dz = -g rho', m = 0) the vertical
    momentum tendency V_m = -Dcal[P'] - g rho' vanishes up to the spectral
    derivative's error, which falls with the element size and with the
    order.  A gravity term of the wrong sign or size leaves V_m ~ g rho'."""
    def err(nez, N):
        qs, rp, g = _hydrostatic_perturbation(nez, N)
        V = oracle.apply_V(nez, N, ZTOP, qs[None])[0].reshape(-1, 3)
        return np.abs(V[1:-1, 1]).max() / np.abs(g * rp).max()
    h = [err(nez, 4) for nez in (2, 4, 8, 16)]
    for a, b in zip(h, h[1:]):
        assert b < a / 6.0, h           # algebraic convergence in the element size
    assert h[-1] < 1e-5, h
    p = [err(8, N) for N in (2, 3, 4, 5)]
    for a, b in zip(p, p[1:]):
        assert b < a / 8.0, p           # and in the order
    assert p[-1] < 1e-5, p


# --------------------------------------------------------------------------
# ARK tableaux (Sec. 4.1, Sec. 6): order conditions of additive RK methods
# --------------------------------------------------------------------------

def _bicolored_trees(order):
    """All rooted trees with <= order vertices whose non-root vertices carry
    a colour (0 explicit, 1 implicit); a tree is (colour, tuple(children))."""
    from itertools import combinations_with_replacement
    by_size = {1: [(None, ())]}

    def colored(size):
        return [(c, ch) for (_, ch) in by_size[size] for c in (0, 1)]
    for size in range(2, order + 1):
        out = []
        # partitions of size-1 into child sizes
        def parts(rem, maxp):
            if rem == 0:
                yield ()
                return
            for p in range(min(rem, maxp), 0, -1):
                for rest in parts(rem - p, p):
                    yield (p,) + rest
        for part in parts(size - 1, size - 1):
            pools = [sorted(set(colored(p)), key=repr) for p in part]
            # multiset of children: group equal sizes
            def build(i, acc):
                if i == len(part):
                    yield tuple(sorted(acc, key=repr))
                    return
                for t in pools[i]:
                    if i > 0 and part[i] == part[i - 1] and repr(t) < repr(acc[-1]):
                        continue
                    yield from build(i + 1, acc + [t])
            for ch in build(0, []):
                out.append((None, ch))
        by_size[size] = sorted(set(out), key=repr)
    return by_size


def _phi(tree, A, At):
    s = A.shape[0]
    v = np.ones(s)
    for ch in tree[1]:
        M = A if ch[0] == 0 else At
        v = v * (M @ _phi(ch, A, At))
    return v


def _gamma(tree):
    def size(t):
        return 1 + sum(size(c) for c in t[1])
    g = size(tree)
    for ch in tree[1]:
        g *= _gamma(ch)
    return g


@pytest.mark.parametrize("name", ["ARK2", "ARK3", "ARK4", "ARS3"])
def test_tableau_structure_and_order_conditions(name):
    t = tableaux.ALL[name]
    A, At, b = t.A, t.At, t.b
    s = t.s
    assert np.allclose(np.triu(A), 0)                       # explicit: strictly lower
    assert np.allclose(np.triu(At, 1), 0)                   # implicit: lower
    assert At[0, 0] == 0.0                                  # first stage explicit
    assert np.allclose(np.diag(At)[1:], t.gamma)            # singly diagonal
    np.testing.assert_allclose(A.sum(1), At.sum(1), atol=1e-15)
    trees = _bicolored_trees(t.order)
    count = 0
    for size in range(1, t.order + 1):
        for tree in trees[size]:
            lhs = b @ _phi(tree, A, At)
            assert abs(lhs - 1.0 / _gamma(tree)) < 1e-14, (name, tree)
            count += 1
    # number of trees with two-coloured non-root vertices: 3, 10, 36 up to order 2, 3, 4
    assert count == {2: 3, 3: 10, 4: 36}[t.order]


def test_ars3_published_values():
    """ARS(3,4,3) (Ascher, Ruuth & Spiteri 1997) at the digits the construction
    publishes, and the singly diagonal L-stable gamma: R(inf) = 0 of its
    implicit part."""
    t = tableaux.ARS3
    assert abs(t.gamma - 0.4358665215) < 1e-10
    np.testing.assert_allclose(t.A[2, :2], [0.3212788860, 0.3966543747], atol=1e-10)
    np.testing.assert_allclose(t.A[3, :3], [-0.105858296, 0.5529291479, 0.5529291479], atol=1e-9)
    np.testing.assert_allclose(t.b, [0.0, 1.208496649, -0.644363171, 0.4358665215], atol=1e-9)
    np.testing.assert_allclose(t.c, [0.0, t.gamma, (1 + t.gamma) / 2, 1.0], atol=1e-15)
    # stiff decay: the implicit stages 2..4 form an L-stable SDIRK, R(inf) = 0
    Ai = t.At[1:, 1:]
    bi = t.b[1:]
    r_inf = 1.0 - bi @ np.linalg.solve(Ai, np.ones(3))
    assert abs(r_inf) < 1e-14


def test_ark2_gamma_and_a32():
    t = tableaux.ARK2
    assert abs(t.gamma - (1 - 1 / math.sqrt(2))) < 1e-16
    assert t.A[2, 1] == 0.5                                 # ARK(2,3,2)b, Sec. 4.1


# --------------------------------------------------------------------------
# Time integration: linear closed form and nonlinear self-convergence
# --------------------------------------------------------------------------

def _linear_exact(nez, N, q_bar, dq0, H, T):
    """dq'/dt = L_RS q' + H, solved with the exponential of the augmented
    matrix [[L, H], [0, 0]]."""
    _, n, _ = oracle.sizes(nez, N)
    E = np.eye(n)
    L = np.stack([oracle.apply_L(nez, N, ZTOP, q_bar, E[j][None])[0] for j in range(n)], 1)
    aug = np.zeros((n + 1, n + 1))
    aug[:n, :n] = L
    aug[:n, n] = H
    y = sla.expm(T * aug) @ np.concatenate([dq0, [1.0]])
    return y[:n]


@pytest.mark.parametrize("name", ["ARK2", "ARK3", "ARK4", "ARS3"])
def test_ark_linear_problem_converges_at_order(name):
    tab = tableaux.ALL[name]
    nez, N = 4, 4
    q_bar = _rest(nez, N)
    z, _ = oracle.column_grid(nez, N, ZTOP)
    rho, _, _, _ = oracle.reference_state(z)
    dq0 = np.zeros((z.size, 3))
    dq0[:, 2] = rho * 1.0 * np.sin(np.pi * z / ZTOP)      # 1 K theta' (IGW profile, Sec. 7.2)
    dq0 = dq0.reshape(-1)
    H = np.zeros_like(dq0)
    H[2::3] = 1e-4 * rho
    # the sin profile is not balanced, so it excites acoustic modes with
    # |lambda| up to 0.38 s^-1 on this column; the asymptotic regime needs
    # steps that resolve them
    T = 8.0
    exact = _linear_exact(nez, N, q_bar, dq0, H, T)
    errs = []
    dts = [2.0, 1.0, 0.5]
    for dt in dts:
        q = q_bar + dq0
        for _ in range(int(round(T / dt))):
            q, info = oracle.lhevi_step(nez, N, ZTOP, tab, dt, q, H[None], lin=2)
            assert info[0] == 0
        errs.append(np.linalg.norm(q[0] - q_bar[0] - exact) / np.linalg.norm(exact))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert min(rates) > tab.order - 0.35, (errs, rates)


def test_lhevi_about_own_state_and_rest_equal_ps_and_rs():
    """The Jacobian-state entry point reduces to LHEVI-PS for q_lin = q^n and
    to LHEVI-RS for q_lin = q_bar, bit for bit."""
    nez, N, dt = 8, 4, 300.0
    qn = _perturbed_state(nez, N, seed=31, amp_w=1.0, amp_th=0.5)[None]
    H = np.zeros_like(qn)
    H[0, 2::3] = 1e-6 * qn[0, 2::3]
    for lin, ql in ((0, qn), (1, _rest(nez, N))):
        ref, _ = oracle.lhevi_step(nez, N, ZTOP, tableaux.ARK3, dt, qn, H, lin=lin)
        got, _ = oracle.lhevi_step(nez, N, ZTOP, tableaux.ARK3, dt, qn, H, lin=0, q_lin=ql)
        assert np.array_equal(ref, got), lin


@pytest.mark.parametrize("name", ["ARK2", "ARK3"])
def test_lagged_jacobian_keeps_order_on_linear_problem(name):
    """Jacobian update interval (Sec. 4.3, the update time-step of Sec. 7.1):
    the implicit operator is L(q_lin) of a state other than the one the ODE is
    linear about, so L and V - L are a different IMEX splitting of the same
    linear problem dq'/dt = L_RS q' + H; the ARK pair still converges at its
    order to the exact (matrix exponential) solution."""
    tab = tableaux.ALL[name]
    nez, N = 4, 4
    q_bar = _rest(nez, N)
    z, _ = oracle.column_grid(nez, N, ZTOP)
    rho, _, _, _ = oracle.reference_state(z)
    dq0 = np.zeros((z.size, 3))
    dq0[:, 2] = rho * 1.0 * np.sin(np.pi * z / ZTOP)
    dq0 = dq0.reshape(-1)
    H = np.zeros_like(dq0)
    H[2::3] = 1e-4 * rho
    q_lin = _perturbed_state(nez, N, seed=32, amp_w=3.0, amp_th=2.0)[None]
    T = 8.0
    exact = _linear_exact(nez, N, q_bar, dq0, H, T)
    errs = []
    for dt in (2.0, 1.0, 0.5):
        q = q_bar + dq0
        for _ in range(int(round(T / dt))):
            q, info = oracle.lhevi_step(nez, N, ZTOP, tab, dt, q, H[None], lin=2, q_lin=q_lin)
            assert info[0] == 0
        errs.append(np.linalg.norm(q[0] - q_bar[0] - exact) / np.linalg.norm(exact))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > tab.order - 0.35, (errs, rates)
    # and it is a different method: the step differs from the L_RS splitting
    q1, _ = oracle.lhevi_step(nez, N, ZTOP, tab, 1.0, q_bar + dq0, H[None], lin=2)
    q2, _ = oracle.lhevi_step(nez, N, ZTOP, tab, 1.0, q_bar + dq0, H[None], lin=2, q_lin=q_lin)
    assert np.linalg.norm(q1 - q2) > 1e-8 * np.linalg.norm(q1 - q_bar - dq0)


@pytest.mark.slow
@pytest.mark.parametrize("name,variant", [("ARK2", "lhevi"), ("ARK3", "lhevi"),
                                          ("ARK2", "nhevi"), ("ARK3", "nhevi")])
def test_nonlinear_wave_self_convergence(name, variant):
    """1-D nonlinear acoustic-gravity wave (theta' = 1 K sin(pi z / z_top)):
    LHEVI-PS and NHEVI-LU steps converge at the tableau's order against a
    fine-step solution of the same method."""
    tab = tableaux.ALL[name]
    nez, N = 4, 4
    q_bar = _rest(nez, N)
    z, _ = oracle.column_grid(nez, N, ZTOP)
    rho, _, _, _ = oracle.reference_state(z)
    dq0 = np.zeros((z.size, 3))
    dq0[:, 2] = rho * 5.0 * np.sin(np.pi * z / ZTOP)
    q0 = q_bar + dq0.reshape(1, -1)
    H = np.zeros_like(q0)
    T = 8.0

    def run(dt):
        q = q0.copy()
        for _ in range(int(round(T / dt))):
            if variant == "lhevi":
                q, info = oracle.lhevi_step(nez, N, ZTOP, tab, dt, q, H, lin=0)
            else:
                q, it, st = oracle.nhevi_step(nez, N, ZTOP, tab, dt, q, H, rtol=1e-10)
                assert st[0] == 0
        return q
    ref = run(1.0 / 32)
    errs = [np.linalg.norm(run(dt) - ref) / np.linalg.norm(ref - q0) for dt in (2.0, 1.0, 0.5)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > tab.order - 0.4, (errs, rates)


@pytest.mark.parametrize("name", ["ARK2", "ARK3"])
def test_lhevi_ark_form_equals_direct_stage_form(name):
    """Sec. 4.3: the ARK form (Eq. lhevi-ark-final-3, solving for q_tt) and the
    direct stage form (I - gamma dt L) Q_i = q^n + dt sum_j [a_ij E(Q_j) +
    at_ij L Q_j], E = H + V - L, give the same step (built here from the
    oracle's stage solve and operator applies)."""
    tab = tableaux.ALL[name]
    nez, N, dt = 4, 4, 300.0
    s = tab.s
    qn = _perturbed_state(nez, N, seed=21, amp_w=3.0, amp_th=1.0)[None]
    sc = oracle.scales(oracle.column_grid(nez, N, ZTOP)[0])
    H = 1e-6 * sc[None] * np.random.default_rng(22).standard_normal(qn.shape)
    H[0, 1] = H[0, -2] = 0.0
    lam = tab.gamma * dt
    Q, E, LQ = [qn], [], []
    for i in range(s):
        if i > 0:
            rhs = qn + dt * sum(tab.A[i, j] * E[j] + tab.At[i, j] * LQ[j] for j in range(i))
            Qi, info = oracle.stage_solve(nez, N, ZTOP, lam, qn, rhs)
            Q.append(Qi)
        LQ.append(oracle.apply_L(nez, N, ZTOP, qn, Q[i]))
        E.append(H + oracle.apply_V(nez, N, ZTOP, Q[i]) - LQ[i])
    direct = qn + dt * sum(tab.b[i] * (E[i] + LQ[i]) for i in range(s))
    ark, info = oracle.lhevi_step(nez, N, ZTOP, tab, dt, qn, H, lin=0)
    assert info[0] == 0
    d = np.linalg.norm(ark - direct) / np.linalg.norm(direct - qn)
    assert d < 1e-10, d


# --------------------------------------------------------------------------
# Set 3C (App. A.1, Eq. set3c; reading R16): unknowns (rho, m, E)
# --------------------------------------------------------------------------

GAMMA = 1004.67 / (1004.67 - 287.17)
CV = 1004.67 - 287.17
G = 9.80616


def _state_3c(nez, N, seed=0, ztop=ZTOP, amp_w=5.0, amp_t=2.0):
    """A non-rest set-3C state built from (rho, w, T): rest density times
    1 +- 1%, w uniform (0 at both ends), T = 300 K +- amp_t; E = rho cv T +
    rho w^2 / 2 + rho g z (internal, kinetic, potential)."""
    g = np.random.default_rng(seed)
    z = oracle.column_grid(nez, N, ztop)[0]
    rho0 = _rest(nez, N, ztop)[0].reshape(-1, 3)[:, 0]
    rho = rho0 * (1 + 0.01 * g.uniform(-1, 1, z.size))
    w = g.uniform(-amp_w, amp_w, z.size)
    w[0] = w[-1] = 0.0
    T = 300.0 + g.uniform(-amp_t, amp_t, z.size)
    E = rho * CV * T + rho * w * w / 2 + rho * G * z
    return np.stack([rho, rho * w, E], 1).reshape(-1)


def test_set3c_rest_state_closed_form_and_equilibrium():
    """The set-3C rest state is the isothermal atmosphere with E = rho cv T0 +
    rho g z (no kinetic energy), and V of it vanishes exactly."""
    nez, N = 8, 4
    z = oracle.column_grid(nez, N, ZTOP)[0]
    with oracle.equation_set(oracle.SET_3C):
        q = _rest(nez, N)
        v = oracle.apply_V(nez, N, ZTOP, q)
    q3 = q[0].reshape(-1, 3)
    rho = 1e5 / (287.17 * 300.0) * np.exp(-z * G / (287.17 * 300.0))
    np.testing.assert_allclose(q3[:, 0], rho, rtol=1e-13)
    np.testing.assert_allclose(q3[:, 2], rho * CV * 300.0 + rho * G * z, rtol=1e-13)
    assert np.array_equal(v, np.zeros_like(v))


@pytest.mark.parametrize("nez,N", [(2, 2), (8, 4), (16, 3)])
def test_set3c_conserves_column_mass_and_total_energy(nez, N):
    """Set 3C is in divergence form with no energy source: with m = 0 at both
    ends the LGL column integrals of V_rho and V_E vanish (App. A.1)."""
    _, M = oracle.column_grid(nez, N, ZTOP)
    q = _state_3c(nez, N, seed=21)
    with oracle.equation_set(oracle.SET_3C):
        v = oracle.apply_V(nez, N, ZTOP, q[None])[0].reshape(-1, 3)
    q3 = q.reshape(-1, 3)
    assert abs(np.dot(M, v[:, 0])) < 1e-13 * np.abs(M * q3[:, 0]).sum()
    assert abs(np.dot(M, v[:, 2])) < 1e-13 * np.abs(M * q3[:, 2]).sum()


@pytest.mark.parametrize("nez,N", [(2, 2), (8, 4), (16, 3)])
def test_set3c_mass_and_momentum_tendencies_equal_set2c(nez, N):
    """The same physical state written in both sets (Theta = rho theta from the
    same p and rho, E = p/(gamma-1) + m^2/(2 rho) + rho g z) gets the same
    continuity and momentum tendencies: both sets carry m and m^2/rho + p."""
    g = np.random.default_rng(22)
    z = oracle.column_grid(nez, N, ZTOP)[0]
    q3 = _state_3c(nez, N, seed=23).reshape(-1, 3)
    rho, m, E = q3[:, 0], q3[:, 1], q3[:, 2]
    p = (GAMMA - 1) * (E - m * m / (2 * rho) - rho * G * z)
    theta = p / (rho * 287.17) * (1e5 / p) ** (287.17 / 1004.67)
    q2 = np.stack([rho, m, rho * theta], 1).reshape(1, -1)
    v2 = oracle.apply_V(nez, N, ZTOP, q2)[0].reshape(-1, 3)
    with oracle.equation_set(oracle.SET_3C):
        v3 = oracle.apply_V(nez, N, ZTOP, q3.reshape(1, -1))[0].reshape(-1, 3)
    np.testing.assert_allclose(v3[:, 0], v2[:, 0], rtol=0, atol=1e-12 * np.abs(v2[:, 0]).max())
    np.testing.assert_allclose(v3[:, 1], v2[:, 1], rtol=0, atol=1e-9 * np.abs(v2[:, 1]).max())
    del g


@pytest.mark.parametrize("nez,N", [(2, 2), (4, 4), (16, 3)])
def test_set3c_linear_operator_is_the_frechet_derivative(nez, N):
    """L(q0) x against central differences of the set-3C V: pins every entry
    of the set-3C flux Jacobian (App. A.3, Eq. set3c_jacobian) and the gravity
    coupling."""
    q0 = _state_3c(nez, N, seed=24)
    g = np.random.default_rng(25)
    with oracle.equation_set(oracle.SET_3C):
        s = oracle.scales(oracle.column_grid(nez, N, ZTOP)[0])
        x = s * g.standard_normal(q0.size)
        x[1] = x[-2] = 0.0
        L = oracle.apply_L(nez, N, ZTOP, q0[None], x[None])[0]
        eps = 1e-5
        fd = (oracle.apply_V(nez, N, ZTOP, (q0 + eps * x)[None])[0]
              - oracle.apply_V(nez, N, ZTOP, (q0 - eps * x)[None])[0]) / (2 * eps)
    assert np.linalg.norm(L - fd) <= 1e-7 * np.linalg.norm(L)


def test_set3c_hydrostatic_state_at_spectral_rate():
    """An isothermal atmosphere at another temperature (T1 = 250 K) is in
    hydrostatic balance, dp/dz = -rho g; written in set 3C its momentum
    tendency is the discretisation error of that balance, which falls at a
    spectral rate with N (pins the pressure recovered from E and the sign of
    the gravity term)."""
    T1 = 250.0
    errs = []
    for N in (2, 4, 6, 8):
        nez = 3
        z = oracle.column_grid(nez, N, ZTOP)[0]
        p = 1e5 * np.exp(-z * G / (287.17 * T1))
        rho = p / (287.17 * T1)
        q = np.stack([rho, np.zeros_like(rho), p / (GAMMA - 1) + rho * G * z], 1).reshape(1, -1)
        with oracle.equation_set(oracle.SET_3C):
            v = oracle.apply_V(nez, N, ZTOP, q)[0].reshape(-1, 3)
        errs.append(np.abs(v[:, 1]).max() / (rho.max() * G))
        assert np.abs(v[:, 0]).max() == 0.0 and np.abs(v[:, 2]).max() == 0.0
    assert errs[0] > 10 * errs[1] > 100 * errs[2], errs
    assert errs[3] < 1e-8, errs


def test_set3c_one_newton_iteration_is_the_lhevi_solve():
    """Sec. 4.3 for set 3C: one Newton iteration on F(q) = q - Lambda V(q) - R
    from q0 solves (I - Lambda L(q0)) q1 = R + Lambda (V(q0) - L(q0) q0)."""
    nez, N, lam = 8, 4, 87.868
    q0 = _state_3c(nez, N, seed=26)[None]
    with oracle.equation_set(oracle.SET_3C):
        R = q0 + 0.01 * oracle.scales(oracle.column_grid(nez, N, ZTOP)[0])[None] * \
            np.random.default_rng(27).standard_normal(q0.shape)
        R[0, 1] = R[0, -2] = 0.0
        q1, it, st = oracle.newton(nez, N, ZTOP, lam, R, q0, rtol=0.0, max_iter=1)
        assert it[0] == 1
        b = R + lam * (oracle.apply_V(nez, N, ZTOP, q0) - oracle.apply_L(nez, N, ZTOP, q0, q0))
        x, info = oracle.stage_solve(nez, N, ZTOP, lam, q0, b)
    assert (info == 0).all()
    np.testing.assert_allclose(q1, x, rtol=1e-12, atol=1e-12 * np.abs(q0).max())


def test_set3c_newton_converges_quadratically():
    nez, N, lam = 8, 4, 87.868
    q0 = _state_3c(nez, N, seed=28, amp_w=20.0, amp_t=5.0)[None]
    with oracle.equation_set(oracle.SET_3C):
        s = oracle.scales(oracle.column_grid(nez, N, ZTOP)[0])
        R = q0.copy()

        def fnorm(q):
            return np.linalg.norm((q - lam * oracle.apply_V(nez, N, ZTOP, q) - R) / s)
        norms = [fnorm(q0)]
        for m in range(1, 5):
            q, it, st = oracle.newton(nez, N, ZTOP, lam, R, q0, rtol=0.0, max_iter=m)
            norms.append(fnorm(q))
    norms = np.array(norms) / norms[0]
    for m in range(3):
        assert norms[m + 1] <= 10.0 * norms[m] ** 2, norms
    assert norms[4] < 1e-12, norms


@pytest.mark.parametrize("nez,N", [(8, 4), (24, 4)])
def test_set3c_stage_solve_matches_refined_dense_solve(nez, N):
    """The set-3C stage solve (band LU of the equilibrated system) against a
    dense LAPACK solve of the same matrix (numpy, equilibrated) refined three
    times with residuals in extended precision: 1e-12."""
    lam = 87.868
    q0 = _state_3c(nez, N, seed=29, amp_w=5.0, amp_t=2.0)[None]
    kl = 3 * (N + 1) - 1
    with oracle.equation_set(oracle.SET_3C):
        s = oracle.scales(oracle.column_grid(nez, N, ZTOP)[0])
        b = q0 + 1e-2 * s * np.random.default_rng(30).standard_normal(q0.shape)
        b[0, 1] = b[0, -2] = 0.0
        x, info = oracle.stage_solve(nez, N, ZTOP, lam, q0, b)
        ab = oracle.assemble_band(nez, N, ZTOP, lam, q0)
    assert (info == 0).all()
    A = oracle.band_to_dense(ab[0] if ab.ndim == 3 else ab, kl, kl)
    As = A * s[None, :] / s[:, None]
    bs = b[0] / s
    y = np.linalg.solve(As, bs)
    for _ in range(3):
        r = (bs.astype(np.longdouble) - As.astype(np.longdouble) @ y.astype(np.longdouble))
        y = y + np.linalg.solve(As, r.astype(np.float64))
    ref = y * s
    assert np.linalg.norm(x[0] - ref) / np.linalg.norm(ref) < 1e-12


# --------------------------------------------------------------------------
# Set 2NC (Sec. 2.1, Eq. set2nc; reading R17 of the C source): unknowns
# (rho, w, theta) in the column, advective momentum and theta equations.
# --------------------------------------------------------------------------

RGAS, CPH = 287.17, 1004.67


def _state_2nc(nez, N, seed=0, ztop=ZTOP, amp_w=5.0, amp_t=2.0):
    """A non-rest set-2NC state: rest density times 1 +- 1%, w uniform (0 at
    both ends), theta = theta_bar +- amp_t."""
    g = np.random.default_rng(seed)
    z = oracle.column_grid(nez, N, ztop)[0]
    with oracle.equation_set(oracle.SET_2NC):
        qr = oracle.reference_q(nez, N, ztop, 1)[0].reshape(-1, 3)
    rho = qr[:, 0] * (1 + 0.01 * g.uniform(-1, 1, z.size))
    w = g.uniform(-amp_w, amp_w, z.size)
    w[0] = w[-1] = 0.0
    th = qr[:, 2] + g.uniform(-amp_t, amp_t, z.size)
    return np.stack([rho, w, th], 1).reshape(-1)


def _smooth_2nc(nez, N, ztop=ZTOP):
    """A smooth non-rest state: every field a few sine or cosine waves over
    the column (w = 0 at both ends)."""
    z = oracle.column_grid(nez, N, ztop)[0]
    with oracle.equation_set(oracle.SET_2NC):
        qr = oracle.reference_q(nez, N, ztop, 1)[0].reshape(-1, 3)
    s = z / ztop
    rho = qr[:, 0] * (1 + 0.01 * np.cos(np.pi * s))
    w = 3.0 * np.sin(np.pi * s) + np.sin(3 * np.pi * s)
    th = qr[:, 2] * (1 + 0.005 * np.sin(2 * np.pi * s))
    return np.stack([rho, w, th], 1).reshape(-1)


def test_set2nc_rest_state_closed_form_and_equilibrium():
    """The set-2NC rest state is the isothermal atmosphere (rho_bar, 0,
    theta_bar = T0 exp(g z / (cp T0))), and V of it vanishes exactly."""
    nez, N = 8, 4
    z = oracle.column_grid(nez, N, ZTOP)[0]
    with oracle.equation_set(oracle.SET_2NC):
        q = _rest(nez, N)
        v = oracle.apply_V(nez, N, ZTOP, q)
        s = oracle.scales(z)
    q3 = q[0].reshape(-1, 3)
    rho = 1e5 / (RGAS * 300.0) * np.exp(-z * G / (RGAS * 300.0))
    np.testing.assert_allclose(q3[:, 0], rho, rtol=1e-13)
    assert np.array_equal(q3[:, 1], np.zeros_like(z))
    np.testing.assert_allclose(q3[:, 2], 300.0 * np.exp(G * z / (CPH * 300.0)), rtol=1e-13)
    assert np.array_equal(v, np.zeros_like(v))
    cs = np.sqrt(GAMMA * RGAS * 300.0)
    np.testing.assert_allclose(s.reshape(-1, 3), np.stack([rho, np.full_like(z, cs), q3[:, 2]], 1),
                               rtol=1e-13)


@pytest.mark.parametrize("nez,N", [(2, 2), (8, 4), (16, 3)])
def test_set2nc_conserves_column_mass(nez, N):
    """The continuity equation keeps its flux form in set 2NC: with w = 0 at
    both ends the LGL column integral of V_rho vanishes."""
    _, M = oracle.column_grid(nez, N, ZTOP)
    q = _state_2nc(nez, N, seed=41)
    with oracle.equation_set(oracle.SET_2NC):
        v = oracle.apply_V(nez, N, ZTOP, q[None])[0].reshape(-1, 3)
    q3 = q.reshape(-1, 3)
    assert abs(np.dot(M, v[:, 0])) < 1e-13 * np.abs(M * q3[:, 0] * q3[:, 1]).sum()


@pytest.mark.parametrize("nez,N", [(2, 2), (8, 4), (16, 3)])
def test_set2nc_continuity_tendency_equals_set2c(nez, N):
    """The same physical state written in sets 2C (rho, rho w, rho theta) and
    2NC (rho, w, theta) gets the same continuity tendency: both take Dcal of
    the mass flux rho w."""
    q = _state_2nc(nez, N, seed=42).reshape(-1, 3)
    rho, w, th = q[:, 0], q[:, 1], q[:, 2]
    q2 = np.stack([rho, rho * w, rho * th], 1).reshape(1, -1)
    v2 = oracle.apply_V(nez, N, ZTOP, q2)[0].reshape(-1, 3)
    with oracle.equation_set(oracle.SET_2NC):
        vn = oracle.apply_V(nez, N, ZTOP, q.reshape(1, -1))[0].reshape(-1, 3)
    np.testing.assert_allclose(vn[:, 0], v2[:, 0], rtol=0, atol=1e-13 * np.abs(v2[:, 0]).max())


def test_set2nc_momentum_and_theta_match_set2c_at_spectral_rate():
    """Sets 2C and 2NC are the same equations written with and without the
    product rule: d(rho w)/dt = rho dw/dt + w drho/dt and d(rho theta)/dt =
    rho dtheta/dt + theta drho/dt.  On a smooth state the discrete tendencies
    satisfy these identities up to the product-rule error of the derivative,
    which falls at a spectral rate with N (pins the advection, pressure and
    gravity terms of V_w and the advection of theta)."""
    em, et = [], []
    for N in (2, 4, 6, 8):
        nez = 6
        q = _smooth_2nc(nez, N).reshape(-1, 3)
        rho, w, th = q[:, 0], q[:, 1], q[:, 2]
        q2 = np.stack([rho, rho * w, rho * th], 1).reshape(1, -1)
        v2 = oracle.apply_V(nez, N, ZTOP, q2)[0].reshape(-1, 3)
        with oracle.equation_set(oracle.SET_2NC):
            vn = oracle.apply_V(nez, N, ZTOP, q.reshape(1, -1))[0].reshape(-1, 3)
        dm = rho * vn[:, 1] + w * vn[:, 0]
        dT = rho * vn[:, 2] + th * vn[:, 0]
        em.append(np.abs(dm - v2[:, 1])[1:-1].max() / np.abs(v2[:, 1]).max())
        et.append(np.abs(dT - v2[:, 2]).max() / np.abs(v2[:, 2]).max())
    for e in (em, et):
        assert e[0] > 10 * e[1] > 100 * e[2] > 1000 * e[3], e
        assert e[3] < 1e-7, e


@pytest.mark.parametrize("nez,N", [(2, 2), (4, 4), (16, 3)])
def test_set2nc_linear_operator_is_the_frechet_derivative(nez, N):
    """L(q0) x against central differences of the set-2NC V: pins the
    Frechet derivative, its point-local terms (w' dw0/dz, w' dtheta0/dz, the
    1/rho factor of the pressure and gravity terms) included.  L couples the
    points of one element only, and neither the continuity nor the theta row
    sees the other end's theta or rho, so A = I - Lambda L lies within
    k_l = k_u = 3N + 1, one inside the 3(N+1) - 1 of the band storage."""
    q0 = _state_2nc(nez, N, seed=43)
    g = np.random.default_rng(44)
    with oracle.equation_set(oracle.SET_2NC):
        s = oracle.scales(oracle.column_grid(nez, N, ZTOP)[0])
        x = s * g.standard_normal(q0.size)
        x[1] = x[-2] = 0.0
        L = oracle.apply_L(nez, N, ZTOP, q0[None], x[None])[0]
        eps = 1e-5
        fd = (oracle.apply_V(nez, N, ZTOP, (q0 + eps * x)[None])[0]
              - oracle.apply_V(nez, N, ZTOP, (q0 - eps * x)[None])[0]) / (2 * eps)
        n, kl = q0.size, 3 * (N + 1) - 1
        Ld = np.stack([oracle.apply_L(nez, N, ZTOP, q0[None], np.eye(n)[j][None])[0]
                       for j in range(n)], 1)
    assert np.linalg.norm(L - fd) <= 1e-7 * np.linalg.norm(L)
    i, j = np.indices(Ld.shape)
    assert np.abs(Ld[np.abs(i - j) >= kl]).max() == 0.0
    assert np.abs(Ld[i - j == kl - 1]).max() > 0.0 and np.abs(Ld[j - i == kl - 1]).max() > 0.0


def test_set2nc_hydrostatic_state_at_spectral_rate():
    """An isothermal atmosphere at T1 = 250 K, written as (rho, 0, theta), is
    in hydrostatic balance; its set-2NC momentum tendency is the discretisation
    error of dp/dz = -rho g divided by rho, which falls at a spectral rate with
    N (pins the EOS, the 1/rho factor and the sign of the gravity term)."""
    T1 = 250.0
    errs = []
    for N in (2, 4, 6, 8):
        nez = 3
        z = oracle.column_grid(nez, N, ZTOP)[0]
        p = 1e5 * np.exp(-z * G / (RGAS * T1))
        rho = p / (RGAS * T1)
        th = T1 * (1e5 / p) ** (RGAS / CPH)
        q = np.stack([rho, np.zeros_like(rho), th], 1).reshape(1, -1)
        with oracle.equation_set(oracle.SET_2NC):
            v = oracle.apply_V(nez, N, ZTOP, q)[0].reshape(-1, 3)
        errs.append(np.abs(v[:, 1]).max() / G)
        assert np.abs(v[:, 0]).max() == 0.0 and np.abs(v[:, 2]).max() == 0.0
    assert errs[0] > 10 * errs[1] > 100 * errs[2] > 1000 * errs[3], errs
    assert errs[3] < 1e-7, errs


def test_set2nc_one_newton_iteration_is_the_lhevi_solve():
    """Sec. 4.3 for set 2NC: one Newton iteration on F(q) = q - Lambda V(q) -
    R from q0 solves (I - Lambda L(q0)) q1 = R + Lambda (V(q0) - L(q0) q0)."""
    nez, N, lam = 8, 4, 87.868
    q0 = _state_2nc(nez, N, seed=45)[None]
    with oracle.equation_set(oracle.SET_2NC):
        R = q0 + 0.01 * oracle.scales(oracle.column_grid(nez, N, ZTOP)[0])[None] * \
            np.random.default_rng(46).standard_normal(q0.shape)
        R[0, 1] = R[0, -2] = 0.0
        q1, it, st = oracle.newton(nez, N, ZTOP, lam, R, q0, rtol=0.0, max_iter=1)
        assert it[0] == 1
        b = R + lam * (oracle.apply_V(nez, N, ZTOP, q0) - oracle.apply_L(nez, N, ZTOP, q0, q0))
        x, info = oracle.stage_solve(nez, N, ZTOP, lam, q0, b)
    assert (info == 0).all()
    np.testing.assert_allclose(q1, x, rtol=1e-12, atol=1e-12 * np.abs(q0).max())


def test_set2nc_newton_converges_quadratically():
    nez, N, lam = 8, 4, 87.868
    q0 = _state_2nc(nez, N, seed=47, amp_w=20.0, amp_t=5.0)[None]
    with oracle.equation_set(oracle.SET_2NC):
        s = oracle.scales(oracle.column_grid(nez, N, ZTOP)[0])
        R = q0.copy()

        def fnorm(q):
            return np.linalg.norm((q - lam * oracle.apply_V(nez, N, ZTOP, q) - R) / s)
        norms = [fnorm(q0)]
        for m in range(1, 5):
            q, it, st = oracle.newton(nez, N, ZTOP, lam, R, q0, rtol=0.0, max_iter=m)
            norms.append(fnorm(q))
    norms = np.array(norms) / norms[0]
    for m in range(3):
        assert norms[m + 1] <= 10.0 * norms[m] ** 2, norms
    assert norms[4] < 1e-12, norms


@pytest.mark.parametrize("nez,N", [(8, 4), (24, 4)])
def test_set2nc_stage_solve_matches_refined_dense_solve(nez, N):
    """The set-2NC stage solve (band LU of the equilibrated system) against a
    dense LAPACK solve of the same matrix (numpy, equilibrated) refined three
    times with residuals in extended precision: 1e-12."""
    lam = 87.868
    q0 = _state_2nc(nez, N, seed=48)[None]
    kl = 3 * (N + 1) - 1
    with oracle.equation_set(oracle.SET_2NC):
        s = oracle.scales(oracle.column_grid(nez, N, ZTOP)[0])
        b = q0 + 1e-2 * s * np.random.default_rng(49).standard_normal(q0.shape)
        b[0, 1] = b[0, -2] = 0.0
        x, info = oracle.stage_solve(nez, N, ZTOP, lam, q0, b)
        ab = oracle.assemble_band(nez, N, ZTOP, lam, q0)
    assert (info == 0).all()
    A = oracle.band_to_dense(ab[0] if ab.ndim == 3 else ab, kl, kl)
    As = A * s[None, :] / s[:, None]
    bs = b[0] / s
    y = np.linalg.solve(As, bs)
    for _ in range(3):
        r = (bs.astype(np.longdouble) - As.astype(np.longdouble) @ y.astype(np.longdouble))
        y = y + np.linalg.solve(As, r.astype(np.float64))
    ref = y * s
    assert np.linalg.norm(x[0] - ref) / np.linalg.norm(ref) < 1e-12


@pytest.mark.parametrize("eqset", ["SET_3C", "SET_2NC"])
def test_newton_gmres_reaches_the_lu_root_in_sets_3c_and_2nc(eqset):
    """The oracle's JFNK-GMRES (Sec. 4.2.1) works from V alone, so it serves
    every equation set: with a small Frechet perturbation and tight
    tolerances it finds the Newton-LU root in sets 3C and 2NC as in set 2C
    (an independent check of each set's analytic Jacobian, which only the
    LU path uses)."""
    nez, N = 8, 4
    lam = tableaux.ARK2.gamma * 300.0
    q0 = (_state_3c(nez, N, seed=61, amp_w=1.0, amp_t=0.5) if eqset == "SET_3C"
          else _state_2nc(nez, N, seed=61, amp_w=1.0, amp_t=0.5))[None]
    n = q0.shape[1]
    with oracle.equation_set(getattr(oracle, eqset)):
        s = oracle.scales(oracle.column_grid(nez, N, ZTOP)[0])
        R = q0 + 1e-3 * s[None] * np.random.default_rng(62).standard_normal(q0.shape)
        R[0, 1] = R[0, -2] = 0.0
        q, it, kit, st = oracle.newton_gmres(nez, N, ZTOP, lam, R, q0, eps=1e-7, rtol=1e-12,
                                             gtol=1e-12)
        qr, _, str_ = oracle.newton(nez, N, ZTOP, lam, R, q0, rtol=1e-12)
    assert st[0] == 0 and str_[0] == 0
    assert np.linalg.norm((q - qr)[0] / s) < 1e-9 * np.linalg.norm((qr - q0)[0] / s)
    assert 1 <= it[0] <= 8 and it[0] <= kit[0] <= it[0] * n
