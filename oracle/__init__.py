"""Plain FP64 CPU oracle for the HEVI vertical column solve (arXiv:2311.11425).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark are the only callers.  The product library never imports
this package, and this package imports nothing from the product.

The arithmetic lives in ``hevi_oracle.c`` (plain C, FP64, no blocking or
fusion); this module compiles it on demand with gcc and exposes it over
ctypes with numpy arrays.  ``tableaux`` holds the ARK coefficients.

Array conventions: one column has n_z = Nez*N + 1 CG points and n = 3 n_z
unknowns ordered point-major, variable-fastest (rho, m = rho w, Theta =
rho theta).  Batched calls take ``[ncols, n]`` float64 arrays and a per-column
model-top array ``ztop`` (metres).
"""

from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

from . import tableaux  # noqa: F401  (re-exported)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hevi_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libhevi_oracle.so")
_lock = threading.Lock()
_lib = None

# gcc flags: no fast-math and no FMA contraction, so x86 and Arm hosts give
# the same rounding.
CFLAGS = ["-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off", "-fno-fast-math"]


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/_build/libhevi_oracle.so``."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            c_int, c_double = ctypes.c_int, ctypes.c_double
            sig = {
                "or_set_equation_set": (c_int, [c_int]),
                "or_lgl": (c_int, [c_int, _D, _D]),
                "or_dmatrix": (c_int, [c_int, _D, _D]),
                "or_column_grid": (c_int, [c_int, c_int, c_double, _D, _D]),
                "or_reference_state": (None, [c_int, _D, _D, _D, _D, _D]),
                "or_scales": (None, [c_int, _D, _D]),
                "or_gbtrf": (c_int, [c_int, c_int, c_int, _D, c_int, _I]),
                "or_gbtrs": (None, [c_int, c_int, c_int, _D, c_int, _I, _D]),
                "or_apply_V": (c_int, [c_int, c_int, c_int, _D, _D, _D]),
                "or_apply_L": (c_int, [c_int, c_int, c_int, _D, _D, _D, _D]),
                "or_assemble_band": (c_int, [c_int, c_int, c_int, _D, c_double, _D, _D, c_int]),
                "or_reference_q": (c_int, [c_int, c_int, c_int, _D, _D]),
                "or_grid": (c_int, [c_int, c_int, c_int, _D, _D, _D]),
                "or_stage_solve": (c_int, [c_int, c_int, c_int, _D, c_double, _D, _D, _D, _I]),
                "or_newton": (c_int, [c_int, c_int, c_int, _D, c_double, _D, _D, c_double,
                                      c_int, _I, _I]),
                "or_lhevi_step": (c_int, [c_int, c_int, c_int, _D, c_int, _D, _D, _D, c_double,
                                          c_int, _D, _D, _D, _I]),
                "or_lhevi_step_about": (c_int, [c_int, c_int, c_int, _D, c_int, _D, _D, _D,
                                                c_double, c_int, _D, _D, _D, _D, _I]),
                "or_newton_gmres": (c_int, [c_int, c_int, c_int, _D, c_double, _D, _D, c_double,
                                            c_double, c_double, c_int, c_int, _I, _I, _I]),
                "or_nhevi_step": (c_int, [c_int, c_int, c_int, _D, c_int, _D, _D, _D, c_double,
                                          _D, _D, c_double, c_int, _D, _I, _I]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


SET_2C, SET_3C, SET_2NC = 0, 1, 2


@contextlib.contextmanager
def equation_set(s: int):
    """Run the oracle calls inside the block with equation set s (SET_2C:
    unknowns rho, m, Theta; SET_3C: rho, m, E, total energy, App. A.1 and
    reading R16 of the C source; SET_2NC: rho, w, theta, the advective set of
    Sec. 2.1, reading R17); set 2C again afterwards."""
    lib = _load()
    if lib.or_set_equation_set(int(s)):
        raise ValueError(f"unknown equation set {s}")
    try:
        yield
    finally:
        lib.or_set_equation_set(SET_2C)


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _ip(a: np.ndarray):
    assert a.dtype == np.intc and a.flags.c_contiguous
    return a.ctypes.data_as(_I)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def sizes(nez: int, N: int):
    """(n_z, n, k) with k = k_l = k_u = 3(N+1) - 1."""
    nz = nez * N + 1
    return nz, 3 * nz, 3 * (N + 1) - 1


def _ztop(ztop, ncols):
    z = np.atleast_1d(_f64(ztop))
    if z.size == 1 and ncols != 1:
        z = np.full(ncols, float(z[0]))
    assert z.size == ncols
    return np.ascontiguousarray(z)


def lgl(N: int):
    """LGL nodes and weights of order N (Sec. 3)."""
    xi, w = np.zeros(N + 1), np.zeros(N + 1)
    if _load().or_lgl(N, _dp(xi), _dp(w)):
        raise ValueError("bad order")
    return xi, w


def dmatrix(N: int) -> np.ndarray:
    """Dhat[k, j] = h_j'(xi_k) (Sec. 3; the paper's D is its transpose)."""
    xi, _ = lgl(N)
    D = np.zeros((N + 1) * (N + 1))
    _load().or_dmatrix(N, _dp(xi), _dp(D))
    return D.reshape(N + 1, N + 1)


def column_grid(nez: int, N: int, ztop: float):
    """Heights z_I and DSS'd diagonal mass M_I of one column (Sec. 3)."""
    nz = nez * N + 1
    z, M = np.zeros(nz), np.zeros(nz)
    if _load().or_column_grid(nez, N, float(ztop), _dp(z), _dp(M)):
        raise ValueError("bad grid")
    return z, M


def reference_state(z):
    """rho_bar, theta_bar, Theta_bar, P_bar = EOS(Theta_bar) at heights z."""
    z = _f64(z)
    out = [np.zeros_like(z) for _ in range(4)]
    _load().or_reference_state(z.size, _dp(z), *[_dp(a) for a in out])
    return tuple(out)


def scales(z) -> np.ndarray:
    """Per-unknown scales (rho_bar, rho_bar c_s, Theta_bar) at heights z."""
    z = _f64(z)
    s = np.zeros(3 * z.size)
    _load().or_scales(z.size, _dp(z), _dp(s))
    return s


def reference_q(nez: int, N: int, ztop, ncols: int = 1) -> np.ndarray:
    nz, n, _ = sizes(nez, N)
    zt = _ztop(ztop, ncols)
    q = np.zeros((ncols, n))
    _load().or_reference_q(ncols, nez, N, _dp(zt), _dp(q))
    return q


def grid(nez: int, N: int, ztop, ncols: int = 1):
    nz, _, _ = sizes(nez, N)
    zt = _ztop(ztop, ncols)
    z, M = np.zeros((ncols, nz)), np.zeros((ncols, nz))
    _load().or_grid(ncols, nez, N, _dp(zt), _dp(z), _dp(M))
    return z, M


def apply_V(nez: int, N: int, ztop, q) -> np.ndarray:
    """Nonlinear vertical operator V(q) (App. A.2), batched over columns."""
    q = _f64(np.atleast_2d(q))
    zt = _ztop(ztop, q.shape[0])
    v = np.zeros_like(q)
    _load().or_apply_V(q.shape[0], nez, N, _dp(zt), _dp(q), _dp(v))
    return v


def apply_L(nez: int, N: int, ztop, q0, x) -> np.ndarray:
    """Linearised vertical operator L(q0) x (Sec. 4.3.1), batched."""
    q0, x = _f64(np.atleast_2d(q0)), _f64(np.atleast_2d(x))
    zt = _ztop(ztop, x.shape[0])
    y = np.zeros_like(x)
    _load().or_apply_L(x.shape[0], nez, N, _dp(zt), _dp(q0), _dp(x), _dp(y))
    return y


def assemble_band(nez: int, N: int, ztop, lam: float, q0, ldab: int | None = None):
    """A = I - Lambda L(q0) in LAPACK band storage, shape [ncols, n, ldab]
    (column j of A is row j of the result: AB[c, j, kl+ku+i-j] = A[i, j])."""
    q0 = _f64(np.atleast_2d(q0))
    nz, n, k = sizes(nez, N)
    ldab = 3 * k + 1 if ldab is None else ldab
    zt = _ztop(ztop, q0.shape[0])
    ab = np.zeros((q0.shape[0], n, ldab))
    if _load().or_assemble_band(q0.shape[0], nez, N, _dp(zt), float(lam), _dp(q0), _dp(ab), ldab):
        raise ValueError("bad ldab")
    return ab


def band_to_dense(ab: np.ndarray, kl: int, ku: int) -> np.ndarray:
    """Expand one LAPACK band array (as returned above, [n, ldab]) to dense."""
    n, ldab = ab.shape
    A = np.zeros((n, n))
    kv = kl + ku
    for j in range(n):
        for i in range(max(0, j - kv), min(n, j + kl + 1)):
            A[i, j] = ab[j, kv + i - j]
    return A


def gbtrf(ab: np.ndarray, kl: int, ku: int):
    """In-place band LU (dgbtrf semantics) of one [n, ldab] band array.
    Returns (info, ipiv) with 0-based pivots."""
    assert ab.dtype == np.float64 and ab.flags.c_contiguous
    n, ldab = ab.shape
    ipiv = np.zeros(n, dtype=np.intc)
    info = _load().or_gbtrf(n, kl, ku, _dp(ab), ldab, _ip(ipiv))
    return info, ipiv


def gbtrs(ab: np.ndarray, kl: int, ku: int, ipiv: np.ndarray, b) -> np.ndarray:
    n, ldab = ab.shape
    x = _f64(b).copy()
    _load().or_gbtrs(n, kl, ku, _dp(ab), ldab, _ip(np.ascontiguousarray(ipiv, dtype=np.intc)),
                     _dp(x))
    return x


def stage_solve(nez: int, N: int, ztop, lam: float, q0, b):
    """x = (I - Lambda L(q0))^-1 b per column (Sec. 4.3); returns (x, info)."""
    q0, b = _f64(np.atleast_2d(q0)), _f64(np.atleast_2d(b))
    zt = _ztop(ztop, b.shape[0])
    x = np.zeros_like(b)
    info = np.zeros(b.shape[0], dtype=np.intc)
    _load().or_stage_solve(b.shape[0], nez, N, _dp(zt), float(lam), _dp(q0), _dp(b), _dp(x),
                           _ip(info))
    return x, info


def newton(nez: int, N: int, ztop, lam: float, R, q_init, rtol: float = 1e-10,
           max_iter: int = 20):
    """NHEVI-LU Newton solve of F(q) = q - Lambda V(q) - R = 0 (Sec. 4.2.3).
    Returns (q, iters, status)."""
    R = _f64(np.atleast_2d(R))
    q = _f64(np.atleast_2d(q_init)).copy()
    zt = _ztop(ztop, q.shape[0])
    it = np.zeros(q.shape[0], dtype=np.intc)
    st = np.zeros(q.shape[0], dtype=np.intc)
    _load().or_newton(q.shape[0], nez, N, _dp(zt), float(lam), _dp(R), _dp(q), float(rtol),
                      int(max_iter), _ip(it), _ip(st))
    return q, it, st


def newton_gmres(nez: int, N: int, ztop, lam: float, R, q_init, eps: float = 0.05,
                 rtol: float = 1e-5, gtol: float = 1e-9, max_newton: int = 30,
                 kmax: int | None = None):
    """NHEVI-GMRES (Sec. 4.2.1): Jacobian-free Newton-Krylov solve of
    F(q) = q - Lambda V(q) - R = 0; Frechet perturbation eps S (reading R14),
    unrestarted GMRES to gtol, Newton stop as ``newton`` (reading R7).
    Returns (q, newton_iters, krylov_iters, status)."""
    R = _f64(np.atleast_2d(R))
    q = _f64(np.atleast_2d(q_init)).copy()
    zt = _ztop(ztop, q.shape[0])
    n = q.shape[1]
    kmax = n if kmax is None else int(kmax)
    it = np.zeros(q.shape[0], dtype=np.intc)
    kit = np.zeros(q.shape[0], dtype=np.intc)
    st = np.zeros(q.shape[0], dtype=np.intc)
    _load().or_newton_gmres(q.shape[0], nez, N, _dp(zt), float(lam), _dp(R), _dp(q), float(eps),
                            float(rtol), float(gtol), int(max_newton), kmax, _ip(it), _ip(kit),
                            _ip(st))
    return q, it, kit, st


def lhevi_step(nez: int, N: int, ztop, tab, dt: float, qn, H, lin: int = 0, q_lin=None):
    """One LHEVI ARK step (Sec. 4.3); lin 0 = PS, 1 = RS, 2 = linear test
    problem V := L_RS (q - q_bar).  With q_lin (state layout, per column) the
    Jacobian is linearised about q_lin instead (a Jacobian kept from an earlier
    step; lin then only selects V: 0 nonlinear, 2 the linear test problem).
    Returns (q_next, info)."""
    qn, H = _f64(np.atleast_2d(qn)), _f64(np.atleast_2d(H))
    zt = _ztop(ztop, qn.shape[0])
    A, At, b = (_f64(tab.A), _f64(tab.At), _f64(tab.b))
    out = np.zeros_like(qn)
    info = np.zeros(qn.shape[0], dtype=np.intc)
    if q_lin is None:
        _load().or_lhevi_step(qn.shape[0], nez, N, _dp(zt), tab.s, _dp(A), _dp(At), _dp(b),
                              float(dt), int(lin), _dp(qn), _dp(H), _dp(out), _ip(info))
    else:
        ql = _f64(np.atleast_2d(q_lin))
        assert ql.shape == qn.shape
        _load().or_lhevi_step_about(qn.shape[0], nez, N, _dp(zt), tab.s, _dp(A), _dp(At), _dp(b),
                                    float(dt), int(lin), _dp(ql), _dp(qn), _dp(H), _dp(out),
                                    _ip(info))
    return out, info


def nhevi_step(nez: int, N: int, ztop, tab, dt: float, qn, H, rtol: float = 1e-10,
               max_iter: int = 20):
    """One NHEVI-LU ARK step (Sec. 4.2).  Returns (q_next, iters, status)."""
    qn, H = _f64(np.atleast_2d(qn)), _f64(np.atleast_2d(H))
    zt = _ztop(ztop, qn.shape[0])
    A, At, b = (_f64(tab.A), _f64(tab.At), _f64(tab.b))
    out = np.zeros_like(qn)
    it = np.zeros(qn.shape[0], dtype=np.intc)
    st = np.zeros(qn.shape[0], dtype=np.intc)
    _load().or_nhevi_step(qn.shape[0], nez, N, _dp(zt), tab.s, _dp(A), _dp(At), _dp(b), float(dt),
                          _dp(qn), _dp(H), float(rtol), int(max_iter), _dp(out), _ip(it), _ip(st))
    return out, it, st
