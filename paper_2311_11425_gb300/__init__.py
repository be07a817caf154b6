"""GB300 (sm_103a) HEVI vertical column solver: Python binding of include/hevi.h.

Argument marshalling only: every step runs in the CUDA library
``_build/libhevi.so`` (built by ``build.py``).  There is no CPU fallback; if
the library is missing or no GPU is present, calls raise.

Low-level functions carry the C names (``hevi_setup``, ``hevi_factor``,
``hevi_stage_solve``, ``hevi_newton_solve``, ``hevi_apply_Lv``, ...) and take
raw device pointers; :class:`Context` wraps them for torch CUDA tensors
(float64, contiguous, packed column-major state layout of the header).
"""

from __future__ import annotations

import ctypes
import os
import weakref

from . import build as _build_mod

__all__ = ["load", "Context", "HeviError", "FP64", "FP32_IR", "tableau", "Tableau"]

FP64, FP32_IR = 0, 1
SET_2C, SET_3C, SET_2NC = 0, 1, 2  # equation sets (hevi_set_equation_set)
STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "out of device memory",
          4: "singular column", 5: "not converged", 6: "non-physical input state",
          7: "device wait past its limit"}
COL_OK, COL_SINGULAR, COL_NOT_CONVERGED, COL_BAD_INPUT = 0, 4, 5, 6


class HeviError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {STATUS.get(code, code)} (status {code})")
        self.code = code


class _SizeClass(ctypes.Structure):
    _fields_ = [("nez", ctypes.c_int32), ("order", ctypes.c_int32)]


class _Grid(ctypes.Structure):
    _fields_ = [("ncols", ctypes.c_int64), ("classes", ctypes.POINTER(_SizeClass)),
                ("nclasses", ctypes.c_int32), ("class_of_col", ctypes.POINTER(ctypes.c_int32)),
                ("z_top", ctypes.POINTER(ctypes.c_double))]


class _Ref(ctypes.Structure):
    _fields_ = [("T0", ctypes.c_double), ("p0", ctypes.c_double), ("R", ctypes.c_double),
                ("cp", ctypes.c_double), ("g", ctypes.c_double)]


_lib = None
_P = ctypes.c_void_p
_D = ctypes.c_double
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64


def load(build: bool = False):
    """Load libhevi.so (compiling it first when `build` is true)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build_mod.LIB
    if build:
        path = _build_mod.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run paper_2311_11425_gb300.build)")
    lib = ctypes.CDLL(path)
    DP = ctypes.POINTER(ctypes.c_double)
    sigs = {
        "hevi_setup": (_I32, [ctypes.POINTER(_P), ctypes.POINTER(_Grid), ctypes.POINTER(_Ref), _I32, _P]),
        "hevi_destroy": (None, [_P]),
        "hevi_set_stream": (_I32, [_P, _P]),
        "hevi_state_size": (_I64, [_P]),
        "hevi_column_offset": (_I64, [_P, _I64]),
        "hevi_device_bytes": (_I64, [_P]),
        "hevi_reference_state": (_I32, [_P, _P]),
        "hevi_factor": (_I32, [_P, _D, _P]),
        "hevi_stage_solve": (_I32, [_P, _P, _P]),
        "hevi_stage_solve_async": (_I32, [_P, _P, _P]),
        "hevi_set_refinement": (_I32, [_P, _D, _I32]),
        "hevi_test_drop_record_copy": (_I32, [_P, _I32]),
        "hevi_set_solve_warps": (_I32, [_P, _I32]),
        "hevi_reference_columns": (_I32, [_P, _I64, _I64, _P]),
        "hevi_set_column_tops": (_I32, [_P, _I64, _I64, DP]),
        "hevi_set_newton_host_check": (_I32, [_P, _I32]),
        "hevi_set_fused_stages": (_I32, [_P, _I32]),
        "hevi_set_equation_set": (_I32, [_P, _I32]),
        "hevi_autotune_solve": (_I32, [_P, _P, _P, _I32, ctypes.POINTER(_I32), DP, DP]),
        "hevi_newton_solve": (_I32, [_P, _D, _P, _P, _D, _I32]),
        "hevi_newton_solve_async": (_I32, [_P, _D, _P, _P, _D, _I32]),
        "hevi_apply_Lv": (_I32, [_P, _P, _P, ctypes.c_int]),
        "hevi_column_status": (_I32, [_P, _P, _P]),
        "hevi_lhevi_step": (_I32, [_P, _I32, DP, DP, DP, _D, _P, _P, _P, _I32]),
        "hevi_nhevi_step": (_I32, [_P, _I32, DP, DP, DP, _D, _P, _P, _P, _D, _I32]),
        "hevi_sync": (_I32, [_P]),
        "hevi_launch_count": (_I64, [_P]),
        "hevi_status_string": (ctypes.c_char_p, [_I32]),
        "hevi_tableau": (_I32, [ctypes.c_char_p, ctypes.POINTER(_I32), DP, DP, DP]),
        "hevi_newton_solve_noalloc": (_I32, [_I32, _I32, _D, _I64, _D, _P, _P, _D, _I32, _P, _P,
                                             _P]),
        "hevi_profile": (_I32, [_P, _I32]),
        "hevi_profile_kinds": (_I32, []),
        "hevi_profile_kind_name": (ctypes.c_char_p, [_I32]),
        "hevi_profile_read": (_I32, [_P, _I32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I64)]),
        "hevi_lhevi_graph_create": (_I32, [_P, _I32, DP, DP, DP, _D, _P, _P, _P, _I32, _I32,
                                           ctypes.POINTER(_P)]),
        "hevi_nhevi_graph_create": (_I32, [_P, _I32, DP, DP, DP, _D, _P, _P, _P, _I32, _D, _I32,
                                           ctypes.POINTER(_P)]),
        "hevi_graph_launch": (_I32, [_P]),
        "hevi_estimate_bytes": (_I64, [ctypes.POINTER(_Grid), _I32, _I32, _I32]),
        "hevi_newton_gmres_solve": (_I32, [_P, _D, _P, _P, _D, _D, _D, _I32, _I32, _P]),
        "hevi_newton_gmres_solve_async": (_I32, [_P, _D, _P, _P, _D, _D, _D, _I32, _I32, _P]),
        "hevi_graph_destroy": (None, [_P]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class Graph:
    """A captured step loop (hevi_graph); keeps its context and buffers alive."""

    def __init__(self, ctx, handle, keep):
        self._ctx, self._h, self._keep = ctx, handle, keep

    def launch(self):
        """hevi_graph_launch: one replay on the context's stream (asynchronous)."""
        if not self._h:
            raise HeviError("graph is closed")
        _check(self._ctx._lib.hevi_graph_launch(self._h), "hevi_graph_launch")

    def close(self):
        if self._h:
            self._ctx._lib.hevi_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Tableau:
    """An ESDIRK tableau (s stages; A explicit, At implicit, b weights)."""

    def __init__(self, name, A, At, b):
        self.name, self.A, self.At, self.b = name, A, At, b

    @property
    def s(self):
        return len(self.b)

    @property
    def gamma(self):
        return float(self.At[1, 1])


def tableau(name: str) -> Tableau:
    """The library's named tableau ("ARK2", "ARK3", "ARK4"), via hevi_tableau."""
    import numpy as np
    lib = load()
    s = _I32()
    A, At, b = np.zeros(64), np.zeros(64), np.zeros(8)
    DP = ctypes.POINTER(ctypes.c_double)
    _check(lib.hevi_tableau(name.encode(), ctypes.byref(s), A.ctypes.data_as(DP),
                            At.ctypes.data_as(DP), b.ctypes.data_as(DP)), "hevi_tableau")
    n = s.value
    return Tableau(name, A[: n * n].reshape(n, n).copy(), At[: n * n].reshape(n, n).copy(),
                   b[:n].copy())


def _check(code: int, where: str):
    if code != 0:
        raise HeviError(code, where)


def _ptr(t, n=None, dtype=None):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if n is not None and t.numel() != n:
        raise ValueError(f"expected {n} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _darr(x):
    import numpy as np
    a = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def hevi_newton_solve_noalloc(nez, order, z_top, ncols, gamma_dt, state, R, status, iters,
                              rtol=1e-10, max_iter=20, stream=None):
    """Newton solve (NHEVI-LU) of `ncols` uniform columns that allocates no device
    memory, for callers that cannot call cudaMalloc (inside another framework's
    memory pool, under an allocator lock, or in a plugin that must not touch the
    device heap).  All scratch lives in a fixed 64 MiB device array of the
    library, shared by every call: calls that overlap on the GPU race.  state
    (in/out), R: float64 CUDA tensors of 3 (nez order + 1) ncols entries; status,
    iters: int32 CUDA tensors of ncols entries (outputs).  Raises HeviError
    (INVALID_ARG) when the columns do not fit the scratch (about 4,000 columns
    of (16, 3) or (10, 4))."""
    import torch
    lib = load()
    n = 3 * (int(nez) * int(order) + 1) * int(ncols)
    st = torch.cuda.current_stream() if stream is None else stream
    code = lib.hevi_newton_solve_noalloc(
        int(nez), int(order), float(z_top), int(ncols), float(gamma_dt),
        _ptr(state, n, torch.float64), _ptr(R, n, torch.float64), float(rtol), int(max_iter),
        _ptr(status, int(ncols), torch.int32), _ptr(iters, int(ncols), torch.int32),
        ctypes.c_void_p(st.cuda_stream))
    if code == 1:
        raise HeviError(1, "hevi_newton_solve_noalloc (bad argument, or the columns do not fit "
                           "the 64 MiB scratch array)")
    _check(code, "hevi_newton_solve_noalloc")
    return state


LHEVI, NHEVI = 1, 2  # step kinds of hevi_estimate_bytes


def hevi_estimate_bytes(classes, class_of_col=None, ncols=None, precision=FP32_IR, kind=0,
                        stages=2) -> int:
    """Device bytes of a context over this column set plus the workspace of its
    first step of `kind` (0 none, LHEVI, NHEVI) with `stages` stages
    (hevi_estimate_bytes); host arithmetic only, no device needed."""
    import numpy as np
    lib = load()
    classes = [tuple(int(v) for v in c) for c in classes]
    if ncols is None:
        ncols = 1 if class_of_col is None else len(class_of_col)
    arr = (_SizeClass * len(classes))(*[_SizeClass(nez, order) for nez, order in classes])
    cptr, cc = None, None
    if class_of_col is not None:
        cc = np.ascontiguousarray(class_of_col, dtype=np.int32)
        cptr = cc.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    grid = _Grid(int(ncols), arr, len(classes), cptr, None)
    b = int(lib.hevi_estimate_bytes(ctypes.byref(grid), int(precision), int(kind), int(stages)))
    if b < 0:
        raise HeviError(1, "hevi_estimate_bytes: invalid arguments")
    return b


class Context:
    """A set of columns on the current CUDA device (wraps ``hevi_ctx``).

    classes: list of (nez, order); class_of_col: per-column class index (or
    None with a single class); z_top: per-column model top in metres (scalar
    broadcasts); precision: FP64 or FP32_IR.
    """

    def __init__(self, classes, z_top, class_of_col=None, ncols=None, precision=FP32_IR,
                 stream=None, ref=None):
        import numpy as np
        import torch
        lib = load()
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device")
        classes = [tuple(int(v) for v in c) for c in classes]
        zt = np.atleast_1d(np.asarray(z_top, dtype=np.float64))
        if ncols is None:
            ncols = zt.size if class_of_col is None else len(class_of_col)
        if zt.size == 1 and ncols > 1:
            zt = np.full(ncols, float(zt[0]))
        zt = np.ascontiguousarray(zt)
        self._keep = [zt]
        arr = (_SizeClass * len(classes))(*[_SizeClass(nez, order) for nez, order in classes])
        cptr = None
        if class_of_col is not None:
            cc = np.ascontiguousarray(class_of_col, dtype=np.int32)
            self._keep.append(cc)
            cptr = cc.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        grid = _Grid(int(ncols), arr, len(classes), cptr,
                     zt.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        refp = None
        if ref is not None:
            refp = ctypes.byref(_Ref(*ref))
        self.stream = torch.cuda.current_stream() if stream is None else stream
        h = ctypes.c_void_p()
        _check(lib.hevi_setup(ctypes.byref(h), ctypes.byref(grid), refp, int(precision),
                              ctypes.c_void_p(self.stream.cuda_stream)), "hevi_setup")
        self._h = h
        self._lib = lib
        self.ncols = int(ncols)
        self.classes = classes
        self.precision = precision
        self.n = int(lib.hevi_state_size(h))
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._graphs = weakref.WeakSet()

    # -- housekeeping ---------------------------------------------------------
    def close(self):
        for g in list(getattr(self, "_graphs", ())):
            g.close()  # a graph must not outlive its context
        if getattr(self, "_h", None):
            self._lib.hevi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_stream(self, stream):
        self.stream = stream
        _check(self._lib.hevi_set_stream(self._h, ctypes.c_void_p(stream.cuda_stream)),
               "hevi_set_stream")

    def offsets(self):
        import numpy as np
        return np.array([self._lib.hevi_column_offset(self._h, i) for i in range(self.ncols + 1)],
                        dtype=np.int64)

    @property
    def device_bytes(self) -> int:
        return int(self._lib.hevi_device_bytes(self._h))

    @property
    def launch_count(self) -> int:
        return int(self._lib.hevi_launch_count(self._h))

    def empty(self):
        import torch
        return torch.empty(self.n, dtype=torch.float64, device=self.device)

    def _v(self, t):
        import torch
        return _ptr(t, self.n, torch.float64)

    # -- C calls --------------------------------------------------------------
    def hevi_reference_state(self, out=None):
        out = self.empty() if out is None else out
        _check(self._lib.hevi_reference_state(self._h, self._v(out)), "hevi_reference_state")
        return out

    def hevi_reference_columns(self, first: int, count: int, out):
        """Writes the rest state of the columns [first, first + count) into out."""
        _check(self._lib.hevi_reference_columns(self._h, int(first), int(count), self._v(out)),
               "hevi_reference_columns")
        return out

    def hevi_set_column_tops(self, first: int, z_top):
        """New model tops (m) for the columns [first, first + len(z_top))."""
        import numpy as np
        zt = np.ascontiguousarray(z_top, dtype=np.float64).reshape(-1)
        _check(self._lib.hevi_set_column_tops(self._h, int(first), int(zt.size),
                                              zt.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "hevi_set_column_tops")

    def hevi_set_equation_set(self, eqset: int):
        """SET_2C (rho, m, Theta) or SET_3C (rho, m, E; FP64 contexts only)."""
        _check(self._lib.hevi_set_equation_set(self._h, int(eqset)), "hevi_set_equation_set")

    def hevi_set_newton_host_check(self, on: bool):
        _check(self._lib.hevi_set_newton_host_check(self._h, 1 if on else 0),
               "hevi_set_newton_host_check")

    def hevi_set_fused_stages(self, on: bool):
        _check(self._lib.hevi_set_fused_stages(self._h, 1 if on else 0), "hevi_set_fused_stages")

    def hevi_factor(self, gamma_dt: float, lin_state=None):
        p = None if lin_state is None else self._v(lin_state)
        _check(self._lib.hevi_factor(self._h, float(gamma_dt), p), "hevi_factor")

    def hevi_set_refinement(self, tol: float, max_sweeps: int):
        _check(self._lib.hevi_set_refinement(self._h, float(tol), int(max_sweeps)),
               "hevi_set_refinement")

    def hevi_set_solve_warps(self, warps_per_sm: int):
        _check(self._lib.hevi_set_solve_warps(self._h, int(warps_per_sm)), "hevi_set_solve_warps")

    def hevi_autotune_solve(self, rhs, x=None, reps: int = 3):
        """Times the FP32 stage solve at each launch shape and keeps the
        fastest; returns (warps_per_sm, ms, ms_default)."""
        x = self.empty() if x is None else x
        w, ms, md = _I32(0), ctypes.c_double(0.0), ctypes.c_double(0.0)
        _check(self._lib.hevi_autotune_solve(self._h, self._v(rhs), self._v(x), int(reps),
                                             ctypes.byref(w), ctypes.byref(ms), ctypes.byref(md)),
               "hevi_autotune_solve")
        return int(w.value), float(ms.value), float(md.value)

    def hevi_test_drop_record_copy(self, step: int):
        """Test hook: leave out one record copy per tile so that the solve's
        bounded wait runs out (step < 0 turns it off)."""
        _check(self._lib.hevi_test_drop_record_copy(self._h, int(step)),
               "hevi_test_drop_record_copy")

    def hevi_stage_solve(self, rhs, x=None, blocking=True):
        x = self.empty() if x is None else x
        f = self._lib.hevi_stage_solve if blocking else self._lib.hevi_stage_solve_async
        _check(f(self._h, self._v(rhs), self._v(x)), "hevi_stage_solve")
        return x

    def hevi_newton_solve(self, gamma_dt: float, state, R, rtol=1e-10, max_iter=20, blocking=True):
        f = self._lib.hevi_newton_solve if blocking else self._lib.hevi_newton_solve_async
        _check(f(self._h, float(gamma_dt), self._v(state), self._v(R), float(rtol), int(max_iter)),
               "hevi_newton_solve")
        return state

    def hevi_apply_Lv(self, x, y=None, nonlinear=False):
        y = self.empty() if y is None else y
        _check(self._lib.hevi_apply_Lv(self._h, self._v(x), self._v(y), int(bool(nonlinear))),
               "hevi_apply_Lv")
        return y

    def hevi_column_status(self):
        import torch
        st = torch.empty(self.ncols, dtype=torch.int32, device=self.device)
        it = torch.empty(self.ncols, dtype=torch.int32, device=self.device)
        _check(self._lib.hevi_column_status(self._h, _ptr(st), _ptr(it)), "hevi_column_status")
        return st, it

    def hevi_lhevi_step(self, tab, dt, q_in, H, q_out=None, lin_about_rest=False,
                        refactor=True):
        """One LHEVI step; refactor=False keeps the current factorisation (a
        Jacobian update interval of more than one step)."""
        q_out = self.empty() if q_out is None else q_out
        A, pA = _darr(tab.A)
        At, pAt = _darr(tab.At)
        b, pb = _darr(tab.b)
        mode = 2 if not refactor else int(bool(lin_about_rest))
        _check(self._lib.hevi_lhevi_step(self._h, len(b), pA, pAt, pb, float(dt), self._v(q_in),
                                         self._v(H), self._v(q_out), mode),
               "hevi_lhevi_step")
        return q_out

    def hevi_nhevi_step(self, tab, dt, q_in, H, q_out=None, rtol=1e-10, max_iter=20):
        q_out = self.empty() if q_out is None else q_out
        A, pA = _darr(tab.A)
        At, pAt = _darr(tab.At)
        b, pb = _darr(tab.b)
        _check(self._lib.hevi_nhevi_step(self._h, len(b), pA, pAt, pb, float(dt), self._v(q_in),
                                         self._v(H), self._v(q_out), float(rtol), int(max_iter)),
               "hevi_nhevi_step")
        return q_out

    def hevi_lhevi_graph(self, tab, dt, q_a, q_b, H, nsteps=1, lin_about_rest=False,
                         refactor=True):
        """nsteps LHEVI steps captured into one CUDA graph (hevi_lhevi_graph_create);
        replays ping-pong between q_a and q_b (result in q_b for odd nsteps)."""
        A, pA = _darr(tab.A)
        At, pAt = _darr(tab.At)
        b, pb = _darr(tab.b)
        h = _P()
        _check(self._lib.hevi_lhevi_graph_create(
            self._h, len(b), pA, pAt, pb, float(dt), self._v(q_a), self._v(q_b), self._v(H),
            int(nsteps), 2 if not refactor else int(bool(lin_about_rest)), ctypes.byref(h)),
            "hevi_lhevi_graph_create")
        g = Graph(self, h, (q_a, q_b, H))
        self._graphs.add(g)
        return g

    def hevi_nhevi_graph(self, tab, dt, q_a, q_b, H, nsteps=1, rtol=1e-10, max_iter=20):
        """nsteps NHEVI-LU steps captured into one CUDA graph (hevi_nhevi_graph_create)."""
        A, pA = _darr(tab.A)
        At, pAt = _darr(tab.At)
        b, pb = _darr(tab.b)
        h = _P()
        _check(self._lib.hevi_nhevi_graph_create(
            self._h, len(b), pA, pAt, pb, float(dt), self._v(q_a), self._v(q_b), self._v(H),
            int(nsteps), float(rtol), int(max_iter), ctypes.byref(h)), "hevi_nhevi_graph_create")
        g = Graph(self, h, (q_a, q_b, H))
        self._graphs.add(g)
        return g

    def hevi_newton_gmres_solve(self, gamma_dt, state, R, eps=0.05, rtol=1e-5, gtol=1e-9,
                                max_newton=30, kmax=0, krylov=None, blocking=True):
        """NHEVI-GMRES column solve in place on `state` (hevi_newton_gmres_solve);
        `krylov` (int32 tensor of ncols, optional) receives the Krylov
        iterations per column."""
        fn = (self._lib.hevi_newton_gmres_solve if blocking
              else self._lib.hevi_newton_gmres_solve_async)
        import torch
        kp = _ptr(krylov, self.ncols, torch.int32) if krylov is not None else None
        _check(fn(self._h, float(gamma_dt), self._v(state), self._v(R), float(eps), float(rtol),
                  float(gtol), int(max_newton), int(kmax), kp), "hevi_newton_gmres_solve")
        return state

    def hevi_profile(self, enable: bool):
        _check(self._lib.hevi_profile(self._h, int(bool(enable))), "hevi_profile")

    def hevi_profile_read(self) -> dict:
        """{kind name: (total ms, launches)} of the timed kernels."""
        out = {}
        for k in range(self._lib.hevi_profile_kinds()):
            ms, n = ctypes.c_double(), _I64()
            _check(self._lib.hevi_profile_read(self._h, k, ctypes.byref(ms), ctypes.byref(n)),
                   "hevi_profile_read")
            out[self._lib.hevi_profile_kind_name(k).decode()] = (ms.value, n.value)
        return out

    def hevi_sync(self):
        _check(self._lib.hevi_sync(self._h), "hevi_sync")
