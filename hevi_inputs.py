"""Seeded synthetic inputs for the HEVI column solve.

This module holds only random draws and input shapes: no grid, operator,
reference state or solver arithmetic.  Both the oracle and the CUDA path
consume what it returns, and neither is imported here.

Fields that describe a physical state are returned as *increments* over the
isothermal rest state; each side adds them to its own rest state.  Shapes are
functions of the normalised point index s = I / (n_z - 1) in [0, 1] (the
input does not need the LGL heights), and the amplitude profile
``density_like(s, ztop)`` decays like an isothermal density with an 8.8 km
scale height, which gives the perturbations the vertical structure of the
paper's global runs (Sec. 7) without reproducing the model's reference state.

Workloads (cubed-sphere column counts 6 (Ne N)^2 + 2):
  lhevi_stage   1,538 columns, Nez=8,  N=4, 30 km top, one stage solve.
  lhevi_ark3   86,402 columns, Nez=10, N=4, 30 km top, ARK3 steps of 300 s.
  nhevi_ark2   86,402 columns, Nez=16, N=3, 30 km top, one ARK2 step of 300 s.
  batched      200,000 columns over (Nez, N) in {(8,4),(10,4),(16,3),(24,4)},
               tops uniform in 30-100 km.
"""

from __future__ import annotations

import numpy as np

GAMMA_ARK2 = 1.0 - 1.0 / np.sqrt(2.0)
SIZE_CLASSES = ((8, 4), (10, 4), (16, 3), (24, 4))


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def sizes(nez: int, N: int):
    nz = nez * N + 1
    return nz, 3 * nz


def density_like(s: np.ndarray, ztop) -> np.ndarray:
    """1.16 kg m^-3 * exp(-s ztop / 8.8 km): an input amplitude profile."""
    return 1.16 * np.exp(-np.asarray(s) * np.asarray(ztop)[..., None] / 8.8e3)


def _s(nz: int) -> np.ndarray:
    return np.arange(nz) / (nz - 1)


def cubed_sphere_points(ne: int, order: int) -> np.ndarray:
    """Unique points of an equiangular cubed sphere with ne x ne elements of
    `order` equally spaced intervals per face edge: 6 (ne order)^2 + 2 unit
    vectors, shape [count, 3]."""
    m = ne * order
    a = np.linspace(-np.pi / 4, np.pi / 4, m + 1)
    A, B = np.meshgrid(np.tan(a), np.tan(a), indexing="ij")
    one = np.ones_like(A)
    faces = [(one, A, B), (-one, -A, B), (A, one, B), (-A, -one, B), (A, B, one), (A, -B, -one)]
    pts = np.concatenate([np.stack(f, -1).reshape(-1, 3) for f in faces])
    pts /= np.linalg.norm(pts, axis=1, keepdims=True)
    _, idx = np.unique(np.round(pts, 9), axis=0, return_index=True)
    out = pts[np.sort(idx)]
    assert out.shape[0] == 6 * m * m + 2, out.shape
    return out


def sphere_points_uniform(g: np.random.Generator, count: int) -> np.ndarray:
    v = g.standard_normal((count, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def smooth_sphere_field(g: np.random.Generator, pts: np.ndarray, degree: int = 8) -> np.ndarray:
    """A random polynomial of total degree <= `degree` in (x, y, z) restricted to
    the sphere (hence a spherical-harmonic sum of degree <= `degree`), with
    N(0,1) coefficients, scaled to max |f| = 1."""
    x, y, z = pts.T
    f = np.zeros(len(pts))
    for i in range(degree + 1):
        for j in range(degree + 1 - i):
            for k in range(degree + 1 - i - j):
                f += g.standard_normal() * x**i * y**j * z**k
    return f / np.abs(f).max()


def gaussian_bump(s: np.ndarray, centre: np.ndarray, width: float) -> np.ndarray:
    return np.exp(-(((s[None, :] - centre[:, None]) / width) ** 2))


def lhevi_stage(seed: int = 1, ncols: int = 1538, nez: int = 8, N: int = 4,
                ztop: float = 30e3, dt: float = 300.0) -> dict:
    """One LHEVI stage solve (I - Lambda L) x = b about the rest state.
    b_rho = 0; b_m ~ U(-0.1, 0.1) kg m^-2 s^-1 at interior points, 0 at both
    ends; b_Theta = 1 K * density_like * Gaussian(centre ~ U(0.25, 0.75),
    width 1/15)."""
    g = rng(seed)
    nz, n = sizes(nez, N)
    s = _s(nz)
    zt = np.full(ncols, ztop)
    centre = g.uniform(0.25, 0.75, ncols)
    b = np.zeros((ncols, nz, 3))
    b[:, 1:-1, 1] = g.uniform(-0.1, 0.1, (ncols, nz - 2))
    b[:, :, 2] = 1.0 * density_like(s, zt) * gaussian_bump(s, centre, 1.0 / 15.0)
    return dict(nez=nez, N=N, ncols=ncols, ztop=zt, lam=GAMMA_ARK2 * dt, dt=dt,
                b=b.reshape(ncols, n))


def horizontal_tendency(g: np.random.Generator, pts: np.ndarray, nez: int, N: int,
                        ztop: np.ndarray) -> np.ndarray:
    """Explicit (horizontal) tendency H held constant over a step: amplitude
    1e-3 of a state-like profile per hour, times a smooth random field of
    spherical-harmonic degree <= 8 per variable."""
    nz, n = sizes(nez, N)
    s = _s(nz)
    a = density_like(s, ztop)                                   # [ncols, nz]
    prof = np.stack([a, a * 1.0, a * 300.0 * np.exp(s * ztop[:, None] / 8.8e3 * 0.286)], -1)
    f = np.stack([smooth_sphere_field(g, pts) for _ in range(3)], -1)  # [ncols, 3]
    H = 1e-3 * prof * f[:, None, :] / 3600.0
    H[:, 0, 1] = 0.0
    H[:, -1, 1] = 0.0
    return H.reshape(len(pts), n)


def lhevi_ark3(seed: int = 2, ne: int = 30, nez: int = 10, N: int = 4, ztop: float = 30e3,
               dt: float = 300.0, ncols: int | None = None) -> dict:
    """ARK3 LHEVI steps from rest with a seeded horizontal tendency.  The
    initial state is the rest state itself (no increment)."""
    g = rng(seed)
    pts = cubed_sphere_points(ne, 4)
    if ncols is not None:
        pts = pts[:ncols]
    zt = np.full(len(pts), ztop)
    nz, n = sizes(nez, N)
    return dict(nez=nez, N=N, ncols=len(pts), ztop=zt, dt=dt,
                dq=np.zeros((len(pts), n)), H=horizontal_tendency(g, pts, nez, N, zt))


def state_increment(g: np.random.Generator, nez: int, N: int, ztop: np.ndarray,
                    amp: float = 1.0) -> np.ndarray:
    """Increment on the rest state for NHEVI inputs: m = density_like * w with
    w ~ U(-amp, amp) m/s at interior points; Theta = density_like * theta' with
    theta' an amp K Gaussian (centre U(0.25, 0.75) of the column, width 1/15)
    as in ``lhevi_stage``.  Returns [ncols, n]."""
    ztop = np.asarray(ztop, dtype=np.float64)
    count = ztop.size
    nz, n = sizes(nez, N)
    s = _s(nz)
    a = density_like(s, ztop)
    centre = g.uniform(0.25, 0.75, count)
    dq = np.zeros((count, nz, 3))
    dq[:, 1:-1, 1] = a[:, 1:-1] * amp * g.uniform(-1.0, 1.0, (count, nz - 2))
    dq[:, :, 2] = a * amp * gaussian_bump(s, centre, 1.0 / 15.0)
    return dq.reshape(count, n)


def nhevi_ark2(seed: int = 3, ne: int = 30, nez: int = 16, N: int = 3, ztop: float = 30e3,
               dt: float = 300.0, ncols: int | None = None) -> dict:
    """One NHEVI-LU ARK2 step with H = 0 from the rest state plus the
    increment of ``state_increment``."""
    g = rng(seed)
    count = 6 * (ne * 4) ** 2 + 2 if ncols is None else ncols
    nz, n = sizes(nez, N)
    zt = np.full(count, ztop)
    dq = state_increment(g, nez, N, zt)
    return dict(nez=nez, N=N, ncols=count, ztop=zt, dt=dt, dq=dq, H=np.zeros((count, n)))


def batched(seed: int = 4, ncols: int = 200_000, classes=SIZE_CLASSES,
            ztop_range=(30e3, 100e3), dt: float = 300.0) -> dict:
    """Uneven columns: class id uniform over `classes`, top uniform in
    `ztop_range`; per class the same tendency recipe as ``lhevi_ark3`` with
    horizontal positions uniform on the sphere.  Returns per-class blocks."""
    g = rng(seed)
    cls = g.integers(0, len(classes), ncols)
    zt = g.uniform(*ztop_range, ncols)
    pts = sphere_points_uniform(g, ncols)
    blocks = []
    for c, (nez, N) in enumerate(classes):
        idx = np.nonzero(cls == c)[0]
        blocks.append(dict(nez=nez, N=N, cols=idx, ztop=zt[idx],
                           H=horizontal_tendency(g, pts[idx], nez, N, zt[idx])))
    return dict(ncols=ncols, class_of_col=cls.astype(np.int32), ztop=zt, dt=dt, blocks=blocks)


def pack(blocks, ncols: int):
    """Concatenate per-class [cols, n_c] arrays into one packed vector in column
    order, with offsets; returns (flat, offsets)."""
    n_of = np.zeros(ncols, dtype=np.int64)
    for blk in blocks:
        n_of[blk["cols"]] = 3 * (blk["nez"] * blk["N"] + 1)
    off = np.zeros(ncols + 1, dtype=np.int64)
    np.cumsum(n_of, out=off[1:])
    return n_of, off


def serve_requests(seed: int = 5, count: int = 2000, rate: float = 50.0,
                   cols_range=(2000, 86402), steps_range=(1, 20), classes=SIZE_CLASSES,
                   ztop_range=(30e3, 100e3)) -> list:
    """A stream of serving requests: Poisson arrivals at `rate` per second;
    per request a column count and a step count uniform in their ranges, the
    variant LHEVI or NHEVI with probability 1/2, and columns as in ``batched``
    (class uniform, top uniform, tendency from uniform sphere positions),
    packed in column order.  NHEVI requests also start from the rest state
    plus the increment of ``state_increment`` at amplitude 0.1 (dq; at full
    amplitude a few coarse, tall columns go non-physical within a few steps).  Returns a list of dicts
    (rid, arrival, classes, class_of_col, ztop, steps, variant, H, dq)."""
    g = rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += float(g.exponential(1.0 / rate))
        ncols = int(g.integers(cols_range[0], cols_range[1] + 1))
        steps = int(g.integers(steps_range[0], steps_range[1] + 1))
        variant = "LHEVI" if g.random() < 0.5 else "NHEVI"
        cls = g.integers(0, len(classes), ncols).astype(np.int32)
        zt = g.uniform(*ztop_range, ncols)
        pts = sphere_points_uniform(g, ncols)
        blocks = []
        for c, (nez, N) in enumerate(classes):
            idx = np.nonzero(cls == c)[0]
            blocks.append(dict(nez=nez, N=N, cols=idx,
                               H=horizontal_tendency(g, pts[idx], nez, N, zt[idx])))
        n_of, off = pack(blocks, ncols)
        H = np.zeros(int(off[-1]))
        dq = np.zeros(int(off[-1])) if variant == "NHEVI" else None
        for blk in blocks:
            n = 3 * (blk["nez"] * blk["N"] + 1)
            if len(blk["cols"]):
                pos = (off[blk["cols"]][:, None] + np.arange(n)[None, :]).reshape(-1)
                H[pos] = blk["H"].reshape(-1)
                if dq is not None:
                    dq[pos] = state_increment(g, blk["nez"], blk["N"], zt[blk["cols"]],
                                              amp=0.1).reshape(-1)
        out.append(dict(rid=i, arrival=t, classes=list(classes), class_of_col=cls, ztop=zt,
                        steps=steps, variant=variant, H=H, dq=dq))
    return out


def serve_bank(seed: int = 6, cols_per_class: int = 32768, classes=SIZE_CLASSES,
               ztop_range=(30e3, 100e3), nhevi_amp: float = 0.1) -> list:
    """Column banks for a long serving stream: per size class cols_per_class
    columns drawn as in ``batched`` (model top uniform, tendency H from
    uniform sphere positions) with the NHEVI start increment dq of
    ``state_increment`` at amplitude nhevi_amp (see ``serve_requests``).
    Requests of ``serve_stream`` take windows of these banks, so a stream of
    thousands of large requests needs no per-request field evaluation.
    Returns [dict(cls, ztop [cols], H [cols, n], dq [cols, n])] per class."""
    g = rng(seed)
    bank = []
    for nez, N in classes:
        zt = g.uniform(*ztop_range, cols_per_class)
        pts = sphere_points_uniform(g, cols_per_class)
        H = horizontal_tendency(g, pts, nez, N, zt)
        dq = state_increment(g, nez, N, zt, amp=nhevi_amp)
        bank.append(dict(cls=(nez, N), ztop=zt, H=H, dq=dq))
    return bank


def serve_stream(seed: int = 5, count: int = 2000, rate: float = 50.0,
                 cols_range=(2000, 86402), steps_range=(1, 20), nclasses: int = 4,
                 bank_cols: int = 32768) -> list:
    """A Poisson stream of serving requests over banks of ``serve_bank``:
    arrivals at `rate` per second from the stream's seed; per request, from
    its own seed (the stream seed and its index), a column count and a step
    count uniform in their ranges, the variant LHEVI or NHEVI with probability
    1/2, the columns' classes uniform (a multinomial split of the count) and,
    per class, a window of that class's bank at a uniform start.  Returns a
    list of dicts (rid, arrival, steps, variant, parts=[(class, start, count)])."""
    g = rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += float(g.exponential(1.0 / rate))
        gr = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, i])))
        ncols = int(gr.integers(cols_range[0], cols_range[1] + 1))
        steps = int(gr.integers(steps_range[0], steps_range[1] + 1))
        variant = "LHEVI" if gr.random() < 0.5 else "NHEVI"
        split = gr.multinomial(ncols, [1.0 / nclasses] * nclasses)
        parts = []
        for c, m in enumerate(split):
            m = int(m)
            if m == 0:
                continue
            if m > bank_cols:
                raise ValueError("a class block is larger than its bank")
            parts.append((c, int(gr.integers(0, bank_cols - m + 1)), m))
        out.append(dict(rid=i, arrival=t, steps=steps, variant=variant, parts=parts))
    return out
