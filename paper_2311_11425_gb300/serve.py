"""Continuous serving of column-integration requests from resident slot pools.

A request is a set of columns (size classes, model tops), a horizontal
tendency H held over its steps, a step count and a variant: LHEVI-PS
(Sec. 4.3, one band factorisation per step and one stage solve per implicit
stage) or NHEVI-LU (Sec. 4.2, one Newton solve per implicit stage).

The server is continuous batching over columns.  Each variant owns one
long-lived context, a slot pool: a fixed number of column slots per size
class, laid out class by class in granules of 32 columns (one tile of the
kernels), with its factors, state, tendency and workspace resident on the
device and its own CUDA stream.  The whole pool advances by one time step
per tick (one hevi_lhevi_step or hevi_nhevi_step call over every slot), so
the columns of all admitted requests share each launch the way one large
batch would.  Admitting a request takes free granules for each of its
classes (lowest first; a class block may span several runs), gives those slots the request's model tops
(hevi_set_column_tops) and writes its initial state and tendency into them;
after its last tick its slots are copied to the host and handed back, reset
to the rest state with zero tendency.  Admission and release are stream-
ordered between ticks and allocate no device memory: the pools are the only
device allocations, made once, and together must fit the HBM budget.

Columns are independent in every kernel (one column per lane or thread, its
own stop tests), so a request's result does not depend on which slots it got
or what it was served with: bit for bit the result of the same columns run
alone.  Every step runs in the library's kernels; this module is host-side
scheduling and bookkeeping only.
"""

from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import FP32_IR, LHEVI, NHEVI, Context, hevi_estimate_bytes, tableau

GRANULE = 32  # columns per granule: one tile of the kernels


@dataclass
class Block:
    """Columns of one size class of a request, in the request's order:
    model tops [cols], tendency H and optional initial increment dq (packed
    state layout of these columns, FP64)."""
    cls: tuple                    # (nez, N)
    ztop: np.ndarray
    H: np.ndarray
    dq: np.ndarray | None = None


@dataclass
class Request:
    rid: int
    classes: list = None          # [(nez, N), ...]
    class_of_col: np.ndarray = None   # int32 per column (None with one class)
    ztop: np.ndarray = None       # per-column model top [m]
    steps: int = 1
    variant: str = "LHEVI"        # "LHEVI" or "NHEVI"
    H: np.ndarray = None          # packed state layout (column order), FP64
    arrival: float = 0.0          # seconds after the start of the run
    dq: np.ndarray | None = None  # start from the rest state + dq (None: the rest state)
    blocks: list | None = None    # alternatively the columns as class blocks (Block)
    _grouped: list | None = field(default=None, repr=False, compare=False)

    @property
    def ncols(self) -> int:
        if self.blocks is not None:
            return int(sum(len(b.ztop) for b in self.blocks))
        return len(self.ztop)

    def as_blocks(self):
        """[(Block, cols)]: the request's columns grouped by class; cols are
        the request's column indices of each block (None for ``blocks``
        requests, whose columns are the blocks one after another)."""
        if self.blocks is not None:
            return [(b, None) for b in self.blocks]
        if self._grouped is not None:
            return self._grouped
        cls = (np.zeros(len(self.ztop), np.int32) if self.class_of_col is None
               else np.asarray(self.class_of_col, np.int32))
        n_of = np.array([3 * (nez * N + 1) for nez, N in self.classes], np.int64)[cls]
        off = np.concatenate([[0], np.cumsum(n_of)])
        out = []
        for c, (nez, N) in enumerate(self.classes):
            cols = np.nonzero(cls == c)[0]
            if not len(cols):
                continue
            n = 3 * (nez * N + 1)
            pos = (off[cols][:, None] + np.arange(n)[None, :]).reshape(-1)
            dq = None if self.dq is None else np.asarray(self.dq)[pos]
            out.append((Block((nez, N), np.asarray(self.ztop)[cols], np.asarray(self.H)[pos], dq),
                        cols))
        self._grouped = out
        return out


@dataclass
class Result:
    rid: int
    q: np.ndarray | None          # final state (host, the request's layout); None if not kept
    error: str | None
    arrival: float
    admitted: float
    done: float
    ncols: int
    steps: int
    variant: str = "LHEVI"

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class GranuleAllocator:
    """First-fit allocator of contiguous granule runs in one class's slots."""

    def __init__(self, count: int):
        self.count = int(count)
        self.free = [(0, self.count)]  # disjoint (start, length), sorted by start

    @property
    def free_granules(self) -> int:
        return sum(n for _, n in self.free)

    def alloc(self, n: int):
        """Start of a run of n free granules, or None."""
        for i, (s, m) in enumerate(self.free):
            if m >= n:
                if m == n:
                    self.free.pop(i)
                else:
                    self.free[i] = (s + n, m - n)
                return s
        return None

    def alloc_split(self, n: int):
        """Runs [(start, length)] covering n granules, lowest addresses
        first, or None if fewer than n are free."""
        if self.free_granules < n:
            return None
        out = []
        while n > 0:
            s, m = self.free[0]
            k = min(m, n)
            out.append((s, k))
            if k == m:
                self.free.pop(0)
            else:
                self.free[0] = (s + k, m - k)
            n -= k
        return out

    def release(self, start: int, n: int):
        i = 0
        while i < len(self.free) and self.free[i][0] < start:
            i += 1
        if i > 0:
            ps, pn = self.free[i - 1]
            assert ps + pn <= start, "granules released twice"
        if i < len(self.free):
            assert start + n <= self.free[i][0], "granules released twice"
        self.free.insert(i, (start, n))
        # merge with the neighbours
        if i + 1 < len(self.free) and start + n == self.free[i + 1][0]:
            self.free[i] = (start, n + self.free[i + 1][1])
            self.free.pop(i + 1)
        if i > 0 and self.free[i - 1][0] + self.free[i - 1][1] == start:
            self.free[i - 1] = (self.free[i - 1][0], self.free[i - 1][1] + self.free[i][1])
            self.free.pop(i)


def _slots(classes, slots_per_class) -> list:
    per = ([int(slots_per_class)] * len(classes) if np.isscalar(slots_per_class)
           else [int(s) for s in slots_per_class])
    if len(per) != len(classes) or min(per) < 1:
        raise ValueError("one positive slot count per size class")
    return [-(-s // GRANULE) * GRANULE for s in per]


def pool_bytes(classes, slots_per_class, variant: str, precision=FP32_IR, stages: int = 4) -> int:
    """Device bytes of one slot pool: the context (the library's exact
    estimate for a step of `stages` stages) plus its two state buffers and
    the tendency."""
    cap = _slots(classes, slots_per_class)
    cls = np.repeat(np.arange(len(classes), dtype=np.int32), cap)
    kind = LHEVI if variant == "LHEVI" else NHEVI
    lib = hevi_estimate_bytes([tuple(c) for c in classes], cls, len(cls), precision, kind, stages)
    n = sum(c * 3 * (nez * N + 1) for c, (nez, N) in zip(cap, classes))
    return lib + 3 * n * 8


def _host(x):
    import torch
    return x if isinstance(x, torch.Tensor) else torch.from_numpy(
        np.ascontiguousarray(x, dtype=np.float64).reshape(-1))


@dataclass
class _Part:
    """Columns [lo, lo + ncols) of one class block in the slots [first,
    first + ncols) of a granule run; a, e: their state range in the pool."""
    cls: int
    first: int
    ncols: int
    granule: int
    granules: int
    a: int
    e: int
    block: Block
    lo: int
    cols: np.ndarray | None


@dataclass(eq=False)
class _Placed:
    req: Request
    parts: list                   # [_Part]
    admitted: float
    first_tick: int
    last_tick: int
    done_event: object = None
    bad: object = None            # pinned host flag: a column failed or went non-finite


class SlotPool:
    """One variant's resident context of column slots (see the module text)."""

    def __init__(self, variant, classes, slots_per_class, tab, dt, precision=FP32_IR,
                 rtol=1e-10, max_iter=20):
        import torch
        self.variant = variant
        self.classes = [tuple(c) for c in classes]
        self.cap = _slots(self.classes, slots_per_class)
        self.first_col = np.concatenate([[0], np.cumsum(self.cap)])[:-1].astype(np.int64)
        cls = np.repeat(np.arange(len(self.classes), dtype=np.int32), self.cap)
        self.tab, self.dt, self.rtol, self.max_iter = tab, float(dt), float(rtol), int(max_iter)
        self.stream = torch.cuda.Stream()
        self.ctx = Context(self.classes, 30e3, class_of_col=cls, ncols=len(cls),
                           precision=precision, stream=self.stream)
        if variant == "NHEVI":
            self.ctx.hevi_set_newton_host_check(False)  # a tick never blocks the scheduler
        self.off = self.ctx.offsets()
        with torch.cuda.stream(self.stream):
            self.q = [self.ctx.hevi_reference_state(), self.ctx.hevi_reference_state()]
            self.H = torch.zeros_like(self.q[0])
        self.stage = torch.empty(self.ctx.n, dtype=torch.float64, pin_memory=True)
        self.stage_np = self.stage.numpy()
        self.cur = 0                  # the buffer the next tick reads
        self.alloc = [GranuleAllocator(c // GRANULE) for c in self.cap]
        self.ticks = 0                # ticks enqueued
        self.tick_events = []         # (start, end) of every tick
        self._pending_ends = []       # end events of ticks not yet seen complete
        self.placed: list[_Placed] = []
        self.column_steps = 0         # request column-steps completed
        self.nbytes = self.ctx.device_bytes + 3 * self.ctx.n * 8

    # -- admission and release --------------------------------------------------
    def check(self, req: Request) -> str | None:
        """Why the request can never be placed here, or None."""
        for b, _ in req.as_blocks():
            if tuple(b.cls) not in self.classes:
                return f"size class {tuple(b.cls)} not served"
            c = self.classes.index(tuple(b.cls))
            if -(-len(b.ztop) // GRANULE) > self.alloc[c].count:
                return "more columns of a class than the pool holds"
        return None

    def try_place(self, req: Request, now: float) -> bool:
        """Place the request if each of its class blocks finds enough free
        granules (a block may span several runs); all or nothing."""
        import torch
        blocks = req.as_blocks()
        runs = []
        for b, cols in blocks:
            c = self.classes.index(tuple(b.cls))
            got = self.alloc[c].alloc_split(-(-len(b.ztop) // GRANULE))
            if got is None:
                for c2, got2 in runs:
                    for s2, g2 in got2:
                        self.alloc[c2].release(s2, g2)
                return False
            runs.append((c, got))
        parts = []
        for (b, cols), (c, got) in zip(blocks, runs):
            nez, N = b.cls
            n = 3 * (nez * N + 1)
            lo = 0
            for s0, g in got:
                m = min(g * GRANULE, len(b.ztop) - lo)
                f = int(self.first_col[c] + s0 * GRANULE)
                parts.append(_Part(c, f, m, s0, g, int(self.off[f]), int(self.off[f + m]), b, lo,
                                   None if cols is None else cols[lo:lo + m]))
                lo += m
        with torch.cuda.stream(self.stream):
            q, scratch = self.q[self.cur], self.q[1 - self.cur]
            for pt in parts:
                b, n = pt.block, (pt.e - pt.a) // pt.ncols
                self.ctx.hevi_set_column_tops(pt.first, b.ztop[pt.lo:pt.lo + pt.ncols])
                self.ctx.hevi_reference_columns(pt.first, pt.ncols, q)
                self.H[pt.a:pt.e].copy_(_host(b.H)[pt.lo * n:(pt.lo + pt.ncols) * n],
                                        non_blocking=True)
                if b.dq is not None:
                    # the other buffer is free until the next tick overwrites it
                    scratch[pt.a:pt.e].copy_(_host(b.dq)[pt.lo * n:(pt.lo + pt.ncols) * n],
                                             non_blocking=True)
                    q[pt.a:pt.e].add_(scratch[pt.a:pt.e])
        self.placed.append(_Placed(req, parts, now, self.ticks, self.ticks + req.steps - 1))
        return True

    def _release(self, p: _Placed):
        import torch
        with torch.cuda.stream(self.stream):
            for pt in p.parts:
                self.H[pt.a:pt.e].zero_()
                self.ctx.hevi_reference_columns(pt.first, pt.ncols, self.q[self.cur])
                self.alloc[pt.cls].release(pt.granule, pt.granules)
        self.placed.remove(p)

    # -- ticks -----------------------------------------------------------------
    def needs_tick(self) -> bool:
        return any(p.last_tick >= self.ticks for p in self.placed)

    def inflight(self) -> int:
        while self._pending_ends and self._pending_ends[0].query():
            self._pending_ends.pop(0)
        return len(self._pending_ends)

    def tick(self):
        """Enqueue one time step of every slot; then the copy-out of the
        requests whose last step it was."""
        import torch
        with torch.cuda.stream(self.stream):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            qi, qo = self.q[self.cur], self.q[1 - self.cur]
            if self.variant == "LHEVI":
                self.ctx.hevi_lhevi_step(self.tab, self.dt, qi, self.H, qo)
            else:
                self.ctx.hevi_nhevi_step(self.tab, self.dt, qi, self.H, qo, rtol=self.rtol,
                                         max_iter=self.max_iter)
            e1.record(self.stream)
            self.cur ^= 1
            t = self.ticks
            self.ticks += 1
            self.tick_events.append((e0, e1))
            self._pending_ends.append(e1)
            finishing = [p for p in self.placed if p.last_tick == t]
            if finishing:
                st, _ = self.ctx.hevi_column_status()
            for p in finishing:
                flags = []
                for pt in p.parts:
                    self.stage[pt.a:pt.e].copy_(qo[pt.a:pt.e], non_blocking=True)
                    flags.append((st[pt.first:pt.first + pt.ncols] != 0).any())
                    flags.append((~torch.isfinite(qo[pt.a:pt.e])).any())
                p.bad = torch.empty((), dtype=torch.bool, pin_memory=True)
                p.bad.copy_(torch.stack(flags).any(), non_blocking=True)
                p.done_event = torch.cuda.Event()
                p.done_event.record(self.stream)

    def retire(self, clock, keep_state: bool) -> list:
        out = []
        for p in list(self.placed):
            if p.done_event is None or not p.done_event.query():
                continue
            q = self._gather(p) if keep_state else None
            err = "a column failed or went non-finite" if bool(p.bad.item()) else None
            r = p.req
            self._release(p)
            self.column_steps += r.ncols * r.steps
            out.append(Result(r.rid, q, err, r.arrival, p.admitted, clock(), r.ncols, r.steps,
                              r.variant))
        return out

    def _gather(self, p: _Placed) -> np.ndarray:
        """The request's final state from the staging copy, in its layout."""
        if p.req.blocks is not None:
            return np.concatenate([self.stage_np[pt.a:pt.e] for pt in p.parts])
        req = p.req
        cls = (np.zeros(req.ncols, np.int32) if req.class_of_col is None
               else np.asarray(req.class_of_col, np.int32))
        n_of = np.array([3 * (nez * N + 1) for nez, N in req.classes], np.int64)[cls]
        off = np.concatenate([[0], np.cumsum(n_of)])
        out = np.empty(int(off[-1]))
        for pt in p.parts:
            m = (pt.e - pt.a) // pt.ncols
            pos = (off[pt.cols][:, None] + np.arange(m)[None, :]).reshape(-1)
            out[pos] = self.stage_np[pt.a:pt.e]
        return out

    def close(self):
        self.ctx.close()
        self.q = self.H = None


class Server:
    """Continuous batching of requests over one slot pool per variant.

    classes: the size classes served; slots_per_class: columns per class in
    each pool (an int or one per class, rounded up to granules of 32);
    hbm_budget: device bytes the pools may hold together (checked once, when
    the pools are made: admission then allocates nothing); tab / dt: the ARK
    tableau (name) and step; rtol / max_iter: the Newton stop of NHEVI-LU;
    inflight: ticks enqueued ahead per pool; keep_state: return each
    request's final state (else only its status and times).
    """

    def __init__(self, classes, slots_per_class=65536, hbm_budget: int = 150 * 10**9,
                 tab: str = "ARK3", dt: float = 300.0, precision=FP32_IR, rtol: float = 1e-10,
                 max_iter: int = 20, inflight: int = 2, variants=("LHEVI", "NHEVI"),
                 keep_state: bool = True):
        self.classes = [tuple(c) for c in classes]
        self.tab = tableau(tab)
        self.budget = int(hbm_budget)
        self.inflight = max(1, int(inflight))
        self.keep_state = bool(keep_state)
        self.pool_bytes = {v: pool_bytes(self.classes, slots_per_class, v, precision, self.tab.s)
                           for v in variants}
        if sum(self.pool_bytes.values()) > self.budget:
            raise ValueError(f"slot pools need {sum(self.pool_bytes.values())} bytes, "
                             f"above the HBM budget of {self.budget}")
        self.pools = {v: SlotPool(v, self.classes, slots_per_class, self.tab, dt, precision,
                                  rtol, max_iter) for v in variants}
        self.device_bytes = sum(p.nbytes for p in self.pools.values())
        self.stats = {}

    def close(self):
        for p in self.pools.values():
            p.close()
        self.pools = {}

    def run(self, requests, realtime: bool = True, time_limit: float | None = None) -> list:
        """Serve `requests`; with realtime, request i becomes visible at
        start + arrival_i (wall clock), otherwise all are queued at once.
        time_limit (s): stop admitting and enqueueing after it, finish the
        ticks in flight and report the requests not completed as such.
        Returns one Result per request, in request order; self.stats holds
        the run's GPU-busy fraction and per-variant figures."""
        import torch
        from collections import deque
        order = sorted(range(len(requests)), key=lambda i: requests[i].arrival)
        pending = deque(requests[i] for i in order)
        queues = {v: deque() for v in self.pools}
        results: dict[int, Result] = {}
        base = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        base.record()
        t0 = time.perf_counter()
        clock = lambda: time.perf_counter() - t0  # noqa: E731
        cut = False
        while pending or any(queues.values()) or any(p.placed for p in self.pools.values()):
            now = clock()
            if time_limit is not None and now > time_limit and not cut:
                cut = True
                for q in queues.values():
                    for r in q:
                        results[r.rid] = Result(r.rid, None, "not admitted within the time limit",
                                                r.arrival, now, now, r.ncols, r.steps, r.variant)
                    q.clear()
                for r in pending:
                    results[r.rid] = Result(r.rid, None, "not admitted within the time limit",
                                            r.arrival, now, now, r.ncols, r.steps, r.variant)
                pending.clear()
            while pending and (not realtime or pending[0].arrival <= now):
                r = pending.popleft()
                pool = self.pools.get(r.variant)
                why = f"variant {r.variant} not served" if pool is None else pool.check(r)
                if why:
                    results[r.rid] = Result(r.rid, None, why, r.arrival, now, now, r.ncols,
                                            r.steps, r.variant)
                else:
                    queues[r.variant].append(r)
            for v, pool in self.pools.items():
                q = queues[v]
                while q and pool.try_place(q[0], now):  # first come, first served
                    q.popleft()
            progressed = False
            for pool in self.pools.values():
                while pool.needs_tick() and pool.inflight() < self.inflight:
                    pool.tick()
                    progressed = True
                for res in pool.retire(clock, self.keep_state):
                    results[res.rid] = res
                    progressed = True
            if not progressed:
                if any(p.placed for p in self.pools.values()):
                    time.sleep(2e-4)
                elif pending and realtime:
                    time.sleep(max(0.0, min(1e-3, pending[0].arrival - clock())))
        torch.cuda.synchronize()
        wall = clock()
        self.stats = self._stats(base, wall)
        return [results[r.rid] for r in requests]

    def _stats(self, base, wall: float) -> dict:
        """GPU-busy fraction (the union of all ticks over the run) and per
        pool its ticks, busy time and served column-steps."""
        spans, out = [], {}
        for v, p in self.pools.items():
            iv = [(base.elapsed_time(a), base.elapsed_time(b)) for a, b in p.tick_events]
            busy = _union_ms(iv)
            spans += iv
            out[v] = {"ticks": p.ticks, "busy_s": busy * 1e-3,
                      "tick_ms_mean": (sum(b - a for a, b in iv) / len(iv)) if iv else None,
                      "slots": int(sum(p.cap)), "request_column_steps": p.column_steps,
                      "column_steps_per_busy_s": (p.column_steps / (busy * 1e-3)) if busy else None}
        busy = _union_ms(spans) * 1e-3
        return {"wall_s": wall, "gpu_busy_s": busy, "gpu_busy_fraction": busy / wall if wall else None,
                "variants": out, "pool_bytes": self.pool_bytes, "hbm_budget": self.budget}


def _union_ms(iv) -> float:
    tot, end = 0.0, -float("inf")
    for a, b in sorted(iv):
        if b <= end:
            continue
        tot += b - max(a, end)
        end = b
    return tot


def latency_stats(results) -> dict:
    """p50 / p99 / max latency (s) and throughput of the served requests,
    overall and per variant."""
    ok = [r for r in results if r.error is None]
    if not ok:
        return {"served": 0, "not_served": len(results)}
    lat = np.array([r.latency for r in ok])
    span = max(r.done for r in ok) - min(r.arrival for r in ok)
    col_steps = sum(r.ncols * r.steps for r in ok)
    out = {"served": len(ok), "not_served": len(results) - len(ok),
           "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
           "max_s": float(lat.max()), "makespan_s": float(span),
           "column_steps_per_s": float(col_steps / span) if span > 0 else None,
           "columns_per_s": float(sum(r.ncols for r in ok) / span) if span > 0 else None}
    for v in sorted({r.variant for r in ok}):
        sub = [r for r in ok if r.variant == v]
        lv = np.array([r.latency for r in sub])
        out[v] = {"served": len(sub), "p50_s": float(np.percentile(lv, 50)),
                  "p99_s": float(np.percentile(lv, 99)),
                  "column_steps": int(sum(r.ncols * r.steps for r in sub))}
    return out
