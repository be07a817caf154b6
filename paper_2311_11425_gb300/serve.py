"""Continuous serving of column-solve requests under an HBM budget.

A request is a set of columns (size classes, model tops), a horizontal
tendency H held over its steps, a step count and a variant: LHEVI-PS
(Sec. 4.3, one band factorisation per step and one stage solve per implicit
stage) or NHEVI-LU (Sec. 4.2, one Newton solve per implicit stage).  Each
admitted request owns a context with its factors, state and workspace resident
on the device and its own CUDA stream; the scheduler keeps a bounded number
of steps in flight per request and admits queued requests in arrival order
whenever the device bytes they need (the library's exact estimate plus their
state buffers) fit the budget.  Kernels of different requests run
concurrently on their streams, so small requests share the GPU the way one
large batch would, and a request finishing frees its memory for the next.

Every step runs in the library's kernels; this module is host-side
scheduling and bookkeeping only.  A request's result does not depend on what
it is served with: its context, buffers and stream are its own and the
kernels are deterministic.
"""

from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import (FP32_IR, LHEVI, NHEVI, Context, HeviError, hevi_estimate_bytes, tableau)


@dataclass
class Request:
    rid: int
    classes: list                 # [(nez, N), ...]
    class_of_col: np.ndarray      # int32 per column (None with one class)
    ztop: np.ndarray              # per-column model top [m]
    steps: int
    variant: str                  # "LHEVI" or "NHEVI"
    H: np.ndarray                 # packed state layout (column order), FP64
    arrival: float = 0.0          # seconds after the start of the run
    q0: np.ndarray | None = None  # initial state; None = the reference state
    dq: np.ndarray | None = None  # with q0 None: start from the reference state + dq

    @property
    def ncols(self) -> int:
        return len(self.ztop)


@dataclass
class Result:
    rid: int
    q: np.ndarray | None          # final state (host), None if rejected / failed
    error: str | None
    arrival: float
    admitted: float
    done: float
    ncols: int
    steps: int

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass(eq=False)
class _Active:
    req: Request
    ctx: Context
    stream: object
    qa: object
    qb: object
    H: object
    nbytes: int
    admitted: float
    enq: int = 0
    events: list = field(default_factory=list)


class Server:
    """Scheduler over one device.

    hbm_budget: bytes the served requests may hold on the device at once.
    tab / dt: the ARK tableau (name) and step; precision: FP32_IR or FP64;
    rtol / max_iter: the Newton stop of NHEVI-LU; inflight: steps enqueued
    ahead per request.
    """

    def __init__(self, hbm_budget: int, tab: str = "ARK3", dt: float = 300.0,
                 precision=FP32_IR, rtol: float = 1e-10, max_iter: int = 20, inflight: int = 2):
        self.budget = int(hbm_budget)
        self.tab = tableau(tab)
        self.dt = float(dt)
        self.precision = precision
        self.rtol, self.max_iter = float(rtol), int(max_iter)
        self.inflight = max(1, int(inflight))
        self.peak_bytes = 0

    def request_bytes(self, r: Request) -> int:
        kind = LHEVI if r.variant == "LHEVI" else NHEVI
        lib = hevi_estimate_bytes(r.classes, r.class_of_col, r.ncols, self.precision, kind,
                                  self.tab.s)
        n = int(r.H.size)
        return lib + 3 * n * 8  # plus q_a, q_b and H

    def _admit(self, r: Request, now: float) -> _Active:
        import torch
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            ctx = Context(r.classes, r.ztop, class_of_col=r.class_of_col, ncols=r.ncols,
                          precision=self.precision, stream=stream)
            H = torch.from_numpy(np.ascontiguousarray(r.H, dtype=np.float64).reshape(-1))
            H = H.pin_memory().to(ctx.device, non_blocking=True)
            if r.q0 is None:
                qa = ctx.hevi_reference_state()
                if r.dq is not None:
                    dq = torch.from_numpy(np.ascontiguousarray(r.dq, dtype=np.float64).reshape(-1))
                    qa += dq.pin_memory().to(ctx.device, non_blocking=True)
            else:
                q0 = torch.from_numpy(np.ascontiguousarray(r.q0, dtype=np.float64).reshape(-1))
                qa = q0.pin_memory().to(ctx.device, non_blocking=True)
            qb = torch.empty_like(qa)
        return _Active(r, ctx, stream, qa, qb, H, self.request_bytes(r), now)

    def _enqueue_step(self, a: _Active):
        import torch
        with torch.cuda.stream(a.stream):
            if a.req.variant == "LHEVI":
                a.ctx.hevi_lhevi_step(self.tab, self.dt, a.qa, a.H, a.qb)
            else:
                a.ctx.hevi_nhevi_step(self.tab, self.dt, a.qa, a.H, a.qb, rtol=self.rtol,
                                      max_iter=self.max_iter)
            ev = torch.cuda.Event()
            ev.record(a.stream)
        a.qa, a.qb = a.qb, a.qa
        a.enq += 1
        a.events.append(ev)

    def run(self, requests, realtime: bool = True) -> list[Result]:
        """Serve `requests`; with realtime, request i becomes visible at
        start + arrival_i (wall clock), otherwise all are queued at once.
        Returns one Result per request, in request order."""
        import torch
        order = sorted(range(len(requests)), key=lambda i: requests[i].arrival)
        pending = [requests[i] for i in order]
        queue: list[Request] = []
        active: list[_Active] = []
        results: dict[int, Result] = {}
        in_use = 0
        t0 = time.perf_counter()
        clock = lambda: time.perf_counter() - t0  # noqa: E731
        while pending or queue or active:
            now = clock()
            while pending and (not realtime or pending[0].arrival <= now):
                queue.append(pending.pop(0))
            # admission in arrival order under the budget
            while queue:
                r = queue[0]
                need = self.request_bytes(r)
                if need > self.budget:
                    queue.pop(0)
                    results[r.rid] = Result(r.rid, None, "exceeds the HBM budget", r.arrival,
                                            now, now, r.ncols, r.steps)
                    continue
                if in_use + need > self.budget:
                    break
                queue.pop(0)
                try:
                    a = self._admit(r, now)
                except HeviError as e:
                    results[r.rid] = Result(r.rid, None, str(e), r.arrival, now, clock(),
                                            r.ncols, r.steps)
                    continue
                in_use += need
                self.peak_bytes = max(self.peak_bytes, in_use)
                active.append(a)
            # keep up to `inflight` steps queued per request
            for a in active:
                while a.enq < a.req.steps and len(a.events) < self.inflight:
                    self._enqueue_step(a)
            # retire finished steps and requests
            progressed = False
            for a in list(active):
                while a.events and a.events[0].query():
                    a.events.pop(0)
                    progressed = True
                if a.enq == a.req.steps and not a.events:
                    err = None
                    q = None
                    try:
                        a.ctx.hevi_sync()
                        q = a.qa.cpu().numpy()  # the last step wrote what is now qa
                    except HeviError as e:
                        err = str(e)
                    results[a.req.rid] = Result(a.req.rid, q, err, a.req.arrival, a.admitted,
                                                clock(), a.req.ncols, a.req.steps)
                    a.ctx.close()
                    a.qa = a.qb = a.H = None  # the request's buffers go back to the pool
                    active.remove(a)
                    in_use -= a.nbytes
                    progressed = True
            if not progressed:
                if active:
                    time.sleep(2e-4)
                elif pending and realtime:
                    time.sleep(max(0.0, min(1e-3, pending[0].arrival - clock())))
        torch.cuda.synchronize()
        return [results[r.rid] for r in requests]


def latency_stats(results) -> dict:
    """p50 / p99 / max latency (s) and throughput of the served requests."""
    ok = [r for r in results if r.error is None]
    if not ok:
        return {"served": 0}
    lat = np.array([r.latency for r in ok])
    span = max(r.done for r in ok) - min(r.arrival for r in ok)
    col_steps = sum(r.ncols * r.steps for r in ok)
    return {"served": len(ok), "rejected": len(results) - len(ok),
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "max_s": float(lat.max()), "makespan_s": float(span),
            "column_steps_per_s": float(col_steps / span) if span > 0 else None}
