#!/usr/bin/env python
"""Benchmark of the HEVI vertical column solve on GB300.

Workload (one "step"): one LHEVI ARK3 time step (Sec. 4.3, Sec. 6) on
86,402 columns of Nez = 10 elements of order N = 4 (41 points, 123 unknowns)
with a 30 km top and dt = 300 s: one band factorisation linearised about q^n,
three implicit stage solves (FP32 LU + FP64 iterative refinement), the
vertical operator applies and the stage combinations, advancing the state in
place from rest under a seeded horizontal tendency.  Metric: implicit column
stage solves per second (3 x columns per step), whole job.

Also reported: the same step with plain FP64 factors (one column per thread),
an end-to-end number through the C ABI with host buffers, per-kernel times
from CUDA events on the library's stream, the dominant kernel's roofline, SM
clocks during the timed region, and the FP64 CPU oracle timed on the host
cores on a bounded sample of the same workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""

from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NE, NEZ, ORDER, ZTOP, DT = 30, 10, 4, 30e3, 300.0
NCOLS = 6 * (NE * 4) ** 2 + 2          # 86,402 cubed-sphere columns
NZ = NEZ * ORDER + 1
NUNK = 3 * NZ
K_BAND = 3 * (ORDER + 1) - 1
LDAB = 3 * K_BAND + 1
STAGES = 3                              # implicit stages of ARK3
WORKLOAD = (f"lhevi_ark3: {NCOLS} columns, Nez={NEZ}, N={ORDER}, ztop=30 km, dt=300 s, "
            f"ARK3 (3 implicit stages), LHEVI-PS, seeded horizontal tendency")

# Algorithmic bytes of one column stage solve: FP32 factors (ldab n 4), pivots
# (n bytes) and b, x, q0 (3 n 8); FP64 plain: FP64 factors, int pivots, b, x.
BYTES_SOLVE_FP32IR = LDAB * NUNK * 4 + NUNK + 3 * NUNK * 8
BYTES_SOLVE_FP64 = LDAB * NUNK * 8 + NUNK * 4 + 2 * NUNK * 8


def factor_flops(n=NUNK, k=K_BAND):
    """FP32 flops of one band LU with partial pivoting (dgbtrf loop counts)."""
    f = 0
    for j in range(n):
        nr = min(k, n - 1 - j)
        nc = min(2 * k, n - 1 - j)
        f += nr + 2 * nr * nc
    return f


# DRAM bytes (read + write) per launch of the dominant kernels from one ncu
# capture of `python bench.py --ncu-case solve|factor` (the summaries under
# profiles/ give the commands), valid only for the kernel source they were
# taken from: the SHA-256 of the kernel file at capture time.
NCU_TRAFFIC = {
    "k_solve_ir": {"bytes": 5747106304, "sha256": "789402adba2d5dc127ace1b65664104d0290a7d6097cf9c4ef0f29e48b056947"},
    "k_solve_tail": {"bytes": 1846539520, "sha256": "789402adba2d5dc127ace1b65664104d0290a7d6097cf9c4ef0f29e48b056947"},
    "k_factor_r": {"bytes": 2517796096, "sha256": "789402adba2d5dc127ace1b65664104d0290a7d6097cf9c4ef0f29e48b056947"},
}
KERNEL_SOURCE = os.path.join(ROOT, "paper_2311_11425_gb300", "csrc", "hevi_kernels.cu")


def ncu_traffic(kernel):
    import hashlib
    rec = NCU_TRAFFIC.get(kernel)
    if not rec:
        return None
    with open(KERNEL_SOURCE, "rb") as fh:
        digest = hashlib.sha256(fh.read()).hexdigest()
    return rec["bytes"] if digest == rec["sha256"] else None


def peaks():
    p = {"hbm_gbs": 6777.0, "source": "fallback"}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            m = json.load(fh)
        p["hbm_gbs"] = float(m["hbm_gbs"])
        p["source"] = "measured"
    except Exception:
        pass
    # FP32 ALU peak from unit counts: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz
    p["fp32_tflops"] = 152 * 128 * 2 * 2.07e9 / 1e12
    return p


# ---------------------------------------------------------------------------
# CPU oracle (FP64, host cores)
# ---------------------------------------------------------------------------

def _oracle_chunk(args):
    qn, H, ztop = args
    import oracle
    from oracle import tableaux
    out, info = oracle.lhevi_step(NEZ, ORDER, ztop, tableaux.ARK3, DT, qn, H, lin=0)
    return int((info != 0).sum())


def oracle_sample_inputs(ncols):
    import numpy as np
    import hevi_inputs
    import oracle
    inp = hevi_inputs.lhevi_ark3(seed=2, ncols=ncols)
    q = oracle.reference_q(NEZ, ORDER, ZTOP, ncols)
    return q, inp["H"], np.full(ncols, ZTOP)


def cpu_oracle_rate(pool, cores, target_s=12.0):
    """Time the oracle's LHEVI ARK3 step on a bounded sample of the workload's
    columns, spread over `cores` worker processes.  Returns (col-solves/s, dict)."""
    import numpy as np
    q, H, zt = oracle_sample_inputs(64)
    t0 = time.perf_counter()
    _oracle_chunk((q[:16], H[:16], zt[:16]))
    per_col = (time.perf_counter() - t0) / 16
    ncols = int(max(cores, min(NCOLS, target_s / per_col * cores)))
    q, H, zt = oracle_sample_inputs(ncols)
    chunks = [(q[i::cores], H[i::cores], zt[i::cores]) for i in range(cores)]
    t0 = time.perf_counter()
    bad = sum(pool.map(_oracle_chunk, chunks)) if pool else _oracle_chunk((q, H, zt))
    wall = time.perf_counter() - t0
    rate = STAGES * ncols / wall
    return rate, {"value": rate, "unit": "column-solves/s", "cores": cores, "kind": "oracle",
                  "sample": f"one FP64 oracle LHEVI ARK3 step on the first {ncols} of the "
                            f"{NCOLS} columns ({wall:.1f} s wall over {cores} processes)",
                  "failed_columns": bad}


def make_pool(cores):
    import multiprocessing as mp
    if cores <= 1:
        return None
    return mp.get_context("spawn").Pool(cores)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None

    def __enter__(self):
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if self.uuid:
                cmd += ["-i", self.uuid]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        import statistics
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except Exception:
                continue
            for nm, val in zip(names, f[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_steps(ctx, tab, qa, qb, H, k):
    for _ in range(k):
        ctx.hevi_lhevi_step(tab, DT, qa, H, qb)
        qa, qb = qb, qa
    return qa, qb


def gpu_arm(args, rank, world, local_rank, pool, cores):
    import numpy as np
    import torch
    import hevi_inputs
    import paper_2311_11425_gb300 as hv

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    from paper_2311_11425_gb300.shard import shard_of
    hv.load(build=True)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    # weak scaling: a global grid of world x 86,402 columns, one contiguous
    # shard per rank (each shard a seeded copy of the cubed-sphere workload)
    start, stop = shard_of(world * NCOLS, rank, world)
    assert stop - start == NCOLS
    inp = hevi_inputs.lhevi_ark3(seed=2 + start // NCOLS)
    H = torch.from_numpy(inp["H"].reshape(-1)).to(dev)
    tab = hv.tableau("ARK3")

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    def max_over_ranks(x):
        if not dist:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    results = {}
    for prec in (["FP32_IR", "FP64"] if not args.no_fp64 else ["FP32_IR"]):
        ctx = hv.Context([(NEZ, ORDER)], ZTOP, ncols=NCOLS, precision=getattr(hv, prec),
                         stream=stream)
        qa = ctx.hevi_reference_state()
        qb = torch.empty_like(qa)
        qa, qb = run_steps(ctx, tab, qa, qb, H, args.warmup)
        ctx.hevi_sync()
        steps = args.steps if prec == "FP32_IR" else max(3, args.steps // 3)
        barrier()
        ctx.hevi_profile(True)
        l0 = ctx.launch_count
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        uuid = None
        try:
            uuid = str(torch.cuda.get_device_properties(local_rank).uuid)
            uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
        except Exception:
            pass
        with ClockSampler(uuid) as clk:
            e0.record(stream)
            qa, qb = run_steps(ctx, tab, qa, qb, H, steps)
            e1.record(stream)
            barrier()
        ms = e0.elapsed_time(e1)
        launches = ctx.launch_count - l0
        kern = ctx.hevi_profile_read()
        ctx.hevi_profile(False)
        st = ctx.hevi_sync()
        _, iters = ctx.hevi_column_status()
        ms = max_over_ranks(ms)
        results[prec] = dict(ms_per_step=ms / steps, steps=steps, launches=launches, kernels=kern,
                             clocks=clk.summary(), ir_sweeps_last=float(iters.float().mean()),
                             state_finite=bool(torch.isfinite(qa).all()))
        if prec == "FP32_IR":
            # the same steps with the Jacobian refactored every 5 steps (the
            # paper's default update interval, Sec. 4.3)
            barrier()
            e0.record(stream)
            for k in range(steps):
                ctx.hevi_lhevi_step(tab, DT, qa, H, qb, refactor=(k % 5 == 0))
                qa, qb = qb, qa
            e1.record(stream)
            barrier()
            results["update5"] = dict(ms_per_step=max_over_ranks(e0.elapsed_time(e1)) / steps)
            # end to end through the C ABI with host buffers: H2D of q^n and H
            # from pinned memory, the step, D2H of q^{n+1}, every step
            hq = qa.cpu().pin_memory()
            hH = H.cpu().pin_memory()
            hout = torch.empty_like(hq).pin_memory()
            dq, dH = torch.empty_like(qa), torch.empty_like(H)
            barrier()
            e0.record(stream)
            for _ in range(steps):
                dq.copy_(hq, non_blocking=True)
                dH.copy_(hH, non_blocking=True)
                ctx.hevi_lhevi_step(tab, DT, dq, dH, qb)
                hout.copy_(qb, non_blocking=True)
            e1.record(stream)
            barrier()
            e2e_ms = max_over_ranks(e0.elapsed_time(e1))
            results["e2e"] = dict(ms_per_step=e2e_ms / steps,
                                  h2d=(hq.numel() + hH.numel()) * 8, d2h=hout.numel() * 8)
        ctx.close()
        del ctx
        torch.cuda.empty_cache()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    r = results["FP32_IR"]
    value = world * STAGES * NCOLS / (r["ms_per_step"] * 1e-3)
    # dominant kernel and its roofline
    per = {k: list(v) for k, v in r["kernels"].items() if v[1] > 0}
    dom = max(per, key=lambda k: per[k][0])
    pk = peaks()
    avg_ms = per[dom][0] / per[dom][1]
    if dom == "stage_solve":
        ach = BYTES_SOLVE_FP32IR * NCOLS / (avg_ms * 1e-3) / 1e9
        tr = [ncu_traffic("k_solve_ir"), ncu_traffic("k_solve_tail")]
        roof = {"kernel": "k_solve_ir + k_solve_tail (stage_solve)", "bound": "hbm", "achieved": ach,
                "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": ach / pk["hbm_gbs"],
                "traffic": None if None in tr else sum(tr), "peak_source": pk["source"],
                "algorithmic_bytes_per_launch": BYTES_SOLVE_FP32IR * NCOLS}
    elif dom == "factor":
        ach = factor_flops() * NCOLS / (avg_ms * 1e-3) / 1e12
        roof = {"kernel": "k_factor_r (factor)", "bound": "alu", "achieved": ach,
                "peak": pk["fp32_tflops"], "unit": "TFLOP/s", "frac": ach / pk["fp32_tflops"],
                "traffic": ncu_traffic("k_factor_r"), "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 x 2.07 GHz",
                "algorithmic_flops_per_launch": factor_flops() * NCOLS}
    else:
        roof = {"kernel": dom, "bound": "alu", "achieved": None, "peak": None, "unit": None,
                "frac": None, "traffic": None}
    roof["avg_launch_ms"] = avg_ms
    line = {
        "metric": "columns solved/s (LHEVI ARK3 implicit stage solves, FP32 LU + FP64 refinement, "
                  "1e-10 rel vs FP64 oracle)",
        "value": value,
        "unit": "column-solves/s",
        "n_gpus": world,
        "steps": r["steps"],
        "warmup": args.warmup,
        "ms_per_step": r["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "columns_per_gpu": NCOLS, "nez": NEZ, "order": ORDER,
                   "unknowns_per_column": NUNK, "implicit_stages": STAGES,
                   "precision": "FP32 LU + FP64 refinement",
                   "l2": "working set > L2 (factors 1.9 GB per step); no flush",
                   "parallelism": f"{world} independent column shards, no collective"},
        "e2e": None,
        "gpu_launches": r["launches"],
        "clocks": r["clocks"],
        "roofline": roof,
        "kernels": {k: {"total_ms": v[0], "launches": v[1], "avg_ms": v[0] / v[1]}
                    for k, v in r["kernels"].items() if v[1] > 0},
        "ir_sweeps_mean": r["ir_sweeps_last"],
        "state_finite": r["state_finite"],
    }
    if "e2e" in results:
        e = results["e2e"]
        line["e2e"] = {"value": world * STAGES * NCOLS / (e["ms_per_step"] * 1e-3),
                       "unit": "column-solves/s", "h2d_bytes_per_step": e["h2d"],
                       "d2h_bytes_per_step": e["d2h"], "ms_per_step": e["ms_per_step"]}
    if "update5" in results:
        u = results["update5"]
        line["update_every_5_steps"] = {
            "value": world * STAGES * NCOLS / (u["ms_per_step"] * 1e-3), "unit": "column-solves/s",
            "ms_per_step": u["ms_per_step"],
            "note": "Jacobian refactored every 5 steps (LHEVI with an update interval)"}
    if "FP64" in results:
        f = results["FP64"]
        line["fp64_plain"] = {"value": world * STAGES * NCOLS / (f["ms_per_step"] * 1e-3),
                              "unit": "column-solves/s", "ms_per_step": f["ms_per_step"],
                              "kernels": {k: v[0] / max(1, v[1]) for k, v in f["kernels"].items()
                                          if v[1]}}
    if world == 1 and not args.no_extra:
        line["batched"] = batched_run(args)
        line["nhevi_gmres_vs_lu"] = gmres_run(args)
        line["serving"] = serving_run(args)
    if world == 1 and not args.no_cpu:
        rate, cb = cpu_oracle_rate(pool, cores)
        line["cpu_baseline"] = cb
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# secondary workloads (reported inside the main line, rank 0, one GPU)
# ---------------------------------------------------------------------------

def batched_run(args):
    """Uneven columns: 200,000 columns of four size classes with tops uniform
    in 30-100 km, LHEVI-PS ARK4 steps replayed from a captured graph (two
    steps per replay) and, for comparison, the same steps called one by one."""
    import torch
    import hevi_inputs
    import paper_2311_11425_gb300 as hv
    inp = hevi_inputs.batched(seed=4)
    classes = hevi_inputs.SIZE_CLASSES
    ctx = hv.Context(classes, inp["ztop"], class_of_col=inp["class_of_col"],
                     precision=hv.FP32_IR)
    off = ctx.offsets()
    import numpy as np
    H = np.zeros(ctx.n)
    for blk in inp["blocks"]:
        n = 3 * (blk["nez"] * blk["N"] + 1)
        H[(off[blk["cols"]][:, None] + np.arange(n)[None, :]).reshape(-1)] = blk["H"].reshape(-1)
    H = torch.from_numpy(H).cuda()
    tab = hv.tableau("ARK4")
    stream = torch.cuda.current_stream()
    qa = ctx.hevi_reference_state()
    qb = torch.empty_like(qa)
    g = ctx.hevi_lhevi_graph(tab, inp["dt"], qa, qb, H, nsteps=2)
    reps = max(2, min(10, args.steps // 5))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(2):
        g.launch()
    torch.cuda.synchronize()
    l0 = ctx.launch_count
    e0.record(stream)
    for _ in range(reps):
        g.launch()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_graph = e0.elapsed_time(e1) / (2 * reps)
    launches = (ctx.launch_count - l0) / (2 * reps)
    e0.record(stream)
    for _ in range(reps):
        ctx.hevi_lhevi_step(tab, inp["dt"], qa, H, qb)
        ctx.hevi_lhevi_step(tab, inp["dt"], qb, H, qa)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_calls = e0.elapsed_time(e1) / (2 * reps)
    try:
        ctx.hevi_sync()
        st = "ok"
    except hv.HeviError as e:
        st = str(e)
    finite = bool(torch.isfinite(qa).all())
    g.close()
    ctx.close()
    torch.cuda.empty_cache()
    implicit = tab.s - 1
    return {"workload": f"batched: {inp['ncols']} columns, classes {list(classes)} uniform, "
                        f"ztop U(30, 100) km, LHEVI-PS ARK4 ({implicit} implicit stages), "
                        f"dt={inp['dt']} s, graph of 2 steps per replay",
            "value": implicit * inp["ncols"] / (ms_graph * 1e-3), "unit": "column-solves/s",
            "ms_per_step_graph": ms_graph, "ms_per_step_calls": ms_calls,
            "kernel_launches_per_step": launches, "steps_timed": 2 * reps,
            "status": st, "state_finite": finite}


def gmres_run(args):
    """NHEVI column solves of the NHEVI workload's class ((16, 3), 30 km, the
    rest state plus the seeded increment, Lambda = gamma dt of ARK2 at 300 s) on
    8,192 columns: Newton-LU against JFNK-GMRES at the paper's settings
    (eps 0.05, Newton 1e-5, GMRES 1e-9), same Newton tolerance."""
    import torch
    import hevi_inputs
    import paper_2311_11425_gb300 as hv
    ncols = 8192
    inp = hevi_inputs.nhevi_ark2(seed=3, ncols=ncols)
    ctx = hv.Context([(inp["nez"], inp["N"])], inp["ztop"], precision=hv.FP32_IR)
    q0 = ctx.hevi_reference_state() + torch.from_numpy(inp["dq"].reshape(-1)).cuda()
    lam = hv.tableau("ARK2").gamma * inp["dt"]
    R = q0.clone()
    kry = torch.zeros(ncols, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    for name, solve in (("lu", lambda q: ctx.hevi_newton_solve(lam, q, R, rtol=1e-5)),
                        ("gmres", lambda q: ctx.hevi_newton_gmres_solve(lam, q, R, krylov=kry))):
        q = q0.clone()
        solve(q)  # warm-up (allocates the GMRES scratch)
        reps = 3
        ms = 0.0
        for _ in range(reps):
            q.copy_(q0)
            torch.cuda.synchronize()
            e0.record(stream)
            solve(q)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1) / reps
        _, it = ctx.hevi_column_status()
        out[name] = {"ms": ms, "column_solves_per_s": ncols / (ms * 1e-3),
                     "newton_iters_mean": float(it.float().mean())}
    out["gmres"]["krylov_iters_mean"] = float(kry.float().mean())
    ctx.close()
    torch.cuda.empty_cache()
    return {"workload": f"NHEVI column solves: {ncols} columns of (16, 3), 30 km, "
                        "Lambda = gamma dt (ARK2, 300 s), Newton tolerance 1e-5; GMRES with "
                        "eps 0.05, GMRES tolerance 1e-9, FP64 Krylov",
            "lu": out["lu"], "gmres": out["gmres"],
            "gmres_over_lu_time": out["gmres"]["ms"] / out["lu"]["ms"]}


def serving_run(args):
    """Poisson arrivals at 50/s; per request U{2000..86402} columns of the four
    classes, U{1..20} ARK3 steps, LHEVI or NHEVI-LU with probability 1/2;
    150 GB device budget; latency from arrival to completion."""
    import torch
    import hevi_inputs
    from paper_2311_11425_gb300.serve import Request, Server, latency_stats
    raw = hevi_inputs.serve_requests(seed=5, count=args.serve_requests, rate=50.0)
    reqs = [Request(**r) for r in raw]
    server = Server(hbm_budget=150 * 10**9, tab="ARK3")
    res = server.run(reqs, realtime=True)
    torch.cuda.empty_cache()
    out = {"workload": f"serving: {len(reqs)} requests, Poisson 50/s, columns U(2000, 86402) of "
                       f"4 classes, steps U(1, 20), LHEVI-PS or NHEVI-LU ARK3, budget 150 GB",
           "peak_bytes": server.peak_bytes}
    out.update(latency_stats(res))
    errs = [r.error for r in res if r.error]
    if errs:
        out["errors"] = errs[:3]
    return out


# ---------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle on the host cores
# ---------------------------------------------------------------------------

def reference_arm(args, rank, world, pool, cores):
    if rank != 0:
        return
    rates = []
    for _ in range(args.warmup if args.warmup < 1 else 1):
        cpu_oracle_rate(pool, cores, target_s=2.0)
    samples = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        rate, cb = cpu_oracle_rate(pool, cores, target_s=6.0)
        rates.append(rate)
        samples.append(cb["sample"])
    wall = time.perf_counter() - t0
    import statistics
    value = statistics.median(rates)
    line = {"impl": "reference",
            "metric": "columns solved/s (LHEVI ARK3 implicit stage solves, FP32 LU + FP64 "
                      "refinement, 1e-10 rel vs FP64 oracle)",
            "value": value, "unit": "column-solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": STAGES * NCOLS / value * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": value, "unit": "column-solves/s", "cores": cores,
                             "kind": "oracle", "sample": samples[-1]},
            "e2e": {"value": value, "unit": "column-solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line), flush=True)


def ncu_case(args):
    """A short run of one operation on the benchmark workload for targeted
    ncu captures: setup, one warm-up step, then `--ncu-reps` launches of the
    chosen operation (factor, solve, apply, newton or step)."""
    import torch
    import hevi_inputs
    import paper_2311_11425_gb300 as hv
    hv.load(build=True)
    case = args.ncu_case
    prec = hv.FP64 if args.ncu_fp64 else hv.FP32_IR
    if case == "newton":
        inp = hevi_inputs.nhevi_ark2(seed=3)
        ctx = hv.Context([(inp["nez"], inp["N"])], inp["ztop"], precision=prec)
        q0 = ctx.hevi_reference_state() + torch.from_numpy(inp["dq"].reshape(-1)).cuda()
        for _ in range(args.ncu_reps):
            q = q0.clone()
            ctx.hevi_newton_solve(87.868, q, q0, blocking=False)
        ctx.hevi_sync()
        return
    inp = hevi_inputs.lhevi_ark3(seed=2)
    ctx = hv.Context([(NEZ, ORDER)], ZTOP, ncols=NCOLS, precision=prec)
    tab = hv.tableau("ARK3")
    H = torch.from_numpy(inp["H"].reshape(-1)).cuda()
    qa = ctx.hevi_reference_state()
    qb = torch.empty_like(qa)
    ctx.hevi_lhevi_step(tab, DT, qa, H, qb)
    lam = tab.gamma * DT
    for _ in range(args.ncu_reps):
        if case == "factor":
            ctx.hevi_factor(lam, qb)
        elif case == "solve":
            ctx.hevi_stage_solve(H, qa, blocking=False)
        elif case == "apply":
            ctx.hevi_apply_Lv(qb, qa, nonlinear=True)
        elif case == "step":
            ctx.hevi_lhevi_step(tab, DT, qb, H, qa)
    ctx.hevi_sync()


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the batched-columns and serving sub-measurements")
    ap.add_argument("--serve-requests", type=int, default=24)
    ap.add_argument("--ncu-case", choices=["factor", "solve", "apply", "newton", "step"],
                    help="run only a few launches of one operation (for ncu captures)")
    ap.add_argument("--ncu-reps", type=int, default=2)
    ap.add_argument("--ncu-fp64", action="store_true")
    args = ap.parse_args()
    if args.ncu_case:
        ncu_case(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    cores = os.cpu_count() or 1
    # the oracle's process pool starts (spawn) before any GPU call
    pool = make_pool(cores) if rank == 0 and (args.impl == "reference" or
                                              (world == 1 and not args.no_cpu)) else None
    try:
        if args.impl == "reference":
            reference_arm(args, rank, world, pool, cores)
        else:
            gpu_arm(args, rank, world, local_rank, pool, cores)
    finally:
        if pool:
            pool.close()
            pool.join()


if __name__ == "__main__":
    main()
