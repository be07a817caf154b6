#!/usr/bin/env python
"""Benchmark of the HEVI vertical column solve on GB300.

Workload (one "step"): one LHEVI ARK3 time step (Sec. 4.3, Sec. 6) on
86,402 columns of Nez = 10 elements of order N = 4 (41 points, 123 unknowns)
with a 30 km top and dt = 300 s: one band factorisation linearised about q^n
(FP32, no interchanges, of the equilibrated band), three implicit stage
solves refined with a double-float (about 48-bit) residual, the vertical
operator applies and the stage combinations, advancing the state in place
from rest under a seeded horizontal tendency.  Metric: implicit column stage
solves per second (3 x columns per step), whole job.

Also reported: the same step with plain FP64 factors (partial pivoting, one
column per thread), an end-to-end number through the C ABI with host
buffers, per-kernel times from CUDA events on the library's stream, the
dominant kernel's roofline against measured peaks (HBM copy from the
driver's measurement; FP32 and FP64 from cuBLAS SGEMM / DGEMM timed here), SM
clocks during the timed region, the 1,538-column single-stage latency, the
NHEVI-LU step on 86,402 columns of (16, 3), the batched and serving
workloads, and the FP64 CPU oracle timed on the host cores (all cores and
one core) on bounded samples of the same workload.

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
METRIC = ("columns solved/s (LHEVI ARK3 implicit stage solves; FP32 no-pivot LU of the "
          "equilibrated band + double-float (~48-bit) refinement residual; 1e-10 rel vs FP64 "
          "oracle)")
WORKLOAD = (f"lhevi_ark3: {NCOLS} columns, Nez={NEZ}, N={ORDER}, ztop=30 km, dt=300 s, "
            f"ARK3 (3 implicit stages), LHEVI-PS, seeded horizontal tendency")

# Algorithmic bytes of one column stage solve.  FP32 path: the no-pivot
# factors ((2K + 1) n floats: K multipliers, 1/u_jj and K entries of U per
# step, counted once) and b, x and the linearisation state q0 (3 n 8); FP64
# plain: FP64 factors of partial pivoting (ldab n 8), int pivots, b, x.
BYTES_SOLVE_FP32IR = (2 * K_BAND + 1) * NUNK * 4 + 3 * NUNK * 8
BYTES_SOLVE_FP64 = LDAB * NUNK * 8 + NUNK * 4 + 2 * NUNK * 8


def factor_flops(n=NUNK, k=K_BAND):
    """FP32 flops of one band LU without interchanges (K sub- and K
    super-diagonals): per step nr multipliers and an nr x nc rank-1 update."""
    f = 0
    for j in range(n):
        nr = min(k, n - 1 - j)
        nc = min(k, n - 1 - j)
        f += nr + 2 * nr * nc
    return f


# DRAM bytes (read + write) per launch of the dominant kernels from one ncu
# capture of `python bench.py --ncu-case solve|factor` (the summaries under
# profiles/ give the commands), valid only for the kernel source they were
# taken from: the SHA-256 of the kernel file at capture time.
_NP_SHA = "6e02d2a6011daa9e3cee6e90874fa8398b053bfdaa0e6187b0396706b5ed38b6"
NCU_TRAFFIC = {
    "k_solve_np": {"bytes": 3.792e9, "sha256": _NP_SHA},      # 5.212 TB/s x 0.728 ms
    "k_factor_np": {"bytes": 1.833e9, "sha256": _NP_SHA},     # 1.731 TB/s x 1.059 ms
    # k_apply_rhs_df: its passes differ (the stage combinations fold in a
    # different number of vectors); the capture covers the first pass only,
    # so no per-launch average is recorded
}
KERNEL_SOURCE = os.path.join(ROOT, "paper_2311_11425_gb300", "csrc", "hevi_np.cu")


def apply_bytes_fused(s):
    """Algorithmic bytes per column of one tendency pass of an s-stage LHEVI
    step with the stage combinations folded in, averaged over the s passes.
    Every pass reads H, the reference (rho_bar, P_bar, Theta_bar: one vector)
    and 1/Theta_bar (one double per point).  Pass 0 reads q^n and writes S_0
    and the next right-hand side; pass i (0 < i < s-1) reads q_tt, the i
    earlier Q_j and S_j and q^n and writes Q_i, S_i and the next right-hand
    side; the last pass reads q_tt, the Q_j and S_j before it and q^n and
    writes q^{n+1}.  Vectors of NUNK doubles."""
    vecs = 2 + 3                                    # pass 0: H, ref; q^n, S_0, rhs
    vecs += sum(2 + 5 + 2 * i for i in range(1, s - 1))
    vecs += 2 + 3 + 2 * (s - 1)
    return (vecs / s * NUNK + NZ) * 8


def ncu_traffic(kernel):
    import hashlib
    rec = NCU_TRAFFIC.get(kernel)
    if not rec:
        return None
    with open(KERNEL_SOURCE, "rb") as fh:
        digest = hashlib.sha256(fh.read()).hexdigest()
    return rec["bytes"] if digest == rec["sha256"] else None


_ALU = {}


def alu_peaks():
    """FP32 and FP64 throughput measured on this GPU: cuBLAS SGEMM (TF32 off,
    so on the FP32 pipes) and DGEMM, best of 5 (2 n^3 flops each)."""
    if _ALU:
        return _ALU
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for name, dt, n in (("fp32_tflops", torch.float32, 8192), ("fp64_tflops", torch.float64, 4096)):
            a = torch.randn(n, n, device="cuda", dtype=dt)
            b = torch.randn(n, n, device="cuda", dtype=dt)
            for _ in range(2):
                a @ b
            torch.cuda.synchronize()
            best = None
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                a @ b
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
            _ALU[name] = 2 * n ** 3 / (best * 1e-3) / 1e12
            del a, b
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
        torch.cuda.empty_cache()
    _ALU["method"] = "cuBLAS SGEMM 8192^3 (TF32 off) and DGEMM 4096^3, best of 5, CUDA events"
    return _ALU


def peaks():
    p = {"hbm_gbs": 6777.0, "source": "fallback"}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            m = json.load(fh)
        p["hbm_gbs"] = float(m["hbm_gbs"])
        p["source"] = "measured"
    except Exception:
        pass
    p.update(alu_peaks())
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


def _oracle_warm(_):
    import oracle
    oracle.build()
    q, H, zt = oracle_sample_inputs(2)
    _oracle_chunk((q, H, zt))
    return 0


def cpu_oracle_rate(pool, cores, target_s=12.0):
    """Time the oracle's LHEVI ARK3 step on a bounded sample of the workload's
    columns, spread over `cores` worker processes (each worker has imported and
    run the oracle once before the timed region).  Returns (col-solves/s, dict)."""
    import numpy as np
    if pool:
        pool.map(_oracle_warm, range(cores))
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
            # end to end through the C ABI with host buffers: every step copies
            # its q^n and H from pinned memory and reads q^{n+1} back.  The
            # copies run on their own streams, double-buffered, so that step
            # k+1's inputs arrive and step k-1's result leaves while step k
            # computes (the copy engines work beside the kernels)
            hq = qa.cpu().pin_memory()
            hH = H.cpu().pin_memory()
            hout = [torch.empty_like(hq).pin_memory() for _ in range(2)]
            dq = [torch.empty_like(qa) for _ in range(2)]
            dH = [torch.empty_like(H) for _ in range(2)]
            dout = [torch.empty_like(qa) for _ in range(2)]
            s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
            ev_in = [torch.cuda.Event() for _ in range(2)]
            ev_used = [torch.cuda.Event() for _ in range(2)]
            ev_done = [torch.cuda.Event() for _ in range(2)]
            ev_out = [torch.cuda.Event() for _ in range(2)]
            barrier()
            e0.record(stream)
            s_in.wait_stream(stream)
            s_out.wait_stream(stream)

            def upload(k):
                b = k % 2
                with torch.cuda.stream(s_in):
                    if k >= 2:
                        s_in.wait_event(ev_used[b])  # step k-2 has read these buffers
                    dq[b].copy_(hq, non_blocking=True)
                    dH[b].copy_(hH, non_blocking=True)
                    ev_in[b].record(s_in)

            upload(0)
            for k in range(steps):
                b = k % 2
                if k + 1 < steps:
                    upload(k + 1)
                stream.wait_event(ev_in[b])
                if k >= 2:
                    stream.wait_event(ev_out[b])  # step k-2's result has left dout[b]
                ctx.hevi_lhevi_step(tab, DT, dq[b], dH[b], dout[b])
                ev_used[b].record(stream)
                ev_done[b].record(stream)
                with torch.cuda.stream(s_out):
                    s_out.wait_event(ev_done[b])
                    hout[b].copy_(dout[b], non_blocking=True)
                    ev_out[b].record(s_out)
            stream.wait_stream(s_in)
            stream.wait_stream(s_out)
            e1.record(stream)
            barrier()
            e2e_ms = max_over_ranks(e0.elapsed_time(e1))
            results["e2e"] = dict(ms_per_step=e2e_ms / steps,
                                  h2d=(hq.numel() + hH.numel()) * 8, d2h=hout[0].numel() * 8)
        ctx.close()
        del ctx
        torch.cuda.empty_cache()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    r = results["FP32_IR"]
    value = world * STAGES * NCOLS / (r["ms_per_step"] * 1e-3)
    # dominant kernel and its roofline; the other main kernels beside it
    per = {k: list(v) for k, v in r["kernels"].items() if v[1] > 0}
    dom = max(per, key=lambda k: per[k][0])
    pk = peaks()

    def roofline(kind):
        avg = per[kind][0] / per[kind][1]
        if kind == "stage_solve":
            ach = BYTES_SOLVE_FP32IR * NCOLS / (avg * 1e-3) / 1e9
            return {"kernel": "k_solve_np<4> (stage_solve)", "bound": "hbm", "achieved": ach,
                    "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": ach / pk["hbm_gbs"],
                    "traffic": ncu_traffic("k_solve_np"), "peak_source": pk["source"],
                    "algorithmic_bytes_per_launch": BYTES_SOLVE_FP32IR * NCOLS, "avg_launch_ms": avg}
        if kind == "factor":
            ach = factor_flops() * NCOLS / (avg * 1e-3) / 1e12
            return {"kernel": "k_factor_np<4> (factor)", "bound": "alu", "achieved": ach,
                    "peak": pk["fp32_tflops"], "unit": "TFLOP/s", "frac": ach / pk["fp32_tflops"],
                    "traffic": ncu_traffic("k_factor_np"),
                    "peak_source": "measured (cuBLAS SGEMM, TF32 off)",
                    "algorithmic_flops_per_launch": factor_flops() * NCOLS, "avg_launch_ms": avg}
        if kind == "apply":
            b = apply_bytes_fused(STAGES + 1) * NCOLS
            ach = b / (avg * 1e-3) / 1e9
            return {"kernel": "k_apply_rhs_df<4> (tendency pass with the stage combinations)",
                    "bound": "hbm",
                    "achieved": ach,
                    "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": ach / pk["hbm_gbs"],
                    "traffic": ncu_traffic("k_apply_rhs_df"), "peak_source": pk["source"],
                    "algorithmic_bytes_per_launch": b, "avg_launch_ms": avg}
        return {"kernel": kind, "bound": None, "achieved": None, "peak": None, "unit": None,
                "frac": None, "traffic": None, "avg_launch_ms": avg}

    roof = roofline(dom)
    others = {k: roofline(k) for k in ("stage_solve", "factor", "apply") if k in per and k != dom}
    avg_ms = per[dom][0] / per[dom][1]
    roof["avg_launch_ms"] = avg_ms
    line = {
        "metric": METRIC,
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
                   "precision": "FP32 LU without interchanges of S^-1 A S (S: reference scales); "
                                "refinement residual b - A x in double-float arithmetic (~48 bits) "
                                "on the FP32 pipes; explicit tendency S = H + V(Q) in double-float "
                                "arithmetic rounded to FP64; FP64 reference state, state vectors, "
                                "stage combinations and output",
                   "l2": "working set > L2 (factors 1.36 GB per step); no flush",
                   "parallelism": f"{world} independent column shards, no collective"},
        "e2e": None,
        "gpu_launches": r["launches"],
        "clocks": r["clocks"],
        "roofline": roof,
        "rooflines_other": others,
        "peaks": {k: v for k, v in pk.items()},
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
        line["stage_latency_1538"] = stage_latency(args)
        line["nhevi_lu"] = nhevi_lu_run(args)
        line["equation_sets"] = equation_sets_run(args)
        line["batched"] = batched_run(args)
        line["nhevi_gmres_vs_lu"] = gmres_run(args)
        line["serving"] = serving_run(args)
    if world == 1 and not args.no_cpu:
        rate, cb = cpu_oracle_rate(pool, cores)
        rate1, cb1 = cpu_oracle_rate(None, 1, target_s=6.0)
        cb["one_core"] = {"value": rate1, "cores": 1, "sample": cb1["sample"]}
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
    # launch shape of the single-launch stage solve, chosen by timing before
    # the graph is captured (a captured launch keeps its shape)
    ctx.hevi_factor(tab.gamma * inp["dt"], qa)
    tune_w, tune_ms, tune_default_ms = ctx.hevi_autotune_solve(qa, qb, reps=3)
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
    ctx.hevi_profile(True)
    ctx.hevi_lhevi_step(tab, inp["dt"], qa, H, qb)
    ctx.hevi_lhevi_step(tab, inp["dt"], qb, H, qa)
    prof = ctx.hevi_profile_read()
    ctx.hevi_profile(False)
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
            "stage_solve": "one persistent launch over the tiles of both orders, "
                           "costliest tiles first",
            "autotune": {"solve_warps_per_sm": tune_w, "solve_ms": tune_ms,
                         "solve_ms_default_shape": tune_default_ms},
            "kernel_ms_per_step": {k: v[0] / 2 for k, v in prof.items() if v[1]},
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
    """Config 5: a Poisson stream at 50 requests/s of `--serve-requests`
    requests (2,000 by default: the stream's stated length); per request
    U{2000..86402} columns of the four classes, U{1..20} ARK3 steps, LHEVI-PS
    or NHEVI-LU with probability 1/2, served by continuous batching from one
    resident slot pool per variant inside a 150 GB device budget.  Admission
    stops after `--serve-seconds` of wall time; the requests admitted by then
    are finished and the rest reported as not admitted.  Latency runs from
    arrival to the host's receipt of the result."""
    import torch
    import numpy as np
    import hevi_inputs
    from paper_2311_11425_gb300.serve import Block, Request, Server, latency_stats
    classes = hevi_inputs.SIZE_CLASSES
    bank_cols = 32768
    bank = hevi_inputs.serve_bank(seed=6, cols_per_class=bank_cols)
    Hb = [torch.from_numpy(b["H"].reshape(-1)).pin_memory() for b in bank]
    dqb = [torch.from_numpy(b["dq"].reshape(-1)).pin_memory() for b in bank]
    raw = hevi_inputs.serve_stream(seed=5, count=args.serve_requests, rate=50.0,
                                   bank_cols=bank_cols)
    reqs = []
    for r in raw:
        blocks = []
        for c, s0, m in r["parts"]:
            nez, N = classes[c]
            n = 3 * (nez * N + 1)
            blocks.append(Block((nez, N), bank[c]["ztop"][s0:s0 + m], Hb[c][s0 * n:(s0 + m) * n],
                                dqb[c][s0 * n:(s0 + m) * n] if r["variant"] == "NHEVI" else None))
        reqs.append(Request(rid=r["rid"], steps=r["steps"], variant=r["variant"],
                            arrival=r["arrival"], blocks=blocks))
    server = Server(classes, slots_per_class=args.serve_slots, hbm_budget=150 * 10**9,
                    tab="ARK3", keep_state=False)
    res = server.run(reqs, realtime=True, time_limit=args.serve_seconds)
    stats = server.stats
    server.close()
    del Hb, dqb
    torch.cuda.empty_cache()
    span = max(r.arrival for r in reqs) if reqs else 0.0
    offered = sum(r.ncols * r.steps for r in reqs) / span if span > 0 else None
    out = {"workload": f"serving: {len(reqs)} requests, Poisson 50/s (arrivals over {span:.1f} s), "
                       "columns U(2000, 86402) of 4 classes, steps U(1, 20), LHEVI-PS or "
                       "NHEVI-LU ARK3 (1/2 each), budget 150 GB; NHEVI requests start from rest "
                       "plus the 1 K / 1 m/s increment scaled by 0.1",
           "batching": f"continuous: one resident slot pool per variant, "
                       f"{args.serve_slots} slots per class, no device allocation on admission",
           "admission_limit_s": args.serve_seconds,
           "offered_column_steps_per_s": offered}
    out.update(latency_stats(res))
    out["gpu_busy_fraction"] = stats["gpu_busy_fraction"]
    out["pools"] = stats["variants"]
    out["pool_bytes"] = sum(stats["pool_bytes"].values())
    errs = [r.error for r in res if r.error and not r.error.startswith("not admitted")]
    out["failed"] = len(errs)
    if errs:
        out["errors"] = errs[:3]
    return out


def stage_latency(args):
    """Latency of one LHEVI ARK2 stage solve on the 1,538 columns of (8, 4),
    30 km (the cubed-sphere Ne = 4 point count), FP64 and FP32 + refinement,
    factors about the rest state: per call, CUDA events around the launch
    (device time) and host wall time of the blocking call (launch + wait);
    p50 / p99 over repeats.  This workload is launch-bound."""
    import numpy as np
    import torch
    import hevi_inputs
    import paper_2311_11425_gb300 as hv
    inp = hevi_inputs.lhevi_stage(seed=1)
    out = {"workload": f"stage solve: {inp['ncols']} columns, Nez={inp['nez']}, N={inp['N']}, "
                       f"30 km, Lambda = (1 - 1/sqrt 2) 300 s, one ARK2 stage",
           "unit": "us"}
    stream = torch.cuda.current_stream()
    for prec in ("FP64", "FP32_IR"):
        ctx = hv.Context([(inp["nez"], inp["N"])], inp["ztop"], precision=getattr(hv, prec),
                         stream=stream)
        ctx.hevi_factor(inp["lam"], None)
        b = torch.from_numpy(inp["b"].reshape(-1)).cuda()
        x = ctx.empty()
        for _ in range(10):
            ctx.hevi_stage_solve(b, x)
        dev, wall, fwall = [], [], []
        for _ in range(200):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e0.record(stream)
            ctx.hevi_stage_solve(b, x)  # blocking: launch, wait, status
            e1.record(stream)
            t1 = time.perf_counter()
            torch.cuda.synchronize()
            dev.append(e0.elapsed_time(e1) * 1e3)
            wall.append((t1 - t0) * 1e6)
        for _ in range(50):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.hevi_factor(inp["lam"], None)
            ctx.hevi_stage_solve(b, x)
            fwall.append((time.perf_counter() - t0) * 1e6)
        out[prec] = {"solve_device_p50_us": float(np.percentile(dev, 50)),
                     "solve_device_p99_us": float(np.percentile(dev, 99)),
                     "solve_wall_p50_us": float(np.percentile(wall, 50)),
                     "solve_wall_p99_us": float(np.percentile(wall, 99)),
                     "factor_and_solve_wall_p50_us": float(np.percentile(fwall, 50))}
        ctx.close()
    torch.cuda.empty_cache()
    return out


def equation_sets_run(args, steps=10, warmup=3):
    """The headline step (LHEVI-PS ARK3, 86,402 columns of (10, 4), 30 km,
    dt = 300 s) in equation sets 3C (rho, m, E) and 2NC (rho, w, theta), from
    each set's rest state plus the increment of ``hevi_inputs.state_increment``
    written in that set's unknowns (w' and a 1 K Gaussian: m' = rho' w', E' =
    cv rho' T' in set 3C; w' and theta' themselves in set 2NC), H = 0.  Set 3C
    on both precisions, set 2NC on the FP64 path (the one it has)."""
    import numpy as np
    import torch
    import hevi_inputs
    import paper_2311_11425_gb300 as hv
    cv = 1004.67 - 287.17
    g = hevi_inputs.rng(7)
    zt = np.full(NCOLS, 30e3)
    dq = hevi_inputs.state_increment(g, NEZ, ORDER, zt).reshape(NCOLS, -1, 3)
    amp = hevi_inputs.density_like(np.arange(NZ) / (NZ - 1), zt)
    tab = hv.tableau("ARK3")
    out = {}
    for name, eq, prec in (("3C_FP32_IR", hv.SET_3C, hv.FP32_IR), ("3C_FP64", hv.SET_3C, hv.FP64),
                           ("2NC_FP64", hv.SET_2NC, hv.FP64)):
        inc = dq.copy()
        if eq == hv.SET_3C:
            inc[:, :, 2] *= cv  # rho' T' -> cv rho' T'
        else:
            inc[:, :, 1] /= amp  # m' -> w'
            inc[:, :, 2] /= amp  # Theta' -> theta'
        stream = torch.cuda.current_stream()
        ctx = hv.Context([(NEZ, ORDER)], 30e3, ncols=NCOLS, precision=prec, stream=stream)
        ctx.hevi_set_equation_set(eq)
        q0 = ctx.hevi_reference_state() + torch.from_numpy(inc.reshape(-1)).cuda()
        H = torch.zeros_like(q0)
        qa, qb = q0.clone(), torch.empty_like(q0)
        qa, qb = run_steps(ctx, tab, qa, qb, H, warmup)
        ctx.hevi_sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        qa, qb = run_steps(ctx, tab, qa, qb, H, steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        st, it = ctx.hevi_column_status()
        out[name] = {"value": STAGES * NCOLS / (ms * 1e-3), "unit": "column-solves/s",
                     "ms_per_step": ms, "status_ok": bool((st == 0).all()),
                     "state_finite": bool(torch.isfinite(qa).all()),
                     "ir_sweeps_mean": float(it.float().mean()) if prec == hv.FP32_IR else None}
        del ctx, q0, H, qa, qb
        torch.cuda.empty_cache()
    out["workload"] = ("the headline step (LHEVI-PS ARK3, 86402 columns of (10, 4), 30 km, dt = 300 s) "
                       "in sets 3C and 2NC from rest plus the seeded w' and 1 K Gaussian, H = 0")
    return out


def nhevi_lu_run(args):
    """NHEVI-LU (Sec. 4.2.3) on 86,402 columns of (16, 3), 30 km top: one ARK2
    step of dt = 300 s (two implicit stages, each a Newton solve to the
    configuration's rtol = 1e-10) from the rest state plus the seeded 1 K
    theta' Gaussian and +-1 m/s w; H = 0.  Metric: Newton column solves per
    second (2 x columns per step)."""
    import torch
    import hevi_inputs
    import paper_2311_11425_gb300 as hv
    inp = hevi_inputs.nhevi_ark2(seed=3)
    nez, N, ncols = inp["nez"], inp["N"], inp["ncols"]
    stream = torch.cuda.current_stream()
    ctx = hv.Context([(nez, N)], inp["ztop"], precision=hv.FP32_IR, stream=stream)
    q0 = ctx.hevi_reference_state() + torch.from_numpy(inp["dq"].reshape(-1)).cuda()
    H = torch.zeros_like(q0)
    tab = hv.tableau("ARK2")
    qb = torch.empty_like(q0)
    for _ in range(2):
        ctx.hevi_nhevi_step(tab, inp["dt"], q0, H, qb, rtol=1e-10)
    ctx.hevi_sync()
    reps = 3
    ctx.hevi_profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        ctx.hevi_nhevi_step(tab, inp["dt"], q0, H, qb, rtol=1e-10)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    kern = ctx.hevi_profile_read()
    ctx.hevi_profile(False)
    try:
        ctx.hevi_sync()
        st = "ok"
    except hv.HeviError as e:
        st = str(e)
    _, it = ctx.hevi_column_status()
    pk = peaks()
    k = {a: {"total_ms": b[0] / reps, "launches": b[1] / reps} for a, b in kern.items() if b[1]}
    fac = kern.get("factor", (0.0, 0))
    nunk = 3 * (nez * N + 1)
    kb = 3 * (N + 1) - 1
    roof = None
    if fac[1]:
        avg = fac[0] / fac[1]
        fl = factor_flops(nunk, kb) * ncols
        roof = {"kernel": "k_factor_np<3> (factor of J(q_m))", "bound": "alu",
                "achieved": fl / (avg * 1e-3) / 1e12, "peak": pk["fp32_tflops"],
                "unit": "TFLOP/s", "frac": fl / (avg * 1e-3) / 1e12 / pk["fp32_tflops"],
                "peak_source": "measured (cuBLAS SGEMM, TF32 off)",
                "algorithmic_flops_per_launch": fl, "avg_launch_ms": avg}
    del ctx
    torch.cuda.empty_cache()
    return {"workload": f"NHEVI-LU ARK2 step: {ncols} columns, Nez={nez}, N={N}, 30 km, dt=300 s, "
                        "Newton rtol 1e-10 (2 implicit stages)",
            "value": 2 * ncols / (ms * 1e-3), "unit": "column-solves/s", "ms_per_step": ms,
            "newton_iters_last_stage_mean": float(it.float().mean()),
            "newton_iters_last_stage_max": int(it.max()), "status": st,
            "kernels_per_step": k, "roofline": roof}


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
            "metric": METRIC,
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
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="wall-time limit on admission in the serving measurement")
    ap.add_argument("--serve-slots", type=int, default=65536,
                    help="column slots per size class in each serving pool")
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
