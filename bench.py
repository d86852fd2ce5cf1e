"""Benchmark of the matrix-free prism-gravity operator on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload paper_210x210x75] [--precision mixed|fp64]

One step = one forward product d = G m plus one adjoint product G^T r (the
two operator applications of every CG iteration, Section 2.2) on the
paper-scale synthetic workload (210 x 210 x 75 mesh of 100 m cubes = 3,307,500
prisms, 178,797 stations).  The metric is prism-station pairs per second:
2 * N * M pairs per step.  Inputs stay resident; L2 is flushed between timed
steps (a 256 MB write outside the timed events).

Printed as one JSON line (rank 0).  Extra keys: roofline of the dominant
kernel (MUFU-bound, "alu"), e2e (same metric through host buffers), the
oracle timed on the host cores (cpu_baseline), the mixed-vs-FP64-oracle error
on the oracle's sample stations, FP64-mode throughput on the 80 x 80 x 40
workload, the error of the literal FP32 corner-term scheme there (against the
FP64 mode, beside the mixed scheme's), and the inversion time to relative
residual 1e-6 (mixed and FP64), and a bounded replay of the serving stream
(first 64 jobs).
Under torchrun (N > 1) every rank runs an independent replica (the operator
is single-GPU; replicas only) and `value` is the total over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

MUFU_PER_CLK_SM = 16          # reciprocal square roots per clock per SM (MUFU unit count)
SM_MAX_MHZ = 2032.0
DFMA_PER_CLK_SM = 1.65        # FP64 pipe operations per clock per SM (measured by grav_bench_pipes)
FP64_OPS_PER_PSI = 98         # FP64 pipe operations per Eq. 2-3 evaluation (ncu, k_adj64 on 80x80x40)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="paper_210x210x75")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--near-cells", type=float, default=8.0)
    ap.add_argument("--no-extras", action="store_true", help="skip fp64/inversion/cpu extras")
    ap.add_argument("--no-bench-inversion", action="store_true",
                    help="extras without the inversion of the bench workload itself (~40 s at paper scale)")
    ap.add_argument("--cpu-stations", type=int, default=16)
    ap.add_argument("--cpu-cells", type=int, default=48)
    ap.add_argument("--serve", action="store_true",
                    help="replay the seeded 256-job Poisson request stream through the serving scheduler")
    ap.add_argument("--serve-jobs", type=int, default=256)
    ap.add_argument("--serve-rate", type=float, default=20.0)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--invert", action="store_true", help="time one data-space inversion on --workload")
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--max-iter", type=int, default=5000)
    ap.add_argument("--reorth", type=int, default=1000,
                    help="--invert: residuals kept for reorthogonalised CG (0 = plain CG)")
    ap.add_argument("--precond", default="none", choices=["none", "jacobi", "nystrom"])
    ap.add_argument("--nys-rank", type=int, default=0, help="--precond nystrom: sketch size (0: automatic)")
    ap.add_argument("--nys-coarsen", type=int, default=0,
                    help="--precond nystrom: coarsening factor per axis (0: automatic)")
    ap.add_argument("--refine", type=int, default=0,
                    help="--invert --precision fp64: at most this many mixed-precision refinement steps "
                         "(FP64 residuals) instead of FP64 CG (0: FP64 CG)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if s[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples),
                "power_w_max": max(float(s[3]) for s in self.samples if s[3].replace(".", "").isdigit())
                if any(s[3].replace(".", "").isdigit() for s in self.samples) else None}


def oracle_sample(wl, n_st, n_cells, seed=0):
    """Times the CPU oracle on a bounded sample of the workload: the forward
    for n_st stations over the full mesh, the adjoint for n_cells cells over
    all stations.  Returns (pairs_per_s, seconds, threads, station idx, d_ref)."""
    import oracle
    rng = np.random.Generator(np.random.PCG64(100 + seed))
    idx = np.sort(rng.choice(wl.survey.n, n_st, replace=False))
    cells = np.sort(rng.choice(wl.mesh.ncells, n_cells, replace=False))
    r = synth.random_vector(wl.survey.n, 77)
    sub = wl.survey.subset(idx)
    t0 = time.perf_counter()
    d_ref = oracle.forward(wl.mesh, sub, wl.m)
    t1 = time.perf_counter()
    nx, ny = wl.mesh.nx, wl.mesh.ny
    for k in cells:
        i, j, l = k % nx, (k // nx) % ny, k // (nx * ny)
        one = synth.Mesh(wl.mesh.xe[i:i + 2].copy(), wl.mesh.ye[j:j + 2].copy(), wl.mesh.ze[l:l + 2].copy())
        oracle.adjoint(one, wl.survey, r)
    t2 = time.perf_counter()
    pairs = n_st * wl.mesh.ncells + n_cells * wl.survey.n
    return pairs / (t2 - t0), t2 - t0, oracle.get_threads(), idx, d_ref, (t1 - t0, t2 - t1)


def bench_config(args, M, N, ws):
    """The workload description both arms print (the reference arm times the
    oracle on a bounded sample of this same workload)."""
    return {"workload": args.workload, "cells": M, "stations": N, "precision": args.precision,
            "near_cells": args.near_cells, "l2": "flushed between steps (256 MB write)",
            "parallelism": "replicas" if ws > 1 else "single-gpu"}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    wl = synth.make_workload(args.workload)
    pairs_step = 2 * wl.survey.n * wl.mesh.ncells
    vals, secs = [], []
    for _ in range(args.warmup):
        oracle_sample(wl, 2, 4)
    for s in range(args.steps):
        pps, sec, th, _, _, _ = oracle_sample(wl, args.cpu_stations, args.cpu_cells, seed=s)
        vals.append(pps)
        secs.append(sec)
    v = statistics.median(vals)
    sample_pairs = args.cpu_stations * wl.mesh.ncells + args.cpu_cells * wl.survey.n
    line = {
        "impl": "reference", "metric": "prism-station pairs/s for G.m and G^T r", "value": v, "unit": "pairs/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(secs) / len(secs),
        "ms_per_step_basis": (f"measured: each timed step runs the oracle on a sample of {sample_pairs:.4g} "
                              f"pairs of the workload; one full step ({pairs_step:.4g} pairs) would take "
                              f"{pairs_step / v:.4g} s at the measured rate (extrapolated, not run)"),
        "sample_pairs_per_step": sample_pairs, "full_step_ms_extrapolated": pairs_step / v * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(args, wl.mesh.ncells, wl.survey.n, ws),
        "cpu_baseline": {"value": v, "unit": "pairs/s", "cores": th, "kind": "oracle",
                         "sample": f"forward of {args.cpu_stations} seeded stations over all {wl.mesh.ncells} "
                                   f"cells + adjoint of {args.cpu_cells} seeded cells over all {wl.survey.n} "
                                   f"stations, per step"},
        "e2e": {"value": v, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def aggregate(t_local_ms, ws, pairs_step, steps, device):
    """Whole-job throughput of `ws` replicas: the timed region is the MAX over
    ranks of each rank's device time (all-reduce when ws > 1), and every rank
    processed `steps` steps of `pairs_step` pairs.  Returns (t_ms, pairs/s)."""
    t = float(t_local_ms)
    if ws > 1:
        import torch
        import torch.distributed as dist
        tt = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    return t, ws * pairs_step * steps / (t * 1e-3)


def measured_traffic(kernel_name, args):
    """DRAM bytes per launch of `kernel_name` from the committed full-size ncu
    capture, if it was taken on this workload and the kernel sources are
    unchanged since (sha256 recorded with the capture)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic_paper_210x210x75_mixed.json")
    if args.workload != "paper_210x210x75" or args.precision != "mixed" or not os.path.exists(path):
        return None
    rec = json.load(open(path))
    if rec.get("near_cells") != args.near_cells:
        return None
    src = b"".join(open(os.path.join(ROOT, f), "rb").read() for f in rec["source_files"])
    if hashlib.sha256(src).hexdigest() != rec["source_sha256"]:
        return None
    k = rec["kernels"].get(kernel_name.replace(" ", ""))
    return None if k is None else k["dram_read_bytes"] + k["dram_write_bytes"]


def flush_l2(buf):
    buf.add_(1.0)


def run_ours(args):
    import torch
    import paper_2602_03857_b300 as g

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    wl = synth.make_workload(args.workload)
    N, M = wl.survey.n, wl.mesh.ncells
    S = g.Survey(wl.survey.x, wl.survey.y, wl.survey.z)
    opts = {"precision": args.precision, "near_cells": args.near_cells}
    t0 = time.perf_counter()
    plan = g.Plan(wl.mesh, S, **opts)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    m = torch.tensor(wl.m, dtype=torch.float64, device=dev)
    r = torch.tensor(synth.random_vector(N, 77), dtype=torch.float64, device=dev)
    d = torch.empty(N, dtype=torch.float64, device=dev)
    gt = torch.empty(M, dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > 126 MB L2
    stream = torch.cuda.current_stream()

    def step():
        plan.forward(m, out=d)
        plan.adjoint(r, out=gt)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    plan.timing(True, read=True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = g.launch_count()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush_l2(flush)
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    launches = g.launch_count() - launches0
    stages = plan.timing(False, read=True)
    ms = [a.elapsed_time(b) for a, b in ev]
    pairs_step = 2.0 * N * M
    t_total, value = aggregate(sum(ms), ws, pairs_step, args.steps, dev)

    # e2e: same metric through the public API with pinned host buffers
    hm = torch.tensor(wl.m, dtype=torch.float64).pin_memory()
    hr = torch.tensor(synth.random_vector(N, 77), dtype=torch.float64).pin_memory()
    hd = torch.empty(N, dtype=torch.float64).pin_memory()
    hg = torch.empty(M, dtype=torch.float64).pin_memory()
    md = torch.empty_like(m)
    rd = torch.empty_like(r)

    def e2e_step():
        md.copy_(hm, non_blocking=True)
        plan.forward(md, out=d)
        hd.copy_(d, non_blocking=True)
        rd.copy_(hr, non_blocking=True)
        plan.adjoint(rd, out=gt)
        hg.copy_(gt, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    e_ms = []
    for k in range(args.steps):
        flush_l2(flush)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e2e_step()
        b.record(stream)
        b.synchronize()
        e_ms.append(a.elapsed_time(b))
    e2e_value = ws * pairs_step * args.steps / (sum(e_ms) * 1e-3)

    # roofline of the dominant kernel (MUFU reciprocal square root per pair)
    fwd_ms, fwd_n = stages["fwd_main"]
    adj_ms, adj_n = stages["adj_main"]
    dom = "fwd_main" if fwd_ms >= adj_ms else "adj_main"
    dms, dn = stages[dom]
    if args.precision == "mixed":
        units_launch = float(N) * M          # one MUFU rsqrt per (station, cell) pair
        peak = 148 * MUFU_PER_CLK_SM * SM_MAX_MHZ * 1e6 / 1e9
        peak_basis = f"148 SMs x {MUFU_PER_CLK_SM} MUFU/clk x {SM_MAX_MHZ:.0f} MHz (MUFU unit count x max SM clock)"
    else:
        units_launch = float(N) * (wl.mesh.nx + 1) * (wl.mesh.ny + 1) * (wl.mesh.nz + 1)   # Psi per (station, node)
        peak = 148 * DFMA_PER_CLK_SM * SM_MAX_MHZ * 1e6 / FP64_OPS_PER_PSI / 1e9
        peak_basis = (f"148 SMs x {DFMA_PER_CLK_SM} FP64 ops/clk x {SM_MAX_MHZ:.0f} MHz / {FP64_OPS_PER_PSI} FP64 ops "
                      "per Psi (ncu instruction count)")
    achieved = units_launch / (dms / max(dn, 1) * 1e-3) / 1e9
    desc = plan.describe()
    kernel_name = desc["fwd_kernel"] if dom == "fwd_main" else desc["adj_kernel"]
    traffic = measured_traffic(kernel_name, args)
    roof = {"bound": "alu", "kernel": kernel_name, "achieved": achieved, "peak": peak,
            "unit": "G rsqrt/s (MUFU, 1 per pair)" if args.precision == "mixed" else "G node-evals/s",
            "frac": achieved / peak, "traffic": traffic,
            "traffic_note": "ncu dram__bytes_read+write per launch at full size (profiles/), null if the "
                            "kernel sources changed since the capture",
            "peak_basis": peak_basis,
            "stage_ms_per_launch": {k: (v[0] / max(v[1], 1)) for k, v in stages.items()}}

    line = {
        "metric": "prism-station pairs/s for G.m and G^T r", "value": value, "unit": "pairs/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": bench_config(args, M, N, ws),
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": "pairs/s", "h2d_bytes_per_step": 8 * (M + N),
                "d2h_bytes_per_step": 8 * (N + M)},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "plan_setup_s": setup_s, "plan_bytes": plan.nbytes,
    }
    if ws == 1 and not args.no_extras:   # the CPU baseline and the extras run at N = 1 only
        extras(args, g, torch, wl, plan, d, line)
    plan.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


def extras(args, g, torch, wl, plan, d, line):
    # CPU oracle on a bounded sample; its forward sample also measures the
    # error of this run's result against the FP64 oracle
    # (4x the stations and 2x the cells of one reference-arm step: ~10-15 s of CPU work)
    n_st, n_cells = 4 * args.cpu_stations, 2 * args.cpu_cells
    pps, sec, th, idx, d_ref, (tf, ta) = oracle_sample(wl, n_st, n_cells)
    line["cpu_baseline"] = {"value": pps, "unit": "pairs/s", "cores": th, "kind": "oracle",
                            "sample": f"forward of {n_st} seeded stations over all {wl.mesh.ncells} "
                                      f"cells + adjoint of {n_cells} seeded cells over all {wl.survey.n} "
                                      f"stations ({sec:.1f} s)"}
    dg = d.cpu().numpy()[idx]
    line["error_vs_fp64_oracle"] = {
        "max_abs_mgal": float(np.abs(dg - d_ref).max()),
        "rel_to_max_abs": float(np.abs(dg - d_ref).max() / np.abs(d_ref).max()),
        "stations_checked": int(len(idx))}
    # FP64 mode throughput and mixed/FP64 ratio on the 80x80x40 workload
    wl2 = synth.make_workload("vslab_80x80x40")
    S2 = g.Survey(wl2.survey.x, wl2.survey.y, wl2.survey.z)
    res = {}
    for prec in ("fp64", "mixed"):
        p2 = g.Plan(wl2.mesh, S2, precision=prec)
        m2 = torch.tensor(synth.random_vector(wl2.mesh.ncells, 3, 100.0), device="cuda")
        r2 = torch.tensor(synth.random_vector(wl2.survey.n, 4), device="cuda")
        p2.forward(m2); p2.adjoint(r2)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        p2.forward(m2); p2.adjoint(r2)
        b.record(); b.synchronize()
        res[prec] = 2.0 * wl2.survey.n * wl2.mesh.ncells / (a.elapsed_time(b) * 1e-3)
        p2.close()
    line["fp64_vs_mixed"] = {"workload": "vslab_80x80x40", "fp64_pairs_per_s": res["fp64"],
                             "mixed_pairs_per_s": res["mixed"], "mixed_over_fp64": res["mixed"] / res["fp64"]}
    # stored G (FP64 mode, cache_g): build once, then each product streams
    # N x M x 8 bytes from HBM; against the matrix-free FP64 products above
    m2 = torch.tensor(synth.random_vector(wl2.mesh.ncells, 3, 100.0), device="cuda")
    r2 = torch.tensor(synth.random_vector(wl2.survey.n, 4), device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pc = g.Plan(wl2.mesh, S2, precision="fp64", cache_g=True)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    if pc.describe().get("stored_g"):
        dc, ac = pc.forward(m2), pc.adjoint(r2)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(); dc = pc.forward(m2); ev[1].record(); ac = pc.adjoint(r2); ev[2].record()
        ev[2].synchronize()
        tf, ta = ev[0].elapsed_time(ev[1]) * 1e-3, ev[1].elapsed_time(ev[2]) * 1e-3
        gbytes = 8.0 * wl2.survey.n * wl2.mesh.ncells / 1e9
        p64 = g.Plan(wl2.mesh, S2, precision="fp64")
        d64, a64 = p64.forward(m2), p64.adjoint(r2)
        p64.close()
        peak = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")))["hbm_gbs"] \
            if os.path.exists(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) else 6400.0
        line["stored_g_fp64"] = {
            "workload": "vslab_80x80x40", "g_bytes": gbytes * 1e9, "build_s": build_s,
            "forward_ms": tf * 1e3, "adjoint_ms": ta * 1e3,
            "pairs_per_s": 2.0 * wl2.survey.n * wl2.mesh.ncells / (tf + ta),
            "forward_gbs": gbytes / tf, "adjoint_gbs": gbytes / ta, "hbm_peak_gbs": peak,
            "forward_frac": gbytes / tf / peak, "adjoint_frac": gbytes / ta / peak,
            "rel_diff_vs_matrix_free": max(float((dc - d64).abs().max() / d64.abs().max()),
                                           float((ac - a64).abs().max() / a64.abs().max())),
            "what": "G formed once in FP64 (cache_g), stored as double-float pairs and streamed per product (double-float arithmetic); algorithmic bytes = N x M x 8 per product"}
    pc.close()
    # the literal FP32 corner-term scheme (forward only) against the FP64 mode
    # on every station of the 80x80x40 workload, next to the mixed scheme
    mv = torch.tensor(wl2.m, device="cuda")
    ref = g.forward(mv, wl2.mesh, S2, precision="fp64")
    corner = {}
    for prec in ("mixed_corner", "mixed"):
        p2 = g.Plan(wl2.mesh, S2, precision=prec)
        p2.forward(mv)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        dv = p2.forward(mv)
        b.record(); b.synchronize()
        corner[prec] = {"rel_err_to_max": float((dv - ref).abs().max() / ref.abs().max()),
                        "forward_ms": a.elapsed_time(b)}
        p2.close()
    line["fp32_corner_vs_mixed"] = {"workload": "vslab_80x80x40", "stations_checked": wl2.survey.n,
                                    "reference": "FP64 mode", **corner}
    # inversion time to relative residual 1e-6, mixed and FP64 (data from the FP64 forward)
    wl1 = synth.make_workload("block_20x20x10")
    S1 = g.Survey(wl1.survey.x, wl1.survey.y, wl1.survey.z)
    d1 = g.forward(torch.tensor(wl1.m, device="cuda"), wl1.mesh, S1, precision="fp64").cpu().numpy()
    d1 = synth.add_noise(d1, wl1.noise_abs, wl1.noise_rel, 0)
    inv = {}
    for prec in ("fp64", "mixed"):
        g.datainv(torch.tensor(d1, device="cuda"), wl1.mesh, S1, precision=prec, tol=1e-6)
        mm, info = g.datainv(torch.tensor(d1, device="cuda"), wl1.mesh, S1, precision=prec, tol=1e-6)
        inv[prec] = {"seconds": info["seconds"], "iters": info["iters"], "true_rel_res": info["true_rel_res"]}
    line["inversion_to_1e-6"] = {"workload": "block_20x20x10", **inv}
    # mixed inversion at 150 x 150 x 60 cells x 22,801 stations (data from the mixed forward)
    wl3 = synth.make_workload("dipdyke_150x150x60")
    S3 = g.Survey(wl3.survey.x, wl3.survey.y, wl3.survey.z)
    d3 = g.forward(torch.tensor(wl3.m, device="cuda"), wl3.mesh, S3, precision="mixed")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mm, info = g.datainv(d3, wl3.mesh, S3, precision="mixed", tol=1e-6, max_iter=5000, check_stations=64)
    torch.cuda.synchronize()
    line["inversion_to_1e-6_150x150x60"] = {
        "workload": "dipdyke_150x150x60", "precision": "mixed", "seconds": time.perf_counter() - t0,
        "iters": info["iters"], "true_rel_res": info["true_rel_res"],
        "fp64_rel_err_of_predicted_data": info["fp64_rel_err"],
        "what": "one grav_datainv_solve call: plan set-up, trace, reorthogonalised CG, recovery"}
    t0 = time.perf_counter()
    mm, info = g.datainv(d3, wl3.mesh, S3, precision="mixed", tol=1e-6, max_iter=5000, check_stations=64,
                         precond="nystrom")
    torch.cuda.synchronize()
    line["inversion_to_1e-6_150x150x60_nystrom"] = {
        "workload": "dipdyke_150x150x60", "precision": "mixed", "seconds": time.perf_counter() - t0,
        "iters": info["iters"], "true_rel_res": info["true_rel_res"],
        "fp64_rel_err_of_predicted_data": info["fp64_rel_err"],
        "what": "as above with the randomized Nystrom preconditioner (automatic rank and coarsening; sketch "
                "included)"}
    # inversion time to 1e-6 at 80 x 80 x 40 cells x 6,561 stations, FP64 against mixed
    # (data: the FP64 forward of the slab model plus 1 % + 0.01 mGal seeded noise)
    d2 = g.forward(torch.tensor(wl2.m, device="cuda"), wl2.mesh, S2, precision="fp64").cpu().numpy()
    d2 = torch.tensor(synth.add_noise(d2, wl2.noise_abs, wl2.noise_rel, 0), device="cuda")
    vs = {}
    for key, prec, pc, refine, cache in (("fp64", "fp64", "nystrom", 0, False),
                                         ("fp64_stored_g", "fp64", "none", 0, True),
                                         ("fp64_refined", "fp64", "none", 8, False),
                                         ("mixed", "mixed", "none", 0, False)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mm, info = g.datainv(d2, wl2.mesh, S2, precision=prec, tol=1e-6, max_iter=5000, precond=pc,
                             check_stations=64 if prec == "mixed" else 0, refine=refine, cache_g=cache)
        torch.cuda.synchronize()
        vs[key] = {"seconds": time.perf_counter() - t0, "precond": pc, "iters": info["iters"],
                   "converged": info["converged"], "true_rel_res": info["true_rel_res"]}
        if prec == "mixed":
            vs[key]["fp64_rel_err_of_predicted_data"] = info["fp64_rel_err"]
        if refine:
            vs[key]["refine_steps"] = info["outer"]
    line["inversion_to_1e-6_vslab_80x80x40"] = {
        "workload": "vslab_80x80x40", **vs, "fp64_over_mixed_seconds": vs["fp64"]["seconds"] / vs["mixed"]["seconds"],
        "fp64_refined_over_mixed_seconds": vs["fp64_refined"]["seconds"] / vs["mixed"]["seconds"],
        "fp64_stored_g_over_mixed_seconds": vs["fp64_stored_g"]["seconds"] / vs["mixed"]["seconds"],
        "what": "one grav_datainv_solve call each (plan set-up, trace, CG to a true relative residual of 1e-6, "
                "recovery); fp64: FP64 CG with the Nystrom preconditioner (sketch included; without it ~100 s); "
                "fp64_stored_g: FP64 CG with G formed once in FP64 and stored as double-float pairs (cache_g; "
                "13.4 GB, build included; products in double-float arithmetic); fp64_refined: the same FP64 system by mixed-precision iterative refinement (mixed "
                "CG corrections, FP64 residuals; true_rel_res is the FP64 residual, iters the mixed CG "
                "iterations)"}
    # the serving loop on the first 64 jobs of the seeded request stream
    line["serving_64_jobs"] = serve_replay(g, torch, 64, 20.0, 8)
    # an inversion stream on one survey (80 x 80 x 40 cells x 6,561 stations, 16 data
    # vectors at 20/s, mixed, tol 1e-4): resident plans against a plan per job
    line["serving_same_survey_16_inversions"] = {
        "workload": "vslab_80x80x40, 16 inversions of different data on one survey, 20/s, 4 slots",
        "resident_plans": same_survey_stream(g, torch, wl2, S2, True),
        "plan_per_job": same_survey_stream(g, torch, wl2, S2, False)}
    # FP64 mode at paper scale, bounded: the operator pair on 1,024 of the stations
    if args.workload == "paper_210x210x75":
        sub = wl.survey.subset(np.linspace(0, wl.survey.n - 1, 1024).astype(int))
        Ss = g.Survey(sub.x, sub.y, sub.z)
        p64 = g.Plan(wl.mesh, Ss, precision="fp64")
        m64 = torch.tensor(wl.m, device="cuda")
        r64 = torch.tensor(synth.random_vector(sub.n, 5), device="cuda")
        p64.forward(m64); p64.adjoint(r64)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        p64.forward(m64); p64.adjoint(r64)
        b.record(); b.synchronize()
        ms64 = a.elapsed_time(b)
        p64.close()
        line["fp64_paper_scale_1024_stations"] = {
            "pairs_per_s": 2.0 * sub.n * wl.mesh.ncells / (ms64 * 1e-3), "ms_per_pair_of_products": ms64,
            "what": "FP64 forward + adjoint on all 3,307,500 cells and 1,024 evenly spaced stations of the bench "
                    "workload; the full survey at this rate is the FP64 operator pair's cost per CG iteration"}
    if args.precision == "mixed" and not args.no_bench_inversion:
        # the bench workload itself (210 x 210 x 75 cells x 178,797 stations by default):
        # data = the last timed forward product (mixed operator), Nystrom-preconditioned CG
        S0 = g.Survey(wl.survey.x, wl.survey.y, wl.survey.z)
        dd = d.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mm, info = g.datainv(dd, wl.mesh, S0, precision="mixed", near_cells=args.near_cells, tol=1e-6,
                             max_iter=5000, check_stations=64, precond="nystrom")
        torch.cuda.synchronize()
        line["inversion_to_1e-6_" + args.workload + "_nystrom"] = {
            "workload": args.workload, "precision": "mixed", "seconds": time.perf_counter() - t0,
            "iters": info["iters"], "converged": info["converged"], "true_rel_res": info["true_rel_res"],
            "nys_setup_s": info["nys_setup_s"], "nys_shift_over_lambda": info["nys_shift"],
            "fp64_rel_err_of_predicted_data": info["fp64_rel_err"],
            "what": "one grav_datainv_solve call on the bench workload (data: its mixed forward product), "
                    "Nystrom-preconditioned, sketch and plan set-up included"}


def run_serve(args):
    import torch
    import paper_2602_03857_b300 as g
    torch.cuda.set_device(0)
    print(json.dumps(serve_replay(g, torch, args.serve_jobs, args.serve_rate, args.serve_slots)), flush=True)


def serve_replay(g, torch, n_jobs, rate, slots):
    """Request-loop benchmark: jobs arrive at their seeded Poisson times (rate
    `rate`), each a forward or an inversion (mixed precision, CG tolerance
    1e-4 as in the paper's inner CG) on its own mesh and survey; latency =
    completion - submission (steady clock inside libgrav)."""
    jobs = synth.serving_jobs(n_jobs, rate, seed=0)
    prepared = []
    for j in jobs:
        S = g.Survey(j.survey.x, j.survey.y, j.survey.z)
        m = torch.tensor(j.m, dtype=torch.float64, device="cuda")
        if j.kind == "forward":
            inp, out = m, torch.empty(j.survey.n, dtype=torch.float64, device="cuda")
        else:
            inp = g.forward(m, j.mesh, S, precision="mixed")
            out = torch.empty(j.mesh.ncells, dtype=torch.float64, device="cuda")
        prepared.append((j, S, inp, out))
    torch.cuda.synchronize()
    ctx = g.Context(0)
    ctx.serve_config(slots)
    opts = dict(precision="mixed", tol=1e-4, max_iter=500, check_stations=16)
    t0 = time.perf_counter()
    ids = []
    for j, S, inp, out in prepared:
        delay = j.arrival_s - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        ids.append(ctx.submit(j.kind, j.mesh, S, inp, out, **opts))
    results = [ctx.wait(i, 3600.0) for i in ids]
    wall = time.perf_counter() - t0
    lat, lat_f, lat_i, busy, errs = [], [], [], [], []
    pairs = 0.0
    pairs_done = 0.0   # operator pairs the jobs evaluated (far field, every product counted)
    for (j, S, inp, out), i in zip(prepared, ids):
        st, inf = ctx.poll(i)
        e = inf["fp64_rel_err"]
        if e >= 0:
            errs.append(e)
        npm = float(j.survey.n) * j.mesh.ncells
        # inversion: diag/trace (1 pass), 2 passes per CG iteration, the final
        # true residual (2) and recovery (1); forward: 1 pass
        pairs_done += npm * (2 * inf["iters"] + 4) if j.kind != "forward" else npm
        ts, tb, te = ctx.job_times(i)
        lat.append(te - ts)
        (lat_f if j.kind == "forward" else lat_i).append(te - ts)
        busy.append((tb, te))
        pairs += float(j.survey.n) * j.mesh.ncells
    ctx.close()
    pct = lambda v, q: float(np.percentile(np.array(v), q)) if v else None
    line = {"metric": "serving latency and throughput (mixed precision)", "jobs": len(jobs),
            "arrival_rate_hz": rate, "slots": slots, "wall_s": wall,
            "throughput_jobs_per_s": len(jobs) / wall,
            "offered_load_jobs_per_s": len(jobs) / max(j.arrival_s for j in jobs),
            "p50_latency_s": pct(lat, 50), "p99_latency_s": pct(lat, 99),
            "forward": {"n": len(lat_f), "p50_s": pct(lat_f, 50), "p99_s": pct(lat_f, 99)},
            "invert": {"n": len(lat_i), "p50_s": pct(lat_i, 50), "p99_s": pct(lat_i, 99)},
            "results": {str(k): results.count(k) for k in sorted(set(results))},
            "fp64_rel_err": {"jobs_checked": len(errs), "stations_per_job": 16,
                             "median": pct(errs, 50), "max": max(errs) if errs else None,
                             "what": "max |mixed - FP64| of each job's output (forward: d; inversion: G m_out) "
                                     "at 16 stations, relative to max |g| over the job's survey"},
            "pairs_per_forward_pass_total": pairs, "pairs_evaluated": pairs_done,
            "achieved_pairs_per_s": pairs_done / wall, "data": "synthetic",
            "config": {"workload": "serving mix: 50k-500k cubic prisms (25-100 m), 1k-20k stations, "
                                   "block/dyke models, forward or inversion 50/50", "tol": 1e-4}}
    return line


def same_survey_stream(g, torch, wl, S, resident):
    """16 inversion jobs on one mesh and survey (different data: the forward of
    the workload's model scaled and shifted per job), Poisson arrivals at
    20/s through 4 slots; returns latency percentiles, jobs/s and how many
    plans the scheduler built."""
    rng = np.random.Generator(np.random.PCG64(4242))
    d0 = g.forward(torch.tensor(wl.m, device="cuda"), wl.mesh, S, precision="mixed")
    datas = [d0 * float(0.5 + k / 16.0) + float(0.01 * k) for k in range(16)]
    outs = [torch.empty(wl.mesh.ncells, dtype=torch.float64, device="cuda") for _ in datas]
    arrivals = np.cumsum(rng.exponential(1.0 / 20.0, len(datas)))
    torch.cuda.synchronize()
    ctx = g.Context(0)
    ctx.serve_config(4)
    ctx.plan_cache(16 if resident else 0)
    opts = dict(precision="mixed", tol=1e-4, max_iter=500)
    t0 = time.perf_counter()
    ids = []
    for t_arr, dk, ok in zip(arrivals, datas, outs):
        delay = t_arr - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        ids.append(ctx.submit("invert", wl.mesh, S, dk, ok, **opts))
    res = [ctx.wait(i, 600.0) for i in ids]
    wall = time.perf_counter() - t0
    lat = [ctx.job_times(i)[2] - ctx.job_times(i)[0] for i in ids]
    setup = [ctx.job_plan(i)["setup_s"] for i in ids]
    st = ctx.serve_stats()
    ctx.close()
    return {"jobs": len(ids), "ok": res.count(0), "wall_s": wall, "jobs_per_s": len(ids) / wall,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "plans_built": st["plans_built"], "plans_reused": st["plans_reused"],
            "plan_setup_s_total": float(sum(setup))}


def run_invert(args):
    """Time to relative residual args.tol for the data-space inversion of
    Eq. 10-11 on args.workload: data d = G m_true from the FP64 operator when
    it is affordable (else the mixed one), then m = W^-2 G^T y by CG with the
    operator of args.precision; the clock covers plan set-up, diag/trace, CG
    and the final recovery (one call of grav_datainv_solve)."""
    import torch
    import paper_2602_03857_b300 as g
    torch.cuda.set_device(0)
    wl = synth.make_workload(args.workload)
    S = g.Survey(wl.survey.x, wl.survey.y, wl.survey.z)
    m = torch.tensor(wl.m, dtype=torch.float64, device="cuda")
    data_prec = "fp64" if wl.survey.n * wl.mesh.ncells <= 2e9 else "mixed"
    d = g.forward(m, wl.mesh, S, precision=data_prec, near_cells=args.near_cells)
    torch.cuda.synchronize()
    opts = dict(precision=args.precision, near_cells=args.near_cells, tol=args.tol, max_iter=args.max_iter,
                precond=args.precond, check_stations=64 if args.precision != "fp64" else 0, reorth=args.reorth,
                nys_rank=args.nys_rank, nys_coarsen=args.nys_coarsen, refine=args.refine)
    t0 = time.perf_counter()
    m_out, info = g.datainv(d, wl.mesh, S, **opts)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    misfit = g.forward(m_out, wl.mesh, S, precision=data_prec, near_cells=args.near_cells) - d
    line = {"metric": "inversion time to relative residual", "workload": args.workload,
            "precision": args.precision, "precond": args.precond, "reorth": args.reorth, "tol": args.tol,
            "nys_rank": args.nys_rank if args.precond == "nystrom" else None,
            "seconds": wall,
            "iters": info["iters"],
            "converged": info["converged"], "true_rel_res": info["true_rel_res"], "lambda": info["lambda"],
            "cells": wl.mesh.ncells, "stations": wl.survey.n, "data_operator": data_prec,
            "rms_misfit_mgal": float(torch.sqrt(torch.mean(misfit * misfit))),
            "rms_data_mgal": float(torch.sqrt(torch.mean(d * d))), "data": "synthetic",
            "fp64_rel_err_of_predicted_data": info["fp64_rel_err"]}
    if args.precond == "nystrom":
        line["nys_setup_s"] = info["nys_setup_s"]
        line["nys_shift_over_lambda"] = info["nys_shift"]
    if args.refine:
        line["refine_steps"] = info["outer"]
        line["what"] = ("FP64 system solved by mixed-precision iterative refinement: iters counts the mixed CG "
                        "iterations, true_rel_res is the FP64 operator's residual")
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.serve:
        run_serve(args)
    elif args.invert:
        run_invert(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
