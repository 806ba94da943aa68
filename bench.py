#!/usr/bin/env python
"""Tile Cholesky benchmark on GB300: TFLOP/s = (n^3/3) / time, one JSON line on rank 0.

A step is one pass of the whole hot path over one synthetic Matern covariance matrix that
is already resident in HBM: (precision map, for mixed-precision workloads) + factorization
A = L L^T + a 1-RHS solve with iterative refinement + the Gaussian log-likelihood (Eq. 1).
The value counts only the n^3/3 flops of the factorization, so the solve's time is
overhead in the number.  Inputs are larger than L2 (tens of GB), so no flush is needed.

Multi-GPU: a single factorization needs a per-column exchange to shard, so N GPUs run N
independent replicas (one matrix each, seed + rank): weak scaling, no data-path
collective; a barrier and a max-reduction of the timing are the only collectives.

--impl reference times the CPU oracle (plain FP64 Cholesky, OpenMP) on a bounded sample
of the same workload (leading principal submatrix) on this machine's host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2410_09819_gb300 import inputs  # noqa: E402

METRIC = "Cholesky TFLOP/s (n^3/3) MxP vs FP64 on 1 GB300 at stated error; OOC link GB/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP64_FLOPS_PER_CLK_SM = 4.0   # GB300: 2 DFMA per clock per SM (nominal 1.25 TFLOP/s / 152 SMs / 2.07 GHz)
NSM = 152
CPU_SAMPLE_N = 8192


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="fp64_n65536", choices=sorted(inputs.WORKLOADS))
    ap.add_argument("--n", type=int, default=0, help="override n (smaller quick runs)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=CPU_SAMPLE_N)
    return ap.parse_args()


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return p, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": max(power) if power else None}


def kernel_source_sha() -> str:
    src = os.path.join(ROOT, "paper_2410_09819_gb300", "csrc", "k_fp64.cu")
    with open(src, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def profiled_traffic(kernel_tag: str, sha: str):
    """DRAM bytes per launch of the dominant kernel from a committed ncu summary, if the
    kernel source has not changed since it was captured (else None)."""
    path = os.path.join(ROOT, "profiles", f"{kernel_tag}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m_sha = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", text)
    m_tr = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m_sha or not m_tr or m_sha.group(1) != sha:
        return None
    return float(m_tr.group(1))


# --------------------------------------------------------------------------- our arm
def run_ours(args, ws, rank, local):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2410_09819_gb300 import tile_chol as tc

    w = inputs.WORKLOADS[args.workload]
    n = args.n or w.n
    b = w.tile
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    H = tc.Handle(local, stream=stream.cuda_stream)
    nt = tc.ntiles(n, b)
    T = tc.tile_count(n, b)
    seed = w.seed + 1000 * rank
    pts = inputs.uniform_points(n, seed, w.morton)
    A = torch.empty(T * b * b, dtype=torch.float64, device=dev)
    tc.tc_matern_tiles(H.h, n, b, torch.from_numpy(pts).to(dev), w.sigma2, w.range_a, w.nu, w.nugget, A)
    y = torch.from_numpy(inputs.gaussian(n, 1, seed + 7)[:, 0].copy()).to(dev)
    x = torch.empty_like(y)
    pmap = torch.zeros(nt * nt, dtype=torch.uint8, device=dev) if w.mixed else None
    loglik_launches = 2 * nt            # forward substitution + one dot product

    def step():
        st, ss = tc.tc_stats(), tc.tc_stats()
        if w.mixed:
            tc.tile_chol_precision_map(H.h, n, b, A, w.eps_high, w.band, w.prec_set, pmap)
        info = tc.tile_chol_factor(H.h, n, b, A, pmap, st)
        if info:
            raise RuntimeError(f"factorization failed at column {info}")
        tc.tile_chol_solve(H.h, 1, y, n, x, n, 2, 1e-13, ss)
        ll = tc.tile_chol_loglik(H.h, y)
        return st, ss, ll

    for _ in range(args.warmup):
        step()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    upd_flops = upd_ms = 0.0
    launches = 0
    agg = None
    for _ in range(args.steps):
        st, ss, ll = step()
        upd_flops += st.update_flops[0]
        upd_ms += st.t_update_ms[0]
        launches += st.kernel_launches + ss.kernel_launches + loglik_launches
        agg = (st, ss, ll)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if ws > 1:
        dist.barrier()
    t = ev0.elapsed_time(ev1) / 1e3
    if ws > 1:
        tt = torch.tensor([t], device=dev, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    flops = n ** 3 / 3.0
    value = ws * flops * args.steps / t / 1e12
    st, ss, ll = agg

    # roofline of the dominant kernel (FP64 SYRK/GEMM update on the DFMA pipe): ALU peak
    # = 152 SMs x 4 FP64 flops per clock x the maximum SM clock
    pk, pk_kind = peaks()
    fp64_peak = NSM * FP64_FLOPS_PER_CLK_SM * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    achieved = (upd_flops / (upd_ms / 1e3) / 1e12) if upd_ms > 0 else None
    sha = kernel_source_sha()
    traffic = profiled_traffic("dgemm_update_fp64_n65536", sha) if (n == 65536 and not w.mixed) else None
    roofline = {"kernel": "k_dgemm_update", "bound": "alu", "achieved": achieved, "peak": round(fp64_peak, 4),
                "unit": "TFLOP/s", "frac": (achieved / fp64_peak) if achieved else None, "traffic": traffic,
                "peak_source": f"ALU: 152 SMs x 4 FP64 flop/clk x {pk_kind} max SM clock",
                "update_share_of_step": (upd_ms / 1e3) / t if t > 0 else None}

    # end to end: the same step through host (pinned) buffers, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        Ah = torch.empty(A.numel(), dtype=torch.float64, pin_memory=True)
        Ah.copy_(A)
        del A                          # the end-to-end step reads A from host memory only
        torch.cuda.empty_cache()
        yh = y.cpu().pin_memory()
        xh = torch.empty_like(yh).pin_memory()
        maph = torch.zeros(nt * nt, dtype=torch.uint8, pin_memory=True) if w.mixed else None
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if w.mixed:
            tc.tile_chol_precision_map(H.h, n, b, Ah, w.eps_high, w.band, w.prec_set, maph)
        tc.tile_chol_factor(H.h, n, b, Ah, maph, None)
        tc.tile_chol_solve(H.h, 1, yh, n, xh, n, 2, 1e-13, None)
        ll_h = tc.tile_chol_loglik(H.h, yh)
        e1.record(stream)
        torch.cuda.synchronize()
        te = max(e0.elapsed_time(e1) / 1e3, time.perf_counter() - t0)
        if ws > 1:
            tt = torch.tensor([te], device=dev, dtype=torch.float64)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            te = float(tt.item())
        h2d = Ah.numel() * 8 * (2 if w.mixed else 1) + 2 * n * 8
        d2h = n * 8 + 8
        e2e = {"value": ws * flops / te / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "loglik_matches_device": bool(abs(ll_h - ll) <= 1e-9 * abs(ll))}
        del Ah

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(w, min(args.cpu_sample, n), pts)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if not w.mixed else "f64+f32/tf32+f16+e4m3",
            "data": "synthetic", "impl": "ours",
            "config": {"workload": w.name, "n": n, "tile": b, "nu": w.nu, "range": w.range_a, "sigma2": w.sigma2,
                       "nugget": w.nugget, "points": "seeded uniform in [0,1]^2" + (", Morton-sorted" if w.morton else ""),
                       "precision": "per-tile map" if w.mixed else "FP64", "parallelism": f"replicas x{ws}",
                       "l2": "inputs larger than L2 (no flush needed)",
                       "step": "map+factor+solve(1 RHS, <=2 refinement)+loglik" if w.mixed
                       else "factor+solve(1 RHS, <=2 refinement)+loglik"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk,
            "gpu_launches": launches,
            "detail": {"t_factor_ms": st.t_ms, "t_update_ms": list(st.t_update_ms), "t_potrf_ms": st.t_potrf_ms,
                       "t_trsm_ms": st.t_trsm_ms, "t_convert_ms": st.t_convert_ms, "t_solve_ms": ss.t_ms,
                       "berr": ss.berr, "refine_iters": ss.refine_iters, "loglik": ll,
                       "update_tflops_by_prec": [(st.update_flops[p] / st.t_update_ms[p] / 1e9) if st.t_update_ms[p] else None
                                                 for p in range(4)],
                       "tiles_by_prec": list(st.tiles), "kernel_source_sha": sha},
        }
        print(json.dumps(line), flush=True)
    H.close()


def cpu_baseline(w, ns, pts):
    """The oracle (plain FP64 Cholesky, OpenMP) on the leading ns x ns principal submatrix."""
    import oracle
    A = oracle.matern(pts[:ns], w.sigma2, w.range_a, w.nu, w.nugget)
    t0 = time.perf_counter()
    oracle.cholesky(A)
    t = time.perf_counter() - t0
    return {"value": ns ** 3 / 3.0 / t / 1e12, "unit": "TFLOP/s", "cores": oracle.threads(), "kind": "oracle",
            "sample": f"leading {ns}x{ns} principal submatrix of the workload, one factorization ({t:.1f} s)"}


# --------------------------------------------------------------------- reference arm
def run_reference(args, ws, rank):
    if rank != 0:
        return
    import oracle
    w = inputs.WORKLOADS[args.workload]
    n = args.n or w.n
    ns = min(args.cpu_sample, n)
    pts = inputs.uniform_points(n, w.seed, w.morton)[:ns]
    A = oracle.matern(pts, w.sigma2, w.range_a, w.nu, w.nugget)
    for _ in range(args.warmup):
        oracle.cholesky(A)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.cholesky(A)
    t = time.perf_counter() - t0
    value = ns ** 3 / 3.0 * args.steps / t / 1e12
    sample = f"leading {ns}x{ns} principal submatrix of {w.name}, one oracle factorization per step"
    line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": w.name, "n": n, "tile": w.tile, "sample_n": ns},
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": oracle.threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    ws, rank, local = dist_info()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    try:
        run_ours(args, ws, rank, local)
    finally:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
