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
CPU_SAMPLE_N = 12288
OOC_MXP_EPS, OOC_MXP_BAND = 1e-9, 2
DEFAULT_WORKLOAD = "mxp4_n131072"     # the metric's configuration: four precisions, n = 131072


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(inputs.WORKLOADS) + ["batched"])
    ap.add_argument("--count", type=int, default=512, help="batched workload: number of matrices")
    ap.add_argument("--fp64-mode", type=int, default=2, choices=[0, 1, 2],
                    help="FP64 updates: 0 DFMA pipe, 1 emulated on FP8 tensor cores (exact digit planes), "
                         "2 as 1 plus inverse-based TRSM in mixed precision")
    ap.add_argument("--fp32-updates", type=int, default=0, choices=[0, 1],
                    help="FP32 output tiles with emulated FP64: 0 on 10 digit planes, 1 as TF32 x 3")
    ap.add_argument("--n", type=int, default=0, help="override n (smaller quick runs)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the accuracy probes after the timed region (the all-FP64 reference factor of the "
                         "four-precision line among them): a launch list then holds the timed step's kernels only")
    ap.add_argument("--cpu-sample", type=int, default=CPU_SAMPLE_N)
    ap.add_argument("--sweep", action="store_true",
                    help="accuracy / performance sweep of Section V: weak, medium, strong correlation x "
                         "accuracy levels 1e-5 .. 1e-11 (one JSON object; --n sets the order, default 65536)")
    ap.add_argument("--no-baselines", action="store_true",
                    help="skip the comparison factorizations of the FP64 workload (this library's FP64 path, "
                         "its DFMA engine, cuSOLVER potrf); the four-precision line keeps its all-FP64 factor "
                         "of the same matrix (accuracy reference and MxP-vs-FP64 multiple)")
    ap.add_argument("--ooc-policy", default="V3", choices=["V3", "V2", "V1", "async", "sync"],
                    help="out-of-core scheduling policy (Section III-C)")
    ap.add_argument("--ooc-eviction", default="lru", choices=["lru", "min"],
                    help="out-of-core eviction: least recently used, or Belady's MIN over the static schedule")
    ap.add_argument("--peaks", action="store_true",
                    help="measure the dense tensor-core peaks (cuBLAS FP8 / FP16 / BF16 / TF32 / FP64 GEMMs, "
                         "burst and sustained) and the pinned host-link rates; one JSON line")
    ap.add_argument("--ooc-mxp", action="store_true",
                    help="out-of-core workload in four precisions (map at eps_high 1e-9, FP64 band 2)")
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


def kernel_source_sha(name: str = "k_ozaki.cu") -> str:
    """First 16 hex digits of the SHA-256 of a kernel source file (the dominant kernel's by
    default): a committed ncu summary names the sha it was captured at."""
    src = os.path.join(ROOT, "paper_2410_09819_gb300", "csrc", name)
    with open(src, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


# --------------------------------------------------------------------------- our arm
def _tile_order(nt):
    import numpy as np
    i, j = np.tril_indices(nt)
    order = np.argsort(i * (i + 1) // 2 + j)
    return i[order], j[order]


def tiles_matvec(P, n, b, x, dev, kind):
    """Products with a matrix held as packed lower tiles P (tile layout, each tile column-major),
    in harness-side torch FP64 (for the accuracy probes, outside every timed region).
    kind "sym": the symmetric matrix (diagonal tiles symmetrised from their lower triangle);
    "L": the lower-triangular factor; "Lt": its transpose.  P may sit in host memory (it is
    then streamed to the device in chunks of 256 MB)."""
    import torch
    nt = -(-n // b)
    ti, tj = _tile_order(nt)
    X = torch.zeros(nt * b, dtype=torch.float64, device=dev)
    X[:n] = x
    X = X.view(nt, b)
    Y = torch.zeros(nt, b, dtype=torch.float64, device=dev)
    T = P.view(-1, b, b)                       # T[t] = tile (i, j) transposed
    chunk = max(1, (1 << 28) // (b * b * 8))
    for s0 in range(0, len(ti), chunk):
        ii = torch.from_numpy(ti[s0:s0 + chunk]).to(dev)
        jj = torch.from_numpy(tj[s0:s0 + chunk]).to(dev)
        Tt = T[s0:s0 + chunk].to(dev, non_blocking=True)
        diag = ii == jj
        if bool(diag.any()):
            Tt = Tt.clone()
            low = torch.triu(Tt[diag])         # the tile's lower triangle, transposed
            Tt[diag] = low + torch.triu(low, 1).transpose(1, 2) if kind == "sym" else low
        if kind in ("sym", "L"):
            Y.index_add_(0, ii, torch.bmm(X[jj].unsqueeze(1), Tt).squeeze(1))
        if kind == "sym":
            o = ~diag
            if bool(o.any()):
                Y.index_add_(0, jj[o], torch.bmm(Tt[o], X[ii[o]].unsqueeze(2)).squeeze(2))
        elif kind == "Lt":
            Y.index_add_(0, jj, torch.bmm(Tt, X[ii].unsqueeze(2)).squeeze(2))
    return Y.reshape(-1)[:n]


def factor_probe_berr(A, L, n, b, dev, nprobe=3, seed=5):
    """Random-probe backward error of a factor: max over Gaussian x of
    ||(A - L L^T) x|| / ||A x||, which estimates ||A - L L^T||_F / ||A||_F."""
    import torch
    g = torch.Generator(device=dev).manual_seed(seed)
    worst = 0.0
    for _ in range(nprobe):
        x = torch.randn(n, dtype=torch.float64, device=dev, generator=g)
        Ax = tiles_matvec(A, n, b, x, dev, "sym")
        LLx = tiles_matvec(L, n, b, tiles_matvec(L, n, b, x, dev, "Lt"), dev, "L")
        worst = max(worst, float((Ax - LLx).norm() / Ax.norm()))
    return worst


# Output precision -> (kernel, dtype its tensor work runs in, nominal ratio of that dtype's
# dense peak to BF16's).  FP64 and FP32 output tiles are updated on E4M3 digit planes.
KERNELS = {0: ("k_zgemm<14> (FP64 outputs, E4M3 digit planes)", "e4m3", 2.0),
           1: ("k_zgemm<10> (FP32 outputs, E4M3 digit planes)", "e4m3", 2.0),
           2: ("k_qgemm<2> (FP16 outputs)", "fp16", 1.0),
           3: ("k_qgemm<3> (FP8 E4M3 outputs)", "e4m3", 2.0)}


def committed_profile(tag: str, source: str = "k_ozaki.cu") -> dict:
    """The committed ncu summary profiles/<tag>.md of the dominant kernel: the kernel-source
    sha it was captured at (compared with the current sha of its source file) and its
    per-launch figures."""
    path = os.path.join(ROOT, "profiles", f"{tag}.md")
    try:
        text = open(path).read()
    except OSError:
        return {"file": f"profiles/{tag}.md", "present": False}
    m = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", text)
    out = {"file": f"profiles/{tag}.md", "present": True, "kernel_source_sha": m.group(1) if m else None}
    out["matches_current_source"] = bool(m) and m.group(1) == kernel_source_sha(source)
    for key in ("dram_bytes_per_launch", "l2_to_sm_bytes_per_launch", "tensor_active_pct", "launch_ms"):
        mm = re.search(rf"{key}:\s*([0-9.eE+-]+)", text)
        if mm:
            out[key] = float(mm.group(1))
    return out


def probed_peaks() -> dict:
    """Dense GEMM peaks measured on this machine's GB300 by ``bench.py --peaks`` (the committed
    summary profiles/peaks_gb300.md carries them as a JSON line), or {} if absent."""
    try:
        text = open(os.path.join(ROOT, "profiles", "peaks_gb300.md")).read()
        m = re.search(r"^peaks_json:\s*(\{.*\})\s*$", text, flags=re.M)
        return json.loads(m.group(1)) if m else {}
    except (OSError, ValueError):
        return {}


MIXED_KERNELS = {0: "k_zgemm64 (FP64 outputs of a mixed map, 128 x 64 items, E4M3 digit planes)",
                 1: "k_zgemm64 (FP32 outputs of a mixed map, 128 x 64 items, E4M3 digit planes)"}


def tensor_rooflines(st, t_step, fp32_updates, mixed=False):
    """Per-precision tensor-core rooflines of the updates: executed tensor flops
    (tc_stats.tensor_flops) over the CUDA-event time of that precision's update launches,
    against the dtype's dense peak = measured BF16 (sustained: the kernels run inside a
    seconds-long step) x the nominal ratio (FP8 2, FP16 1, TF32 1/2)."""
    pk, pk_kind = peaks()
    bf16 = pk.get("bf16_tflops_sustained") or pk["bf16_tflops"]
    out = []
    for p in range(4):
        ms = st.t_update_ms[p]
        if ms <= 0 or st.tensor_flops[p] <= 0:
            continue
        name, dt, ratio = KERNELS[p]
        if mixed and p in MIXED_KERNELS:
            name = MIXED_KERNELS[p]
        if p == 1 and fp32_updates:
            name, dt, ratio = "k_qgemm<1> (FP32 outputs, TF32 x 3)", "tf32", 0.5
        executed = st.tensor_flops[p] / (ms / 1e3) / 1e12
        peak = bf16 * ratio
        probe = probed_peaks().get(f"{dt}_sustained")
        out.append({"precision": ["fp64", "fp32", "fp16", "fp8"][p], "kernel": name, "bound": "tensor",
                    "achieved": executed, "peak": peak, "unit": "TFLOP/s", "frac": executed / peak,
                    "peak_source": f"{pk_kind} bf16 sustained x nominal {dt}/bf16 ratio {ratio:g}",
                    "peak_probe": probe, "frac_of_probe": (executed / probe) if probe else None,
                    "algorithmic_tflops": st.update_flops[p] / (ms / 1e3) / 1e12,
                    "executed_per_algorithmic": st.tensor_flops[p] / st.update_flops[p],
                    "t_ms": ms, "share_of_step": (ms / 1e3) / t_step if t_step > 0 else None,
                    "launches": st.update_launches[p]})
    return out


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
    H = tc.Handle(local, stream=stream.cuda_stream, fp64_mode=args.fp64_mode, fp32_updates=args.fp32_updates)
    nt = tc.ntiles(n, b)
    T = tc.tile_count(n, b)
    seed = w.seed + 1000 * rank
    pts = inputs.uniform_points(n, seed, w.morton)
    A = torch.empty(T * b * b, dtype=torch.float64, device=dev)
    tc.tc_matern_tiles(H.h, n, b, torch.from_numpy(pts).to(dev), w.sigma2, w.range_a, w.nu, w.nugget, A)
    y = torch.from_numpy(inputs.gaussian(n, 1, seed + 7)[:, 0].copy()).to(dev)
    x = torch.empty_like(y)
    pmap = torch.zeros(nt * nt, dtype=torch.uint8, device=dev) if w.mixed else None

    def step():
        st, ss = tc.tc_stats(), tc.tc_stats()
        if w.mixed:
            tc.tile_chol_precision_map(H.h, n, b, A, w.eps_high, w.band, w.prec_set, pmap)
        info = tc.tile_chol_factor(H.h, n, b, A, pmap, st)
        if info:
            raise RuntimeError(f"factorization failed at column {info}")
        # one refined solve (FP64 refinement wins back the accuracy of a mixed-precision factor),
        # then Eq. 1 with the quadratic form y^T x of that solution; the plain quadratic form of
        # the factor is reported beside it in the accuracy block
        tc.tile_chol_solve(H.h, 1, y, n, x, n, 2, 1e-14, ss)
        ll = tc.tile_chol_loglik_solved(H.h, y, x)
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
    marks = [ev0]                       # per-step boundaries on the same stream (best / median)
    factor_ms = []
    for _ in range(args.steps):
        st, ss, ll = step()
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        marks.append(e)
        factor_ms.append(st.t_ms)
        upd_flops += st.update_flops[0]
        upd_ms += st.t_update_ms[0]
        # the refined log-likelihood repeats the solve's launches (plus its dot product)
        # factor + solve (counted by the library) + the log-likelihood's dot product + the map's
        # tile sums of squares (one launch for a device matrix)
        launches += st.kernel_launches + ss.kernel_launches + 1 + (1 if w.mixed else 0)
        agg = (st, ss, ll)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if ws > 1:
        dist.barrier()
    t = ev0.elapsed_time(ev1) / 1e3
    step_ms = [a.elapsed_time(c) for a, c in zip(marks[:-1], marks[1:])]
    if ws > 1:
        tt = torch.tensor([t], device=dev, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    flops = n ** 3 / 3.0
    value = ws * flops * args.steps / t / 1e12
    st, ss, ll = agg
    t_step = t / args.steps

    # rooflines: per output precision on the tensor cores (the FP64 outputs' k_zgemm is the
    # dominant kernel), or the FP64 pipe for the DFMA engine
    pk, pk_kind = peaks()
    by_prec = tensor_rooflines(st, t_step, args.fp32_updates, w.mixed) if args.fp64_mode >= 1 else []
    if args.fp64_mode >= 1 and by_prec:
        roofline = dict(by_prec[0])
        roofline["traffic"] = None
        roofline["traffic_note"] = ("DRAM bytes per launch are not captured at this size; the committed "
                                    "ncu summary of k_zgemm gives them for its captured case")
    else:
        fp64_peak = NSM * FP64_FLOPS_PER_CLK_SM * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        achieved = (upd_flops / (upd_ms / 1e3) / 1e12) if upd_ms > 0 else None
        roofline = {"kernel": "k_dgemm_update", "bound": "alu", "achieved": achieved, "peak": round(fp64_peak, 4),
                    "unit": "TFLOP/s", "frac": (achieved / fp64_peak) if achieved else None, "traffic": None,
                    "peak_source": f"ALU: 152 SMs x 4 FP64 flop/clk x {pk_kind} max SM clock",
                    "share_of_step": (upd_ms / 1e3) / t if t > 0 else None}
    ksrc = "k_ozaki64.cu" if w.mixed else "k_ozaki.cu"
    roofline["kernel_source"] = f"csrc/{ksrc}"
    roofline["kernel_source_sha"] = kernel_source_sha(ksrc)
    roofline["profile"] = committed_profile("zgemm_mxp4_n32768" if w.mixed else "zgemm_fp64_n16384", ksrc)

    # accuracy of a mixed-precision factorization, outside the timed region: random-probe
    # backward error of the factor, Eq. 1 with the plain and the refined quadratic form, Eq. 3
    # at y = 0, against the same matrix factored with an all-FP64 map (the FP64 path, whose
    # factorization time is the MxP-vs-FP64 comparison)
    accuracy = None
    comparisons = {} if (rank == 0 and ws == 1) else None
    Ah = None
    if not w.mixed and not args.no_accuracy:
        # the FP64 line states its factor's backward error too (A and L both fit on the device)
        L = torch.empty(T * b * b, dtype=torch.float64, device=dev)
        tc.tile_chol_get_factor(H.h, L)
        accuracy = {"factor_berr_probe": factor_probe_berr(A, L, n, b, dev),
                    "factor_berr_probe_method": "max over 3 Gaussian x of ||(A - L L^T) x|| / ||A x|| (torch FP64 "
                                                "products with the packed tiles of A and of the factor)",
                    "solve_berr_refined": ss.berr,
                    "meaning": "normwise backward error of the factor; the emulated FP64 updates are normwise "
                               "FP64 (relative to each tile pair's scale)"}
        del L
        torch.cuda.empty_cache()
    if w.mixed and not args.no_accuracy:
        ld_mxp = tc.tile_chol_logdet(H.h)
        ll_plain = tc.tile_chol_loglik(H.h, y)
        ll_ref5, berr_mxp = tc.tile_chol_loglik_refined(H.h, y, 5, 1e-14)
        # the probe needs L and A at once: A moves to pinned host memory (streamed from there)
        Ah = torch.empty(A.numel(), dtype=torch.float64, pin_memory=True)
        Ah.copy_(A)
        del A
        A = None
        torch.cuda.empty_cache()
        L = torch.empty(T * b * b, dtype=torch.float64, device=dev)
        tc.tile_chol_get_factor(H.h, L)
        probe_mxp = factor_probe_berr(Ah, L, n, b, dev)
        del L
        torch.cuda.empty_cache()
        s64 = tc.tc_stats()
        if tc.tile_chol_factor(H.h, n, b, Ah, None, s64) == 0:
            ld64 = tc.tile_chol_logdet(H.h)
            ll64, berr64 = tc.tile_chol_loglik_refined(H.h, y, 5, 1e-14)
            ll64_plain = tc.tile_chol_loglik(H.h, y)
            accuracy = {
                "factor_berr_probe": probe_mxp,
                "factor_berr_probe_method": "max over 3 Gaussian x of ||(A - L L^T) x|| / ||A x|| (torch FP64 "
                                            "products with the packed tiles of A and of the factor)",
                "accuracy_level_eps_high": w.eps_high,
                "loglik_fp64": ll64, "loglik_mxp": ll, "loglik_rel_err": abs(ll - ll64) / abs(ll64),
                "loglik_mxp_unrefined": ll_plain,
                "loglik_unrefined_rel_err": abs(ll_plain - ll64) / abs(ll64),
                "loglik_fp64_unrefined": ll64_plain,
                "loglik_mxp_refined_5": ll_ref5, "loglik_refined_5_rel_err": abs(ll_ref5 - ll64) / abs(ll64),
                "logdet_fp64": ld64, "logdet_mxp": ld_mxp, "logdet_rel_err": abs(ld_mxp - ld64) / abs(ld64),
                "kl_divergence": 0.5 * (ld_mxp - ld64),
                "solve_berr_mxp_refined": berr_mxp, "solve_berr_fp64_refined": berr64,
                "reported_loglik": "Eq. 1 with the quadratic form of a refined solve (FP64 iterative "
                                   "refinement on the MxP factor); the plain form is loglik_mxp_unrefined",
                "reference": "same matrix, all-FP64 map, same engine (the FP64 path), refined solve"}
            if comparisons is not None:
                comparisons["fp64_same_engine"] = {
                    "value": flops / (s64.t_ms / 1e3) / 1e12, "unit": "TFLOP/s", "t_factor_ms": s64.t_ms,
                    "mxp_t_factor_ms": st.t_ms, "mxp_factor_speedup": s64.t_ms / st.t_ms,
                    "what": "this library's FP64 path (all-FP64 map) on the same matrix, one factorization"}

    # end to end: the same step through host (pinned) buffers, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        if Ah is None:
            Ah = torch.empty(A.numel(), dtype=torch.float64, pin_memory=True)
            Ah.copy_(A)
            del A                      # the end-to-end step reads A from host memory only
            A = None
            torch.cuda.empty_cache()
        yh = y.cpu().pin_memory()
        xh = torch.empty_like(yh).pin_memory()
        maph = torch.zeros(nt * nt, dtype=torch.uint8, pin_memory=True) if w.mixed else None

        def e2e_step():
            # the user's calls on host buffers: map and factor from one copy of A over the link
            if w.mixed:
                tc.tile_chol_factor_mapped(H.h, n, b, Ah, w.eps_high, w.band, w.prec_set, maph, None)
            else:
                tc.tile_chol_factor(H.h, n, b, Ah, None, None)
            tc.tile_chol_solve(H.h, 1, yh, n, xh, n, 2, 1e-14, None)
            return tc.tile_chol_loglik_solved(H.h, yh, xh)

        e2e_step()                     # warm-up: the handle's device copy of A is allocated once
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ll_h = e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        te = max(e0.elapsed_time(e1) / 1e3, time.perf_counter() - t0)
        if ws > 1:
            tt = torch.tensor([te], device=dev, dtype=torch.float64)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            te = float(tt.item())
        h2d = Ah.numel() * 8 + 3 * n * 8          # A once; y for the solve, y and x for Eq. 1
        d2h = n * 8 + 8
        e2e = {"value": ws * flops / te / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "loglik_matches_device": bool(abs(ll_h - ll) <= 1e-9 * abs(ll))}
    if A is None:
        A = Ah                         # the matrix now lives in pinned host memory

    if comparisons is not None and not w.mixed and not args.no_baselines:
        comparisons.update(fp64_baselines(tc, n, b, A, local, stream))
    H.close()
    del A, Ah
    torch.cuda.empty_cache()
    if comparisons is not None and w.mixed and not args.no_baselines:
        # the FP64 workload (n = 65536, tile 1024): this library's FP64 path, its DFMA engine
        # and cuSOLVER potrf on the same matrix, measured in the same run
        comparisons["fp64_n65536"] = fp64_workload_comparisons(tc, local, stream)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(w, min(args.cpu_sample, n), pts)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": ("f64" if args.fp64_mode == 0 else "f64 (updates emulated on e4m3 tensor cores)")
            if not w.mixed else "f64+f32+f16+e4m3 (f64/f32 updates on e4m3 digit planes)",
            "data": "synthetic", "impl": "ours",
            "config": workload_config(w, n, b, ws),
            "roofline": roofline,
            "roofline_by_precision": by_prec,
            "accuracy": accuracy,
            "comparisons": comparisons,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk,
            "gpu_launches": launches,
            "detail": {"t_factor_ms": st.t_ms, "t_update_ms": list(st.t_update_ms), "t_potrf_ms": st.t_potrf_ms,
                       "t_trsm_ms": st.t_trsm_ms, "t_convert_ms": st.t_convert_ms, "t_solve_ms": ss.t_ms,
                       "berr": ss.berr, "refine_iters": ss.refine_iters, "loglik": ll,
                       "update_tflops_by_prec": [(st.update_flops[p] / st.t_update_ms[p] / 1e9) if st.t_update_ms[p] else None
                                                 for p in range(4)],
                       "tensor_flops_by_prec": list(st.tensor_flops),
                       "tiles_by_prec": list(st.tiles), "kernel_source_sha": kernel_source_sha(ksrc),
                       "step_ms": step_ms, "step_ms_best": min(step_ms), "step_ms_median": float(np.median(step_ms)),
                       "factor_ms_steps": factor_ms,
                       "tflops_factor_only_best": flops / (min(factor_ms) / 1e3) / 1e12},
        }
        print(json.dumps(line), flush=True)


def fp64_workload_comparisons(tc, local, stream):
    """The FP64 workload (Matern nu = 1/2, range 0.05, n = 65536, tile 1024), outside the timed
    region: this library's FP64 path (fp64_mode 2, one factorization after one warm-up), then
    its DFMA engine and cuSOLVER potrf (fp64_baselines)."""
    import torch
    w = inputs.WORKLOADS["fp64_n65536"]
    n, b = w.n, w.tile
    dev = torch.device("cuda", local)
    A = torch.empty(tc.tile_count(n, b) * b * b, dtype=torch.float64, device=dev)
    out = {"workload": w.name, "n": n, "tile": b}
    with tc.Handle(local, stream=stream.cuda_stream, fp64_mode=2) as H:
        tc.tc_matern_tiles(H.h, n, b, torch.from_numpy(w.points()).to(dev), w.sigma2, w.range_a, w.nu, w.nugget, A)
        tc.tile_chol_factor(H.h, n, b, A, None, None)
        st = tc.tc_stats()
        if tc.tile_chol_factor(H.h, n, b, A, None, st) == 0:
            out["fp64_path"] = {"value": n ** 3 / 3.0 / (st.t_ms / 1e3) / 1e12, "unit": "TFLOP/s",
                                "t_factor_ms": st.t_ms,
                                "what": "this library, fp64_mode 2 (updates and TRSM on E4M3 digit planes)"}
    torch.cuda.empty_cache()
    out.update(fp64_baselines(tc, n, b, A, local, stream))
    del A
    torch.cuda.empty_cache()
    return out


def workload_config(w, n, b, ws):
    """The `config` object of a line for an in-core workload (both arms print the same)."""
    return {"workload": w.name, "n": n, "tile": b, "nu": w.nu, "range": w.range_a, "sigma2": w.sigma2,
            "nugget": w.nugget, "points": "seeded uniform in [0,1]^2" + (", Morton-sorted" if w.morton else ""),
            "precision": "per-tile map" if w.mixed else "FP64", "parallelism": f"replicas x{ws}",
            "l2": "inputs larger than L2 (no flush needed)",
            "step": ("map+" if w.mixed else "") + "factor+refined solve (1 RHS, <=2 FP64 refinement steps)"
                    "+loglik (Eq. 1) from that solve"}


def fp64_baselines(tc, n, b, A, local, stream):
    """Context numbers on the same matrix, outside the timed region: cuSOLVER potrf (through
    torch.linalg.cholesky on the dense matrix) and this library's FP64 path on the DFMA pipe
    (fp64_mode 0).  Each is one factorization after a small warm-up."""
    import torch
    out = {}
    dev = torch.device("cuda", local)
    flops = n ** 3 / 3.0
    # DFMA path
    with tc.Handle(local, stream=stream.cuda_stream, fp64_mode=0) as H0:
        st = tc.tc_stats()
        if tc.tile_chol_factor(H0.h, n, b, A, None, st) == 0:
            out["fp64_dfma_path"] = {"value": flops / (st.t_ms / 1e3) / 1e12, "unit": "TFLOP/s",
                                     "t_factor_ms": st.t_ms, "what": "this library, fp64_mode 0 (DFMA updates)"}
    torch.cuda.empty_cache()
    # cuSOLVER: dense lower triangle assembled from the tiles (plumbing only)
    Ad = A if A.is_cuda else A.to(dev)
    D = torch.zeros((n, n), dtype=torch.float64, device=dev)
    nt = -(-n // b)
    off = 0
    for m in range(nt):
        row = Ad[off:off + (m + 1) * b * b].view(m + 1, b, b).permute(2, 0, 1).reshape(b, (m + 1) * b)
        r1 = min((m + 1) * b, n)
        D[m * b:r1, :min((m + 1) * b, n)] = row[:r1 - m * b, :min((m + 1) * b, n)]
        off += (m + 1) * b * b
    del Ad
    D.tril_()                            # diagonal tiles may hold their upper part too
    D += D.T.triu(1)                     # the symmetric matrix
    torch.linalg.cholesky_ex(D[:2048, :2048])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    Lc, info = torch.linalg.cholesky_ex(D)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    if int(info.item()) == 0:
        out["cusolver_potrf"] = {"value": flops / t / 1e12, "unit": "TFLOP/s", "t_factor_ms": t * 1e3,
                                 "what": "torch.linalg.cholesky (cuSOLVER potrf) on the dense n x n matrix"}
    del D, Lc
    torch.cuda.empty_cache()
    return out


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
    if args.workload == "batched":
        return run_reference_batched(args, ws)
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
            "config": dict(workload_config(w, n, w.tile, ws), sample_n=ns),
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": oracle.threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def common_line(ws, args, value, t, metric_cfg, dtype):
    return {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic", "impl": "ours",
            "config": metric_cfg}


def fp64_roofline(upd_flops, upd_ms, t):
    pk, pk_kind = peaks()
    fp64_peak = NSM * FP64_FLOPS_PER_CLK_SM * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    achieved = (upd_flops / (upd_ms / 1e3) / 1e12) if upd_ms > 0 else None
    return {"kernel": "k_dgemm_update", "bound": "alu", "achieved": achieved, "peak": round(fp64_peak, 4),
            "unit": "TFLOP/s", "frac": (achieved / fp64_peak) if achieved else None, "traffic": None,
            "peak_source": f"ALU: 152 SMs x 4 FP64 flop/clk x {pk_kind} max SM clock",
            "update_share_of_step": (upd_ms / 1e3) / t if t > 0 else None}


def zgemm_roofline(upd_flops, upd_ms, t):
    """Emulated FP64 update: 105 E4M3 plane-pair products per FP64 product, so the tensor work
    is 105 x the algorithmic flops; the roofline is the FP8 dense peak (measured BF16 x the
    nominal FP8/BF16 ratio 2), reported both as executed and as algorithmic FP64 flops."""
    pk, pk_kind = peaks()
    fp8_peak = (pk.get("bf16_tflops_sustained") or pk["bf16_tflops"]) * 2.0
    alg = (upd_flops / (upd_ms / 1e3) / 1e12) if upd_ms > 0 else None
    executed = alg * 105 if alg else None
    return {"kernel": "k_zgemm", "bound": "tensor", "achieved": executed, "peak": fp8_peak, "unit": "TFLOP/s",
            "frac": (executed / fp8_peak) if executed else None, "traffic": None,
            "peak_source": f"{pk_kind} bf16 sustained x nominal fp8/bf16 ratio 2",
            "algorithmic_fp64_tflops": alg, "pairs_per_fp64_product": 105,
            "update_share_of_step": (upd_ms / 1e3) / t if t > 0 else None}


def max_over_ranks(t, ws, dev):
    if ws == 1:
        return t
    import torch
    import torch.distributed as dist
    tt = torch.tensor([t], device=dev, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


# --------------------------------------------------------------------------- batched
def run_batched(args, ws, rank, local):
    """Many uneven SPD Matern matrices (n log-uniform in [64, 4096], range U[0.02, 0.2], nu in
    {1/2, 3/2, 5/2}, nugget 1e-4): per-matrix precision maps (FP64 diagonal, FP16/FP8 off-diagonal
    where the criterion at eps_high = 1e-7 allows, FP64 elsewhere), one graph-replayed batched
    factorization, 16-RHS solves refined to backward error <= 1e-13, log-likelihoods.  The tile
    size and the FP64 update engine come from the autotuner (timed on this batch)."""
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2410_09819_gb300 import autotune
    from paper_2410_09819_gb300 import tile_chol as tc

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    Hgen = tc.Handle(local, stream=stream.cuda_stream)
    bw = inputs.batched_workload(args.count, 5 + 1000 * rank)
    ns = bw.ns
    pts = [torch.from_numpy(bw.points(i)).to(dev) for i in range(len(ns))]
    eps, nrhs = 1e-7, bw.nrhs

    map_store = {}

    def make_inputs(b):
        A_list = []
        sizes = [tc.ntiles(n, b) ** 2 for n in ns]
        flat = torch.zeros(sum(sizes), dtype=torch.uint8, device=dev)
        map_store[b] = flat
        maps = list(torch.split(flat, sizes))
        for i, n in enumerate(ns):
            A = torch.empty(tc.tile_count(n, b) * b * b, dtype=torch.float64, device=dev)
            tc.tc_matern_tiles(Hgen.h, n, b, pts[i], 1.0, bw.ranges[i], bw.nus[i], 1e-4, A)
            A_list.append(A)
        return A_list, maps

    def compute_maps(A_list, maps, b):
        for i, n in enumerate(ns):
            tc.tile_chol_precision_map_noalloc(n, b, A_list[i], eps, 0, 4, maps[i], stream.cuda_stream)
        flat = map_store[b]
        flat[flat == tc.TC_FP32] = tc.TC_FP64

    def make_handle(mode):
        return tc.Handle(local, stream=stream.cuda_stream, fp64_mode=mode, fp32_updates=args.fp32_updates)

    (b, mode), tune = autotune.pick_batched_config(make_handle, ns, make_inputs)
    H = make_handle(mode)
    A_list, maps = make_inputs(b)
    Bh = [inputs.gaussian(n, nrhs, 77 + i) for i, n in enumerate(ns)]
    B = [torch.from_numpy(np.ascontiguousarray(x.T)).to(dev) for x in Bh]
    X = [torch.empty_like(x) for x in B]
    Y = [x[0].contiguous() for x in B]
    flops = sum(n ** 3 / 3.0 for n in ns)

    def step(A_in, maps_in, B_in, X_in, Y_in, make_maps=True):
        st, ss = tc.tc_stats(), tc.tc_stats()
        if make_maps:
            compute_maps(A_in, maps_in, b)
        rc, info, ld = tc.tile_chol_factor_batched(H.h, ns, b, A_in, maps_in, st)
        if rc:
            raise RuntimeError(f"batched factorization failed: {rc}")
        berr = tc.tile_chol_solve_batched(H.h, nrhs, B_in, X_in, 10, 1e-13, ss)
        ll = tc.tile_chol_loglik_batched(H.h, Y_in)
        return st, ss, berr, ll

    # kernels of one factorization: counted while the graph is captured (replays count none)
    st0 = tc.tc_stats()
    compute_maps(A_list, maps, b)
    tc.tile_chol_factor_batched(H.h, ns, b, A_list, maps, st0)
    factor_kernels = st0.kernel_launches
    tensor_flops = sum(st0.tensor_flops)
    for _ in range(args.warmup):
        step(A_list, maps, B, X, Y)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    launches = 0
    t_factor = 0.0
    for _ in range(args.steps):
        st, ss, berr, ll = step(A_list, maps, B, X, Y)
        launches += factor_kernels + 2 * len(ns) + ss.kernel_launches     # maps + factor + solves
        t_factor += st.t_ms
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    t = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, ws, dev)
    value = ws * flops * args.steps / t / 1e12
    nlow = sum(int((m > 1).sum().item()) for m in maps)

    # roofline: the whole graph-replayed factorization against the E4M3 dense peak -- its tensor
    # work (digit planes of the FP64 tiles, FP16 / FP8 tiles) over its wall time; the launches
    # of hundreds of small matrices, not the tensor pipe, bound it
    pk, pk_kind = peaks()
    bf16 = pk.get("bf16_tflops_sustained") or pk["bf16_tflops"]
    t_f = t_factor / args.steps / 1e3
    roofline = None
    if tensor_flops > 0 and t_f > 0:
        ach = tensor_flops / t_f / 1e12
        roofline = {"kernel": "batched factorization (graph of grouped k_zgemm / k_qgemm / POTRF / TRSM launches)",
                    "bound": "tensor", "achieved": ach, "peak": bf16 * 2.0, "unit": "TFLOP/s",
                    "frac": ach / (bf16 * 2.0), "traffic": None,
                    "peak_source": f"{pk_kind} bf16 sustained x nominal e4m3/bf16 ratio 2",
                    "algorithmic_tflops": flops / t_f / 1e12, "t_factor_ms": t_f * 1e3,
                    "kernels_per_factorization": factor_kernels,
                    "us_per_kernel": t_f * 1e6 / max(1, factor_kernels)}
    elif t_f > 0:
        fp64_peak = NSM * FP64_FLOPS_PER_CLK_SM * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        ach = flops / t_f / 1e12
        roofline = {"kernel": "batched factorization (FP64 pipe)", "bound": "alu", "achieved": ach,
                    "peak": fp64_peak, "unit": "TFLOP/s", "frac": ach / fp64_peak, "traffic": None,
                    "peak_source": f"ALU: 152 SMs x 4 FP64 flop/clk x {pk_kind} max SM clock",
                    "kernels_per_factorization": factor_kernels}

    # end to end: the same step from pinned host buffers (the library stages the matrices and
    # right-hand sides; solutions and log-likelihoods come back to host memory)
    e2e = None
    if not args.no_e2e:
        Ah = [a.cpu().pin_memory() for a in A_list]
        mh = [m.cpu().pin_memory() for m in maps]
        Bp = [x.cpu().pin_memory() for x in B]
        Xp = [torch.empty_like(x).pin_memory() for x in Bp]
        Yp = [x.cpu().pin_memory() for x in Y]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(Ah, mh, Bp, Xp, Yp, make_maps=False)     # host maps: the ones computed on the device
        e1.record(stream)
        torch.cuda.synchronize()
        te = max(e0.elapsed_time(e1) / 1e3, time.perf_counter() - t0)
        te = max_over_ranks(te, ws, dev)
        h2d = sum(a.numel() * 8 for a in Ah) + sum(m.numel() for m in mh) + sum(x.numel() * 8 for x in Bp) + \
            sum(y.numel() * 8 for y in Yp)
        d2h = sum(x.numel() * 8 for x in Xp) + 8 * len(ns)
        e2e = {"value": ws * flops / te / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h,
               "note": "precision maps are inputs here (host copies of the device-computed ones)"}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = batched_cpu_sample(bw, 1)
    if rank == 0:
        line = common_line(ws, args, value, t, {
            "workload": "batched", "count": len(ns), "n_range": [min(ns), max(ns)], "tile": b,
            "fp64_engine": {0: "FP64 pipe (DFMA, 64 x 64 blocks)", 2: "E4M3 digit planes (128 x 64 items, mixed maps)"}[mode],
            "autotune_s": {f"b={k[0]},fp64_mode={k[1]}": v for k, v in tune.items()}, "nugget": 1e-4,
            "eps_high": eps, "precision": "FP64 diagonal, FP16/FP8 off-diagonal where allowed, else FP64",
            "nrhs": nrhs, "l2": "total inputs larger than L2", "parallelism": f"replicas x{ws}",
            "step": "maps+graph-replayed batched factor+16-RHS refined solves+logliks"}, "f64+f16+e4m3")
        line["roofline"] = roofline
        line["e2e"] = e2e
        line["cpu_baseline"] = cpu
        line["clocks"] = clk
        line["gpu_launches"] = launches
        line["detail"] = {"max_berr": max(berr), "refine_iters": ss.refine_iters, "low_precision_tiles": nlow,
                          "t_factor_ms": st.t_ms, "t_solve_ms": ss.t_ms, "flops": flops}
        print(json.dumps(line), flush=True)
    H.close()
    Hgen.close()


def batched_cpu_sample(bw, reps):
    """The oracle (plain FP64 Cholesky) on the first matrices of the batch, up to 2e10 flops."""
    import oracle
    idx, fl = [], 0.0
    for i, n in enumerate(bw.ns):
        if fl > 2e10:
            break
        idx.append(i)
        fl += n ** 3 / 3.0
    mats = [oracle.matern(bw.points(i), 1.0, bw.ranges[i], bw.nus[i], 1e-4) for i in idx]
    t0 = time.perf_counter()
    for _ in range(reps):
        for A in mats:
            oracle.cholesky(A)
    t = time.perf_counter() - t0
    return {"value": fl * reps / t / 1e12, "unit": "TFLOP/s", "cores": oracle.threads(), "kind": "oracle",
            "sample": f"first {len(idx)} matrices of the batch ({fl:.2e} flops), one oracle factorization each",
            "seconds": t}


def run_reference_batched(args, ws):
    import oracle
    bw = inputs.batched_workload(args.count, 5)
    # bounded sample: the first matrices of the batch up to ~2e10 flops
    idx, fl = [], 0.0
    for i, n in enumerate(bw.ns):
        if fl > 2e10:
            break
        idx.append(i)
        fl += n ** 3 / 3.0
    mats = [oracle.matern(bw.points(i), 1.0, bw.ranges[i], bw.nus[i], 1e-4) for i in idx]
    for _ in range(args.warmup):
        for A in mats:
            oracle.cholesky(A)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for A in mats:
            oracle.cholesky(A)
    t = time.perf_counter() - t0
    value = fl * args.steps / t / 1e12
    sample = f"first {len(idx)} matrices of the batch ({fl:.2e} flops), oracle factorization each"
    print(json.dumps({"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "impl": "reference", "config": {"workload": "batched", "count": args.count},
                      "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": oracle.threads(),
                                       "kind": "oracle", "sample": sample},
                      "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}), flush=True)


# ------------------------------------------------------------------------ out-of-core
def measure_link(dev):
    import torch
    nb = 1 << 30
    h = torch.empty(nb, dtype=torch.uint8).pin_memory()
    d = torch.empty(nb, dtype=torch.uint8, device=dev)
    best = {}
    for name, fn in (("h2d", lambda: d.copy_(h, non_blocking=True)), ("d2h", lambda: h.copy_(d, non_blocking=True))):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        best[name] = nb / min(ts) / 1e9
    del h, d
    return best


def run_ooc(args, ws, rank, local):
    """Out-of-core FP64 factorization: the tiles live in pinned host memory, the device caches at
    most OOC_CACHE_FRACTION of them (in bytes: with emulated updates a slot also holds the
    tile's digit planes, so fewer tiles fit).  Each step factors a fresh copy of A (restored, untimed,
    before the step: the factorization overwrites A with L)."""
    import torch
    import torch.distributed as dist

    from paper_2410_09819_gb300 import tile_chol as tc

    w = inputs.WORKLOADS[args.workload]
    n = args.n or 65536
    b = w.tile
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    T = tc.tile_count(n, b)
    cap = int(inputs.OOC_CACHE_FRACTION * T * b * b * 8)
    from paper_2410_09819_gb300.ooc_sim import POLICIES, simulate, slots_for_cap
    H = tc.Handle(local, stream=stream.cuda_stream, device_cap_bytes=cap, fp64_mode=args.fp64_mode,
                  ooc=POLICIES.index(args.ooc_policy), ooc_eviction=1 if args.ooc_eviction == "min" else 0)
    link = measure_link(dev)
    pts = inputs.uniform_points(n, w.seed + 1000 * rank, w.morton)
    host0 = torch.empty(T * b * b, dtype=torch.float64, pin_memory=True)
    # generate on the device tile-row by tile-row is not needed: n = 65536 fits; generate and move
    A = torch.empty(T * b * b, dtype=torch.float64, device=dev)
    tc.tc_matern_tiles(H.h, n, b, torch.from_numpy(pts).to(dev), w.sigma2, w.range_a, w.nu, w.nugget, A)
    nt = tc.ntiles(n, b)
    pmap = None
    if args.ooc_mxp:
        # four-precision map from the tile-norm criterion (computed once; the matrix is fixed)
        pmap = torch.zeros(nt * nt, dtype=torch.uint8)
        tc.tile_chol_precision_map(H.h, n, b, A, OOC_MXP_EPS, OOC_MXP_BAND, 4, pmap)
    host0.copy_(A)
    del A
    torch.cuda.empty_cache()
    work = torch.empty_like(host0).pin_memory()
    y = torch.from_numpy(inputs.gaussian(n, 1, 9)[:, 0].copy()).pin_memory()
    x = torch.empty_like(y).pin_memory()

    def step(timed):
        work.copy_(host0)                    # restore A (the factor overwrites it), untimed
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st, ss = tc.tc_stats(), tc.tc_stats()
        e0.record(stream)
        info = tc.tile_chol_factor_ooc(H.h, n, b, work, pmap, st)
        if info:
            raise RuntimeError(f"ooc factorization failed at column {info}")
        tc.tile_chol_solve(H.h, 1, y, n, x, n, 0, 0.0, ss)
        ll = tc.tile_chol_loglik(H.h, y)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3, st, ss, ll

    for _ in range(args.warmup):
        step(False)
    if ws > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    t = 0.0
    for _ in range(args.steps):
        dt, st, ss, ll = step(True)
        t += dt
    clk = clocks.stop()
    t = max_over_ranks(t, ws, dev)
    flops = n ** 3 / 3.0
    value = ws * flops * args.steps / t / 1e12
    h2d, d2h = st.h2d_bytes, st.d2h_bytes
    tf = st.t_ms / 1e3
    ld_run = tc.tile_chol_logdet(H.h)
    accuracy = None
    if args.ooc_mxp:
        # FP64 reference (untimed): the same matrix out of core with an all-FP64 map
        work.copy_(host0)
        s64 = tc.tc_stats()
        if tc.tile_chol_factor_ooc(H.h, n, b, work, None, s64) == 0:
            ll64 = tc.tile_chol_loglik(H.h, y)
            ld64 = tc.tile_chol_logdet(H.h)
            accuracy = {"loglik_fp64": ll64, "loglik_mxp": ll, "loglik_rel_err": abs(ll - ll64) / abs(ll64),
                        "logdet_fp64": ld64, "logdet_mxp": ld_run, "kl_divergence": 0.5 * (ld_run - ld64),
                        "fp64_ooc_h2d_bytes": s64.h2d_bytes, "fp64_ooc_t_factor_ms": s64.t_ms,
                        "reference": "same matrix, out of core, all-FP64 map"}
    if rank == 0:
        line = common_line(ws, args, value, t, {
            "workload": w.name + f"@n={n}", "n": n, "tile": b, "nu": w.nu, "range": w.range_a, "nugget": w.nugget,
            "device_cache_bytes": cap, "matrix_bytes": T * b * b * 8, "host": "pinned",
            "step": "ooc factor (A in host memory, overwritten by L)+streamed 1-RHS solve+loglik",
            "l2": "inputs larger than L2", "parallelism": f"replicas x{ws}",
            "precision": (f"per-tile map, eps_high {OOC_MXP_EPS}, FP64 band {OOC_MXP_BAND}" if args.ooc_mxp
                          else "FP64")},
            ("f64+f32+f16+e4m3" if args.ooc_mxp else
             "f64" if args.fp64_mode == 0 else "f64 (updates emulated on e4m3 tensor cores)"))
        rf = zgemm_roofline if args.fp64_mode >= 1 else fp64_roofline
        line["roofline"] = rf(st.update_flops[0], st.t_update_ms[0], tf)
        if args.fp64_mode >= 1:
            line["roofline"]["kernel"] = "k_zgemm (grouped out-of-core form)"
        line["config"]["fp64_updates"] = "emulated (E4M3 digit planes)" if args.fp64_mode >= 1 else "DFMA"
        # host-link volume of every scheduling policy at this size and cache, from the schedule
        # simulator (which the tests hold equal to the library's counters)
        emu = args.fp64_mode >= 1
        ns = slots_for_cap(cap, n, b, emulated=emu, mixed=args.ooc_mxp)
        pm2 = pmap.numpy().reshape(nt, nt) if pmap is not None else None
        predicted = {}
        for pol in POLICIES:
            r = simulate(n, b, ns, emulated=emu, pmap=pm2, policy=pol)
            predicted[pol] = {"h2d_bytes": r.h2d_bytes, "d2h_bytes": r.d2h_bytes}
        r = simulate(n, b, ns, emulated=emu, pmap=pm2, policy="V3", eviction="min")
        predicted["V3_belady_min"] = {"h2d_bytes": r.h2d_bytes, "d2h_bytes": r.d2h_bytes,
                                      "note": "offline-optimal eviction over the same requests"}
        line["ooc_policy"] = args.ooc_policy
        line["ooc_eviction"] = args.ooc_eviction
        line["ooc_link"] = {"h2d_bytes": h2d, "d2h_bytes": d2h, "h2d_gbs": h2d / tf / 1e9, "d2h_gbs": d2h / tf / 1e9,
                            "policy_volumes_predicted": predicted,
                            "link_peak_gbs": link, "h2d_frac": (h2d / tf / 1e9) / link["h2d"],
                            "cache_hits": st.cache_hits, "cache_misses": st.cache_misses,
                            "evictions": st.evictions, "solve_h2d_note": "solve streams the factor again"}
        line["e2e"] = {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                       "note": "the matrix is host-resident by construction: the device-timed step is end to end"}
        line["cpu_baseline"] = None
        line["clocks"] = clk
        line["gpu_launches"] = st.kernel_launches + ss.kernel_launches
        line["detail"] = {"t_factor_ms": st.t_ms, "t_update_ms": list(st.t_update_ms), "t_trsm_ms": st.t_trsm_ms,
                          "t_potrf_ms": st.t_potrf_ms, "t_convert_ms": st.t_convert_ms, "loglik": ll,
                          "update_launches": list(st.update_launches), "tiles_by_prec": list(st.tiles),
                          "update_tflops_by_prec": [st.update_flops[p] / st.t_update_ms[p] / 1e9
                                                    if st.t_update_ms[p] > 0 else None for p in range(4)]}
        line["accuracy"] = accuracy
        print(json.dumps(line), flush=True)
    H.close()


def run_sweep(args, local):
    """Section V's accuracy study on this library: for each theta set (weak, medium, strong
    correlation) the FP64 factor as reference, then the four-precision factor at each accuracy
    level: log-likelihood (y from the generator), log-determinant, KL divergence (Eq. 3 at
    y = 0), precision mix and factorization TFLOP/s (one timed run after one warm-up)."""
    import torch

    from paper_2410_09819_gb300 import tile_chol as tc
    n = args.n or 65536
    b = 1024 if n >= 16384 else 256
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    nt = tc.ntiles(n, b)
    T = tc.tile_count(n, b)
    out = {"metric": "Section V sweep: KL divergence, log-likelihood error and TFLOP/s vs accuracy level",
           "n": n, "tile": b, "band": 2, "nugget": 1e-6, "points": "seeded uniform in [0,1]^2, Morton-sorted",
           "fp64_mode": args.fp64_mode, "fp32_updates": args.fp32_updates, "rows": []}
    pts = torch.from_numpy(inputs.uniform_points(n, 7, True)).to(dev)
    y = torch.from_numpy(inputs.gaussian(n, 1, 11)[:, 0].copy()).to(dev)
    A = torch.empty(T * b * b, dtype=torch.float64, device=dev)
    pm = torch.zeros(nt * nt, dtype=torch.uint8)
    with tc.Handle(local, stream=stream.cuda_stream, fp64_mode=args.fp64_mode, fp32_updates=args.fp32_updates) as H:
        for name, (s2, beta, nu) in inputs.THETA_SETS.items():
            tc.tc_matern_tiles(H.h, n, b, pts, s2, beta, nu, 1e-6, A)
            st = tc.tc_stats()
            tc.tile_chol_factor(H.h, n, b, A, None, st)
            ld64, ll64 = tc.tile_chol_logdet(H.h), tc.tile_chol_loglik(H.h, y)
            row = {"theta": name, "sigma2": s2, "beta": beta, "nu": nu,
                   "fp64": {"tflops": n ** 3 / 3 / (st.t_ms / 1e3) / 1e12, "logdet": ld64, "loglik": ll64}, "levels": []}
            for eps in inputs.SWEEP_EPS:
                tc.tile_chol_precision_map(H.h, n, b, A, eps, 2, 4, pm)
                tc.tile_chol_factor(H.h, n, b, A, pm, None)          # warm-up (plan, pools)
                st = tc.tc_stats()
                info = tc.tile_chol_factor(H.h, n, b, A, pm, st)
                if info:
                    row["levels"].append({"eps_high": eps, "info": info, "tiles_by_prec": list(st.tiles),
                                          "note": "the low-precision factor lost positive definiteness"})
                    continue
                ld, ll = tc.tile_chol_logdet(H.h), tc.tile_chol_loglik(H.h, y)
                row["levels"].append({"eps_high": eps, "tflops": n ** 3 / 3 / (st.t_ms / 1e3) / 1e12,
                                      "tiles_by_prec": list(st.tiles), "kl_divergence": 0.5 * (ld - ld64),
                                      "loglik_rel_err": abs(ll - ll64) / abs(ll64), "logdet": ld})
            out["rows"].append(row)
    print(json.dumps(out), flush=True)


def run_peaks(local):
    """Dense GEMM peaks of this GPU through cuBLAS (torch.matmul, torch._scaled_mm for E4M3),
    8192^3 (2 N^3 flops): best of 10 launches (burst) and back to back for 4 s (sustained),
    CUDA events on the launching stream; pinned 1 GiB host<->device copies.  The rooflines
    of the update kernels compare against these and against the driver's BF16 measurement."""
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    N = 8192
    out = {"metric": "dense GEMM peaks (TFLOP/s) and pinned host-link rates (GB/s)", "n": N,
           "gpu": torch.cuda.get_device_name(dev), "torch": torch.__version__}
    torch.backends.cuda.matmul.allow_tf32 = True

    def timed(fn, flops):
        fn()
        torch.cuda.synchronize()
        best = 0.0
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            best = max(best, flops / (e0.elapsed_time(e1) / 1e3) / 1e12)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps, t0 = 0, time.perf_counter()
        e0.record()
        while time.perf_counter() - t0 < 4.0:
            for _ in range(8):
                fn()
            reps += 8
            torch.cuda.synchronize()
        e1.record()
        torch.cuda.synchronize()
        return {"burst": best, "sustained": flops * reps / (e0.elapsed_time(e1) / 1e3) / 1e12}

    flops = 2.0 * N ** 3
    clk = ClockSampler(local)
    clk.start()
    for name, dt in (("bf16", torch.bfloat16), ("fp16", torch.float16), ("tf32", torch.float32),
                     ("fp64", torch.float64)):
        a = torch.randn(N, N, device=dev, dtype=torch.float32).to(dt)
        bm = torch.randn(N, N, device=dev, dtype=torch.float32).to(dt)
        out[name] = timed(lambda: torch.matmul(a, bm), flops)
        del a, bm
        torch.cuda.empty_cache()
    try:
        a8 = torch.randn(N, N, device=dev).to(torch.float8_e4m3fn)
        b8 = torch.randn(N, N, device=dev).to(torch.float8_e4m3fn)
        one = torch.ones((), device=dev, dtype=torch.float32)
        out["e4m3"] = timed(lambda: torch._scaled_mm(a8, b8.t(), scale_a=one, scale_b=one,
                                                     out_dtype=torch.bfloat16), flops)
        del a8, b8
    except (RuntimeError, TypeError, AttributeError) as exc:       # pragma: no cover - torch API
        out["e4m3"] = {"error": str(exc)[:200]}
    out["clocks"] = clk.stop()
    out["link_gbs"] = measure_link(dev)
    print(json.dumps(out), flush=True)


def main():
    args = parse_args()
    ws, rank, local = dist_info()
    if args.peaks:
        run_peaks(local)
        return
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.sweep:
        run_sweep(args, local)
        return
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    try:
        if args.workload == "batched":
            run_batched(args, ws, rank, local)
        elif args.workload.startswith("ooc"):
            run_ooc(args, ws, rank, local)
        else:
            run_ours(args, ws, rank, local)
    finally:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
