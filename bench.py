#!/usr/bin/env python
"""Benchmark of the PowerLU hot path (Zhang & Mascagni, arXiv 2002.07138) on GB300.

One step = one fixed-rank PowerLU call (Alg. bpowerlu with Alg. gpowerlu:
Gaussian sketch, v passes over A, LU re-orthogonalisation, QR, final pass,
two LUs and the tail products) through the C ABI, on a seeded synthetic A
already resident in HBM.  Default workload: the mixed-precision one, m = n =
32768, A stored in FP32 (4.3 GB, larger than L2, so no flush is needed
between steps), sigma_i = i^-1.5, k = 256, l = 276, v = 3, passes on TF32
tensor cores; the BF16 and FP8-E4M3 passes are reported beside it.
--workload fixed_rank_8192 runs the 8192^2 FP32 workload, batched_512 the
batch of 512 problems, sparse_32000 PowerLU on a 32000^2 sprand-like matrix
at 0.3% density (FP64 sparse passes; Sec. 6, l = 200).

value = algorithmic pass flops (2 m n l per power pass + 2 m n k for the
last pass) over the whole call time, in TFLOP/s, summed over ranks.
Also reported: ms per pass and TFLOP/s per pass from the pass kernels alone,
the relative Frobenius error, the same call with FP64 passes ("FP64 plain"),
an end-to-end number through host buffers, the roofline of the dominant
kernel (timed live with CUDA events) and the FP64 CPU oracle timed on the
host cores.

--impl reference times the oracle (the plain FP64 CPU implementation of the
paper's algorithms) on the host cores on the same workload and metric.
Multi-GPU (torchrun): replicas only -- every rank factors its own matrix,
no data-path collective; value sums the ranks' work over the slowest rank.
"""
import argparse
import collections
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PowerLU ms & TFLOP/s per pass of A at stated rel. error, mixed vs FP64 plain"

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from
# one ncu capture of the kernel as it stands, keyed by (kernel, workload,
# precision); absent: null.  The 32768^2 entries scale the 16384^2 captures
# by the bytes the kernel streams (A: x4, the m x l panel: x2).
TRAFFIC = {
    # profiles/k_panel_lu_la_mixed_16384.md: 36.25 MB read + 0.10 MB written
    ("k_panel_lu_la", "mixed_32768_k256_l276_v3", "tf32"): 2 * (36.252e6 + 0.100e6),
    ("k_panel_lu_la", "mixed_16384_k256_l276_v3", "tf32"): 36.252e6 + 0.100e6,
    # profiles/k_tc_pass_mixed_16384_tf32.md: mean of the two orientations
    ("k_tc_pass", "mixed_32768_k256_l276_v3", "tf32"): 4 * (1.0927e9 + 0.0071e9),
    ("k_tc_pass", "mixed_16384_k256_l276_v3", "tf32"): 1.0927e9 + 0.0071e9,
}


def workloads():
    import synth
    return {"fixed_rank_8192": synth.FIXED_RANK_8192, "mixed_32768": synth.MIXED_32768,
            "mixed_16384": synth.MIXED_16384,
            "fixed_prec_20000x10000": synth.FIXED_PREC_20000x10000,
            "plain_2000x1500": synth.PLAIN_2000x1500, "batched_512": None,
            "sparse_32000": None}


def batch_specs(count=512, seed=0):
    """The batched workload: sizes from synth.batched_problems; every 8th
    problem runs the single-pass algorithm, the others PowerLU (v = 2, 3)."""
    import synth
    specs = synth.batched_problems(count, seed)
    for i, sp in enumerate(specs):
        sp["algo"] = 1 if i % 8 == 7 else 0
    return specs


def batch_flops(specs):
    f = 0.0
    for sp in specs:
        if sp["algo"] == 1:
            f += 4.0 * sp["m"] * sp["n"] * sp["k"]
        else:
            f += 2.0 * sp["m"] * sp["n"] * (sp["l"] * (sp["v"] - 1) + sp["k"])
    return f


def build_batch(specs, device, dtype):
    import numpy as np
    import torch
    import synth
    mats = []
    for sp in specs:
        sig = synth.sigma_profile("expk", min(sp["m"], sp["n"]), k=sp["k"])
        mats.append(synth.svd_matrix_torch(sp["m"], sp["n"], sig, sp["seed"], device=device,
                                           dtype=dtype))
    return mats


def run_batched(args):
    import numpy as np
    import torch
    import paper_2002_07138_gb300 as plu
    import oracle

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    specs = batch_specs(512, seed=rank)
    mats = build_batch(specs, "cuda", torch.float32)
    stream = torch.cuda.current_stream()
    ctx = plu.Context(local, stream.cuda_stream)
    probs = [dict(A=A, k=sp["k"], l=sp["l"], v=sp["v"], algo=sp["algo"], seed=sp["seed"])
             for A, sp in zip(mats, specs)]
    flops = batch_flops(specs)
    for _ in range(args.warmup):
        plu.plu_batched(ctx, probs, prec=args.prec if args.prec in ("fp32", "fp64") else "fp32")
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    dist_barrier(ws)
    graph_ms, launches, outs = [], 0, None
    t0 = time.perf_counter()
    for _ in range(args.steps):
        outs, rep = plu.plu_batched(ctx, probs, prec=args.prec if args.prec in ("fp32", "fp64") else "fp32")
        graph_ms.append(rep["ms_total"])
        launches += rep["launches"]
    torch.cuda.synchronize()
    wall_ms = 1e3 * (time.perf_counter() - t0) / args.steps
    dist_barrier(ws)
    clk = clocks.stop()
    ms = dist_max(ws, statistics.mean(graph_ms))
    value = flops * ws / (ms / 1e3) / 1e12
    hbm_peak, hbm_src = 6800.0, "fallback (6.8 TB/s)"
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)),
                               "MEASURED_PEAKS.json")) as f:
            hbm_peak, hbm_src = float(json.load(f)["hbm_gbs"]), "measured copy bandwidth"
    except (OSError, KeyError, ValueError):
        pass
    # accuracy over a sample of problems
    errs = []
    for i in range(0, len(specs), 32):
        A = mats[i].double()
        p, q, L, U = outs[i]
        errs.append(float(torch.linalg.norm(A[p.long()][:, q.long()] - L @ U) / torch.linalg.norm(A)))
    cpu = None
    if rank == 0 and not args.skip_cpu:
        t_or = 0.0
        f_or = 0.0
        for i in range(0, 64, 4):
            sp = specs[i]
            Ah = mats[i].double().cpu().numpy()
            t1 = time.perf_counter()
            if sp["algo"] == 1:
                oracle.singlepass(Ah, sp["k"], seed=sp["seed"])
            else:
                oracle.powerlu(Ah, sp["k"], sp["l"], sp["v"], seed=sp["seed"])
            t_or += time.perf_counter() - t1
            f_or += batch_flops([sp])
        cpu = {"value": f_or / t_or / 1e12, "unit": "TFLOP/s", "cores": os.cpu_count(),
               "kind": "oracle", "sample": "16 of the 512 problems (every 4th of the first 64), "
               "%.1f s" % t_or}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.prec != "fp64" else "f64", "data": "synthetic",
            "config": {"workload": "batched_512", "problems": len(specs),
                       "sum_mn": int(sum(sp["m"] * sp["n"] for sp in specs)),
                       "single_pass_problems": int(sum(sp["algo"] for sp in specs)),
                       "pass_precision": "fp32" if args.prec != "fp64" else "fp64",
                       "between_passes": "f64", "l2_flush": "inputs larger than L2",
                       "parallelism": "replicas" if ws > 1 else "single"},
            "wall_ms_per_step": wall_ms,
            "rel_error_sample_max": max(errs), "rel_error_sample_median": statistics.median(errs),
            "gemm_tiles_autotuned": dict(collections.Counter(
                "%dx%d" % t for t in plu.plu_batched_tiles(ctx))),
            "gemm_splitk_autotuned": dict(collections.Counter(
                ("k%d" % kc) if kc else "none" for kc in plu.plu_batched_splitk(ctx))),
            "gpu_launches": launches,
            "clocks": clk,
            # the batch as a whole: the passes' algorithmic bytes (every read of
            # every A) over the graph time, against the measured copy bandwidth
            "roofline": {"bound": "hbm", "achieved": rep["bytes_passes"] / (ms / 1e3) / 1e9,
                         "peak": hbm_peak, "unit": "GB/s",
                         "frac": rep["bytes_passes"] / (ms / 1e3) / 1e9 / hbm_peak,
                         "traffic": None, "peak_source": hbm_src,
                         "kernel": "whole batch graph (the FP64 LUs and CholeskyQR products "
                                   "between the passes bound it, not HBM)"},
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    ctx.close()
    return 0


def pass_flops(m, n, k, l, v):
    return 2.0 * m * n * l * (v - 1) + 2.0 * m * n * k


def panel_kernel_name(rows, cols, sms):
    """The panel LU kernel the library picks for a rows x cols panel (the
    look-ahead kernel when its shared memory fits, as in launch_panel_lu)."""
    nb = min(sms, (rows + 31) // 32, 1024)
    per = -(-rows // nb)
    smem_la = 2 * 32 * per * 8 + 32 * cols * 8 + 32 * 32 * 8 + 2 * per * 4 + 32 * 4 + 64
    return "k_panel_lu_la" if cols > 32 and smem_la <= 210 * 1024 else "k_panel_lu_blocked"


def lu_flops(rows, cols):
    # sum_j 2 (rows - j - 1)(cols - j - 1) + (rows - j - 1) divisions, FP64
    return sum(2.0 * (rows - j - 1) * (cols - j - 1) + (rows - j - 1) for j in range(cols))


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ distributed
def replica_workload(w, rank):
    """Replicas only: rank r factors its own matrix, the workload's recipe
    with seed + r (no data-path collective between ranks)."""
    from dataclasses import replace
    return replace(w, seed=w.seed + rank)


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo")
    return ws, rank, local


def dist_barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def dist_max(ws, x):
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------- reference
def oracle_call(A, w, seed):
    import oracle
    t0 = time.perf_counter()
    p, q, L, U = oracle.powerlu(A, w.k, w.l, w.v, seed=seed)
    return time.perf_counter() - t0, (p, q, L, U)


FULL_ORACLE_MAX_MN = 1 << 27          # larger workloads time a bounded sample


def oracle_sample(A, w, seed):
    """Time the oracle on a bounded sample of the workload: the whole call
    when A is small, otherwise the first pass of Alg. gpowerlu (A^T Omega or
    A Omega) and the LU re-orthogonalisation of its result.  Returns
    (seconds, pass flops of the sample, description)."""
    import oracle
    m, n = A.shape
    if m * n <= FULL_ORACLE_MAX_MN:
        dt, _ = oracle_call(A, w, seed)
        return dt, pass_flops(m, n, w.k, w.l, w.v), "one full oracle PowerLU call"
    t0 = time.perf_counter()
    if w.v % 2 == 0:
        Om = oracle.gaussian_matrix(m, w.l, seed, oracle.STREAM_OMEGA_M)
        Y = A.T @ Om
    else:
        Om = oracle.gaussian_matrix(n, w.l, seed, oracle.STREAM_OMEGA_N)
        Y = A @ Om
    oracle.lu_permuted_L(Y)
    dt = time.perf_counter() - t0
    return dt, 2.0 * m * n * w.l, ("the oracle's first pass of Alg. gpowerlu (one FP64 product "
                                   "with A) and its LU re-orthogonalisation")


def build_host_matrix(w, seed_offset=0):
    """The workload's A as a float64 numpy array (built on the GPU when one is
    present, then copied; otherwise with numpy)."""
    import numpy as np
    try:
        import torch
        if torch.cuda.is_available():
            from dataclasses import replace
            Ad = replace(w, seed=w.seed + seed_offset).build("cuda")
            A = Ad.double().cpu().numpy()
            del Ad
            torch.cuda.empty_cache()
            return np.asfortranarray(A)
    except Exception:
        pass
    from dataclasses import replace
    A = replace(w, seed=w.seed + seed_offset).build("cpu")
    return np.asfortranarray(A.astype(np.float64))


def run_reference(args, w):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return 0
    A = build_host_matrix(w)
    for i in range(args.warmup):
        oracle_sample(A, w, seed=i)
    times = []
    for i in range(args.steps):
        dt, flops, desc = oracle_sample(A, w, seed=i)
        times.append(dt)
    total = sum(times)
    value = flops * args.steps / total / 1e12
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "m": w.m, "n": w.n, "k": w.k, "l": w.l, "v": w.v,
                   "storage": "f64 (host)", "l2_flush": "inputs larger than L2"},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": desc + " per step, on the same matrix"},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ ours
def time_calls(torch, fn, reps, stream):
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    fn()
    torch.cuda.synchronize()
    s.record(stream)
    for _ in range(reps):
        fn()
    e.record(stream)
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


def measure_peaks(torch, plu, ctx, stream, device):
    """The compute ceilings the rooflines divide by, measured here outside the
    timed region (best of several runs, CUDA events), with the SM clock
    sampled meanwhile: FP64 (torch.matmul 4096^3 and the library's own FP64
    GEMM, one 16384^2 x 256 pass), TF32 (torch.matmul 8192^3 with TF32
    allowed) and FP8-E4M3 (torch._scaled_mm 8192^3, when torch has it)."""
    out = {}
    clocks = ClockSampler(device)
    clocks.start()
    time.sleep(0.2)

    def best(fn, reps):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            s0 = torch.cuda.Event(enable_timing=True)
            s1 = torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            fn()
            s1.record(stream)
            torch.cuda.synchronize()
            ts.append(s0.elapsed_time(s1))
        return min(ts)

    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    out["fp64_torch_tflops"] = 2.0 * n ** 3 / best(lambda: a @ b, 5) / 1e9
    del a, b
    m2, c2 = 16384, 256
    A64 = plu.colmajor_empty(m2, m2, dtype=torch.float64)
    A64.normal_()
    X64 = plu.colmajor_empty(m2, c2, dtype=torch.float64)
    X64.normal_()
    Y64 = plu.colmajor_empty(m2, c2, dtype=torch.float64)
    out["fp64_own_gemm_tflops"] = 2.0 * m2 * m2 * c2 / best(
        lambda: plu.plu_pass(ctx, A64, 1, X64, "fp64", out=Y64), 3) / 1e9
    del A64, X64, Y64
    n = 8192
    old_tf32 = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    a = torch.randn(n, n, dtype=torch.float32, device="cuda")
    b = torch.randn(n, n, dtype=torch.float32, device="cuda")
    out["tf32_tflops"] = 2.0 * n ** 3 / best(lambda: a @ b, 10) / 1e9
    torch.backends.cuda.matmul.allow_tf32 = old_tf32
    del a, b
    try:
        a8 = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn)
        b8 = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn).t()
        one = torch.ones((), device="cuda")
        out["fp8_tflops"] = 2.0 * n ** 3 / best(
            lambda: torch._scaled_mm(a8, b8, scale_a=one, scale_b=one, out_dtype=torch.bfloat16),
            10) / 1e9
        del a8, b8
    except Exception as exc:                                   # torch without FP8 GEMM
        out["fp8_tflops"] = None
        out["fp8_note"] = "torch._scaled_mm unavailable: %s" % type(exc).__name__
    torch.cuda.empty_cache()
    out["clocks"] = clocks.stop()
    out["how"] = ("best of 3-10 runs with CUDA events; FP64: torch.matmul 4096^3 and the "
                  "library's FP64 pass (16384^2 x 256); TF32: torch.matmul 8192^3; "
                  "FP8-E4M3: torch._scaled_mm 8192^3")
    out["fp64_tflops"] = max(out["fp64_torch_tflops"], out["fp64_own_gemm_tflops"])
    return out


def leaf_flops(rows, w):
    """FP64 flops of one 32-column leaf of the tensor-core panel LU: the
    elimination inside the leaf, sum_j 2 (rows - j - 1)(w - j - 1)."""
    return sum(2.0 * (rows - j - 1) * (w - j - 1) for j in range(w))


def kernel_rooflines(torch, plu, ctx, Ad, w, prec, stream, peaks):
    """Time each step's kernels alone, at the sizes one call uses, with CUDA
    events on the library's stream.  Returns {name: (ms per launch, launches
    per call, roofline, kernel)}."""
    m, n, k, l, v = w.m, w.n, w.k, w.l, w.v
    X = plu.colmajor_empty(n, l)
    X.normal_()
    Z = plu.colmajor_empty(m, l)
    Z.normal_()
    out = {}
    sm_clock_ghz = peaks["sm_max_mhz"] / 1e3
    fp32_alu = 152 * 128 * 2 * sm_clock_ghz * 1e9 / 1e12          # TFLOP/s
    if peaks.get("fp64_tflops"):
        fp64 = {"bound": "alu", "peak": peaks["fp64_tflops"], "unit": "TFLOP/s",
                "peak_source": "measured FP64 GEMM (of measured, peaks_measured)"}
    else:
        fp64 = {"bound": "alu", "peak": 1.25, "unit": "TFLOP/s",
                "peak_source": "nominal FP64 1.25 TFLOP/s (no measured FP64 peak)"}

    # the passes: A X (trans 0) and A^T X (trans 1) over the l-wide basis
    abytes = m * n * Ad.element_size()
    ms0 = time_calls(torch, lambda: plu.plu_pass(ctx, Ad, 0, X, prec, out=Z), 5, stream)
    ms1 = time_calls(torch, lambda: plu.plu_pass(ctx, Ad, 1, Z, prec, out=X), 5, stream)
    ms = 0.5 * (ms0 + ms1)
    fl = 2.0 * m * n * l
    if prec == "fp64":
        rf = dict(fp64, achieved=fl / ms / 1e9)
    elif prec == "fp32":
        rf = {"bound": "alu", "achieved": fl / ms / 1e9, "peak": fp32_alu, "unit": "TFLOP/s",
              "peak_source": "152 SMs x 128 FP32 lanes x 2 x %.0f MHz" % peaks["sm_max_mhz"]}
    else:
        rf = {"bound": "hbm", "achieved": abytes / ms / 1e6, "peak": peaks["hbm_gbs"],
              "unit": "GB/s", "peak_source": "measured copy bandwidth"}
    rf["ms_trans0"] = ms0
    rf["ms_trans1"] = ms1
    kname = "k_tc_pass" if prec in ("tf32", "bf16", "fp8") else "k_gemm_simt"
    out["pass"] = (ms, v, rf, kname)
    # re-orthogonalising LU of the m x l panel, as the call runs it (the tail's
    # two getrf of m x k and n x k panels run the same kernels).  In the mixed
    # modes the trailing updates run on the tensor cores and the 32-column
    # leaves (k_lu_leaf) carry the FP64 work and the column-step exchanges:
    # their roofline is the FP64 pipe, timed on an m x 32 panel (one leaf).
    tc_lu = prec != "fp64"
    ctx.set_lu_updates(1 if tc_lu else 0)
    Zc = Z.clone()
    ms = time_calls(torch, lambda: (Zc.copy_(Z), plu.plu_lu_reorth(ctx, Zc)), 3, stream)
    ms_copy = time_calls(torch, lambda: Zc.copy_(Z), 3, stream)
    ms = max(ms - ms_copy, 1e-6)
    if tc_lu:
        Z32 = Z[:, :32].clone()
        Zc32 = Z32.clone()
        ms_leaf = time_calls(torch, lambda: (Zc32.copy_(Z32), plu.plu_lu_reorth(ctx, Zc32)), 5,
                             stream)
        ms_leaf = max(ms_leaf - time_calls(torch, lambda: Zc32.copy_(Z32), 5, stream), 1e-6)
        nleaf = -(-l // 32)
        rf_lu = dict(fp64, achieved=leaf_flops(m, 32) / ms_leaf / 1e9)
        rf_lu["ms_whole_lu"] = ms
        rf_lu["fp64_equivalent_tflops_whole_lu"] = lu_flops(m, l) / ms / 1e9
        rf_lu["leaves_per_lu"] = nleaf
        rf_lu["us_per_column_step"] = 1e3 * ms_leaf / 32
        out["panel_lu"] = (ms_leaf, nleaf * (max(v - 2, 0) + 2), rf_lu, "k_lu_leaf")
        out["panel_lu_whole"] = (ms, max(v - 2, 0) + 2, dict(rf_lu), "k_lu_leaf + k_lu_update")
    else:
        out["panel_lu"] = (ms, max(v - 2, 0) + 2, dict(fp64, achieved=lu_flops(m, l) / ms / 1e9),
                           panel_kernel_name(m, l, torch.cuda.get_device_properties(0).multi_processor_count))
    ctx.set_lu_updates(-1)
    # the orthonormalisation of the n x k leading basis columns as the call runs
    # it: FP64 CholeskyQR2 in the FP64 path; in the mixed modes one round whose
    # X^T X and X R^-1 are exact slice products on the BF16 tensor cores (the
    # second round is skipped on the device for this spectrum)
    Xk = X[:, :k].clone()
    Xc = Xk.clone()
    if prec == "fp64":
        qr_call, rounds = (lambda: plu.plu_qr(ctx, Xc)), 2
        qname = "cholqr2 (k_gemm_simt FP64 + Cholesky)"
    else:
        qr_call, rounds = (lambda: plu.plu_cholqr1(ctx, Xc, tc=True)), 1
        qname = "cholqr1 (BF16 tensor-core slice products + FP64 Cholesky)"
    ms = time_calls(torch, lambda: (Xc.copy_(Xk), qr_call()), 3, stream)
    ms_copy = time_calls(torch, lambda: Xc.copy_(Xk), 3, stream)
    ms = max(ms - ms_copy, 1e-6)
    # per round: the symmetric Gram n k^2, the triangular product X R^-1 n k^2,
    # the Cholesky k^3/3 and the triangular inverse k^3/3 (FP64-equivalent flops)
    fl = rounds * (2.0 * n * k * k + 2.0 * k ** 3 / 3.0)
    out["qr"] = (ms, 1, dict(fp64, achieved=fl / ms / 1e9), qname)
    return out


def run_ours(args, w):
    import numpy as np
    import torch
    from dataclasses import replace

    import paper_2002_07138_gb300 as plu

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    device = local
    peaks = {"hbm_gbs": 6791.0, "bf16_tflops": 1934.6, "sm_max_mhz": 2070.0}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks.update(json.load(f))
    except OSError:
        peaks["source"] = "fallback"

    wr = replica_workload(w, rank)
    Ad = wr.build("cuda")                                       # column-major FP32 (or FP64)
    torch.cuda.empty_cache()                                    # drop the generator's temporaries
    stream = torch.cuda.current_stream()
    ctx = plu.Context(device, stream.cuda_stream)
    prec = args.prec
    flops = pass_flops(w.m, w.n, w.k, w.l, w.v)

    def call(seed, A=Ad, pr=prec):
        return plu.plu_powerlu(ctx, A, w.k, w.l, w.v, seed=seed, prec=pr)

    for i in range(args.warmup):
        call(i)
    torch.cuda.synchronize()
    clocks = ClockSampler(device)
    clocks.start()
    time.sleep(0.3)
    dist_barrier(ws)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    reps = []
    for i in range(args.steps):
        reps.append(call(1000 + i)[4])
    ev1.record(stream)
    torch.cuda.synchronize()
    dist_barrier(ws)
    clk = clocks.stop()
    ms_total = ev0.elapsed_time(ev1)
    ms_max = dist_max(ws, ms_total)
    value = flops * args.steps * ws / (ms_max / 1e3) / 1e12
    launches = int(sum(r["launches"] for r in reps))
    ms_pass = statistics.mean(r["ms_passes"] / r["passes"] for r in reps)

    # accuracy of one call (outside the timed region)
    def rel_error(res, A):
        p, q, L, U = res[:4]
        Ap = A.double()[p.long()][:, q.long()]
        return float(torch.linalg.norm(Ap - L @ U) / torch.linalg.norm(A.double()))

    err = rel_error(call(7), Ad)
    opt = float(np.sqrt(np.sum(w.sigma_values()[w.k:] ** 2) / np.sum(w.sigma_values() ** 2)))

    # FP64 plain: the same workload with every step in FP64
    fp64 = {}
    if not args.skip_fp64:
        A64 = synth_colmajor(Ad.double())
        call(0, A64, "fp64")
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        nrep = 2
        t0.record(stream)
        r64 = [call(2000 + i, A64, "fp64")[4] for i in range(nrep)]
        t1.record(stream)
        torch.cuda.synchronize()
        ms64 = t0.elapsed_time(t1) / nrep
        fp64 = {"ms_per_step": ms64,
                "ms_per_pass": statistics.mean(r["ms_passes"] / r["passes"] for r in r64),
                "rel_error": rel_error(call(7, A64, "fp64"), Ad),
                "tflops_per_pass": (flops / w.v) / (statistics.mean(
                    r["ms_passes"] / r["passes"] for r in r64) / 1e3) / 1e12}
        del A64

    # end to end through host buffers: H2D of A, the call, D2H of p, q, L, U
    Ah = torch.empty(Ad.shape[1], Ad.shape[0], dtype=Ad.dtype, pin_memory=True).t()
    Ah.copy_(Ad)
    Ae = plu.colmajor_empty(w.m, w.n, dtype=Ad.dtype)
    ph = torch.empty(w.m, dtype=torch.int32, pin_memory=True)
    qh = torch.empty(w.n, dtype=torch.int32, pin_memory=True)
    Lh = torch.empty(w.k, w.m, dtype=torch.float64, pin_memory=True).t()
    Uh = torch.empty(w.n, w.k, dtype=torch.float64, pin_memory=True).t()

    def e2e_step(seed):
        Ae.copy_(Ah, non_blocking=True)
        p, q, L, U, _ = call(seed, Ae)
        ph.copy_(p, non_blocking=True)
        qh.copy_(q, non_blocking=True)
        Lh.copy_(L, non_blocking=True)
        Uh.copy_(U, non_blocking=True)
        torch.cuda.synchronize()

    e2e_step(0)
    ne = max(2, min(args.steps, 5))
    t0 = time.perf_counter()
    for i in range(ne):
        e2e_step(3000 + i)
    e2e_ms = dist_max(ws, 1e3 * (time.perf_counter() - t0) / ne)
    h2d = w.m * w.n * Ad.element_size()
    d2h = 4 * (w.m + w.n) + 8 * (w.m * w.k + w.k * w.n)

    # measured compute ceilings, then the roofline of the dominant kernel
    # (timed alone, live) and of the pass
    pm = measure_peaks(torch, plu, ctx, stream, device)
    peaks["fp64_tflops"] = pm["fp64_tflops"]
    kr = kernel_rooflines(torch, plu, ctx, Ad, w, prec, stream, peaks)
    share = {name: ms * cnt for name, (ms, cnt, _, _) in kr.items()}
    dom = max((nm for nm in share if nm != "panel_lu_whole"), key=share.get)

    def roofline_of(name):
        ms_k, cnt_k, rf_k, kname = kr[name]
        rf_k = dict(rf_k)
        rf_k["frac"] = rf_k["achieved"] / rf_k["peak"]
        rf_k["traffic"] = TRAFFIC.get((kname, w.name, prec))
        rf_k["kernel"] = kname
        rf_k["ms_per_launch"] = ms_k
        rf_k["share_of_step"] = share[name] / (ms_total / args.steps)
        return rf_k

    rf = roofline_of(dom)
    rf_pass = roofline_of("pass")

    # CPU baseline: the FP64 oracle on the host cores, one call on the same A
    cpu = None
    if rank == 0 and ws == 1 and not args.skip_cpu:
        Ahost = Ad.double().cpu().numpy()
        dt, sfl, desc = oracle_sample(Ahost, w, seed=0)
        del Ahost
        cpu = {"value": sfl / dt / 1e12, "unit": "TFLOP/s", "cores": os.cpu_count(),
               "kind": "oracle", "sample": "%s (FP64, numpy BLAS) on the same %dx%d matrix, "
               "%.1f s" % (desc, w.m, w.n, dt)}
        # beside the sample: one whole oracle call on the 8192^2 fixed-rank
        # workload (k = 100, l = 110, v = 3), which fits in seconds
        w8 = workloads()["fixed_rank_8192"]
        A8 = build_host_matrix(w8)
        dt8, _ = oracle_call(A8, w8, seed=0)
        del A8
        cpu["whole_call_8192"] = {"ms_per_call": 1e3 * dt8, "unit": "ms",
                                  "tflops": pass_flops(w8.m, w8.n, w8.k, w8.l, w8.v) / dt8 / 1e12,
                                  "workload": w8.name}

    # the other mixed precisions on the same matrix (one call each)
    by_prec = {}
    if not args.skip_fp64 and Ad.dtype == torch.float32:
        for pr in ("tf32", "bf16", "fp8"):
            if pr == prec:
                continue
            call(0, Ad, pr)
            torch.cuda.synchronize()
            t0e = torch.cuda.Event(enable_timing=True)
            t1e = torch.cuda.Event(enable_timing=True)
            t0e.record(stream)
            res = call(4000, Ad, pr)
            t1e.record(stream)
            torch.cuda.synchronize()
            by_prec[pr] = {"ms_per_step": t0e.elapsed_time(t1e),
                           "ms_per_pass": res[4]["ms_passes"] / res[4]["passes"],
                           "rel_error": rel_error(res, Ad)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32", "tf32": "tf32", "bf16": "bf16",
                      "fp8": "fp8e4m3", "tf32x3": "tf32x3"}[prec], "data": "synthetic",
            "config": {"workload": w.name, "m": w.m, "n": w.n, "k": w.k, "l": w.l, "v": w.v,
                       "sigma": w.sigma, "storage": "f32" if Ad.dtype == torch.float32 else "f64",
                       "pass_precision": prec, "between_passes": "f64",
                       "l2_flush": "inputs larger than L2 (A is %.0f MB)" % (h2d / 1e6),
                       "parallelism": "replicas" if ws > 1 else "single"},
            "ms_per_pass": ms_pass,
            "tflops_per_pass": (flops / w.v) / (ms_pass / 1e3) / 1e12,
            "rel_error": err, "eckart_young_optimum": opt,
            "fp64_plain": fp64,
            "other_precisions": by_prec,
            "speedup_vs_fp64_plain": (fp64["ms_per_step"] / (ms_max / args.steps)) if fp64 else None,
            "e2e": {"value": flops * ws / (e2e_ms / 1e3) / 1e12, "unit": "TFLOP/s",
                    "ms_per_step": e2e_ms, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clk,
            "roofline": rf,
            "roofline_pass": rf_pass,
            "kernel_ms": {name: {"ms_per_launch": ms, "launches_per_step": cnt}
                          for name, (ms, cnt, _, _) in kr.items()},
            "ms_phase": {nm: statistics.mean(r["ms_phase"][nm] for r in reps)
                         for nm in reps[0]["ms_phase"]},
            "peaks_measured": pm,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    ctx.close()
    return 0


def run_fixed_precision(args, w):
    """PowerLU_FP (Alg. adaptivewithoutupdating + Alg. powerlufp) on the
    fixed-precision workload: chosen rank, relative error, time per call, in
    the requested precision and in FP64 plain."""
    import numpy as np
    import torch
    import paper_2002_07138_gb300 as plu

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    Ad = replica_workload(w, rank).build("cuda")
    torch.cuda.empty_cache()
    stream = torch.cuda.current_stream()
    ctx = plu.Context(local, stream.cuda_stream)

    def call(seed, A, pr):
        return plu.plu_powerlu_fp(ctx, A, w.eps, w.b, w.l, w.v, seed=seed, prec=pr)

    def timed(A, pr, steps, warmup):
        for i in range(warmup):
            call(i, A, pr)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(steps):
            res = call(1000 + i, A, pr)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps, res

    def rel_error(res, A):
        k, p, q, L, U = res[:5]
        Ap = A.double()[p.long()][:, q.long()]
        return float(torch.linalg.norm(Ap - L @ U) / torch.linalg.norm(A.double()))

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    dist_barrier(ws)
    ms, res = timed(Ad, args.prec, args.steps, args.warmup)
    dist_barrier(ws)
    clk = clocks.stop()
    ms = dist_max(ws, ms)
    k, met, rep_ = res[0], res[5], res[6]
    err = rel_error(res, Ad)
    flops = 2.0 * w.m * w.n * w.l * w.v            # v passes over A with l columns
    out = {}
    if not args.skip_fp64:
        A64 = synth_colmajor(Ad.double())
        ms64, r64 = timed(A64, "fp64", 2, 1)
        out = {"ms_per_step": ms64, "rank": r64[0], "rel_error": rel_error(r64, Ad),
               "tolerance_met": r64[5]}
        del A64
    sig = w.sigma_values()
    tail = np.sqrt(np.cumsum((sig ** 2)[::-1])[::-1] / np.sum(sig ** 2))
    svd_rank = int(np.argmax(tail <= w.eps))          # smallest r with ||A - A_r|| <= eps ||A||
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": flops * ws / (ms / 1e3) / 1e12, "unit": "TFLOP/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32", "tf32": "tf32", "bf16": "bf16",
                      "fp8": "fp8e4m3", "tf32x3": "tf32x3"}[args.prec], "data": "synthetic",
            "config": {"workload": w.name, "m": w.m, "n": w.n, "eps": w.eps, "b": w.b, "l": w.l,
                       "v": w.v, "sigma": w.sigma, "pass_precision": args.prec,
                       "between_passes": "f64", "parallelism": "replicas" if ws > 1 else "single"},
            "rank": k, "tolerance_met": met, "rel_error": err, "svd_rank_at_eps": svd_rank,
            "ms_per_pass": rep_["ms_passes"] / max(rep_["passes"], 1),
            "fp64_plain": out,
            "speedup_vs_fp64_plain": (out["ms_per_step"] / ms) if out else None,
            "gpu_launches": rep_["launches"], "clocks": clk,
        }))
    ctx.close()
    return 0


def run_singlepass(args, w):
    """Alg. singlepasslu (Sec. 5) on the workload at rank k: one read of A
    from HBM (column panels re-read from L2), in the requested precision and
    in FP64.  value counts the two products G = A^T Omega, H = A G."""
    import torch
    import paper_2002_07138_gb300 as plu

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    Ad = replica_workload(w, rank).build("cuda")
    torch.cuda.empty_cache()
    stream = torch.cuda.current_stream()
    ctx = plu.Context(local, stream.cuda_stream)
    prec = args.prec if args.prec in ("fp64", "fp32", "tf32", "tf32x3") else "tf32"

    def timed(A, pr, steps, warmup):
        for i in range(warmup):
            plu.plu_singlepass(ctx, A, w.k, seed=i, prec=pr)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(steps):
            res = plu.plu_singlepass(ctx, A, w.k, seed=1000 + i, prec=pr)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps, res

    def rel_error(res, A):
        p, q, L, U = res[:4]
        Ap = A.double()[p.long()][:, q.long()]
        return float(torch.linalg.norm(Ap - L @ U) / torch.linalg.norm(A.double()))

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    dist_barrier(ws)
    ms, res = timed(Ad, prec, args.steps, args.warmup)
    dist_barrier(ws)
    clk = clocks.stop()
    ms = dist_max(ws, ms)
    err = rel_error(res, Ad)
    fp64 = {}
    if not args.skip_fp64:
        A64 = synth_colmajor(Ad.double())
        ms64, r64 = timed(A64, "fp64", 2, 1)
        fp64 = {"ms_per_step": ms64, "rel_error": rel_error(r64, Ad)}
        del A64
    flops = 4.0 * w.m * w.n * w.k
    abytes = w.m * w.n * Ad.element_size()
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": flops * ws / (ms / 1e3) / 1e12, "unit": "TFLOP/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32", "tf32": "tf32", "tf32x3": "tf32x3"}[prec],
            "data": "synthetic",
            "config": {"workload": w.name, "algo": "singlepass", "m": w.m, "n": w.n, "k": w.k,
                       "sigma": w.sigma, "pass_precision": prec, "between_passes": "f64",
                       "parallelism": "replicas" if ws > 1 else "single"},
            "rel_error": err, "hbm_gbs_one_read_of_A": abytes / (ms / 1e3) / 1e9,
            "fp64_plain": fp64,
            "speedup_vs_fp64_plain": (fp64["ms_per_step"] / ms) if fp64 else None,
            "gpu_launches": res[4]["launches"], "clocks": clk,
        }))
    ctx.close()
    return 0


def run_randlu(args, w):
    """The paper's main speed comparison, on this GPU: RandLU (Alg. rlu with
    Alg. basicpoweriteration, p power iterations, 2p + 2 passes over A)
    against PowerLU with the same number of passes (v = 2p + 2), same A, same
    rank and oversampling, same pass precision.  value counts RandLU's pass
    FLOPs (2 m n l per pass, 2 m n k for the pass that forms B)."""
    import numpy as np
    import torch
    import paper_2002_07138_gb300 as plu

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    Ad = replica_workload(w, rank).build("cuda")
    torch.cuda.empty_cache()
    stream = torch.cuda.current_stream()
    ctx = plu.Context(local, stream.cuda_stream)
    prec = args.prec
    piter = args.piter
    v = 2 * piter + 2

    def timed(fn, steps, warmup):
        for i in range(warmup):
            fn(i)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(steps):
            res = fn(1000 + i)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps, res

    def rel_error(res, A):
        p, q, L, U = res[:4]
        Ap = A.double()[p.long()][:, q.long()]
        return float(torch.linalg.norm(Ap - L @ U) / torch.linalg.norm(A.double()))

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    dist_barrier(ws)
    ms, res = timed(lambda s: plu.plu_randlu(ctx, Ad, w.k, w.l, piter, seed=s, prec=prec),
                    args.steps, args.warmup)
    dist_barrier(ws)
    clk = clocks.stop()
    ms = dist_max(ws, ms)
    err = rel_error(res, Ad)
    ms_p, res_p = timed(lambda s: plu.plu_powerlu(ctx, Ad, w.k, w.l, v, seed=s, prec=prec),
                        args.steps, args.warmup)
    err_p = rel_error(res_p, Ad)
    flops = 2.0 * w.m * w.n * (w.l * (v - 1) + w.k)
    sig = w.sigma_values()
    opt = float(np.sqrt(np.sum(sig[w.k:] ** 2) / np.sum(sig ** 2)))
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": flops * ws / (ms / 1e3) / 1e12, "unit": "TFLOP/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32"}.get(prec, prec), "data": "synthetic",
            "config": {"workload": w.name, "algo": "randlu", "m": w.m, "n": w.n, "k": w.k,
                       "l": w.l, "power_iterations": piter, "passes": v, "sigma": w.sigma,
                       "pass_precision": prec, "between_passes": "f64",
                       "parallelism": "replicas" if ws > 1 else "single"},
            "rel_error": err, "eckart_young_optimum": opt,
            "powerlu_same_passes": {"v": v, "ms_per_step": ms_p, "rel_error": err_p},
            "speedup_powerlu_vs_randlu": ms / ms_p,
            "gpu_launches": res[4]["launches"], "clocks": clk,
        }))
    ctx.close()
    return 0


# ---------------------------------------------------------------- sparse
SPARSE = {"name": "sparse_32000_d0.003_k200_l200_v4", "n": 32000, "density": 0.003,
          "k": 200, "l": 200, "v": 4, "seed": 0}


def sparse_host(seed):
    import synth
    sp = SPARSE
    rp, ci, val = synth.sprand_csr(sp["n"], sp["n"], sp["density"], seed)
    return rp, ci, val


def sparse_pass_bytes(n, nnz, cols):
    """Algorithmic bytes of one sparse pass: the CSR arrays (8 B value +
    4 B index per nonzero, the row pointers), X read once and Y written once."""
    return nnz * 12.0 + (n + 1) * 8.0 + 2.0 * n * cols * 8.0


def sparse_rel_error(torch, m, rp, ci, val, p, q, L, U):
    """||A - P^T L U Q||_F / ||A||_F for a sparse A (CUDA CSR tensors rp, ci,
    val) without forming L U: ||A||^2 = sum val^2, <A, P^T L U Q> one k-length
    dot product per nonzero, ||L U||^2 = trace((L^T L)(U U^T)).  Measurement
    only (torch), outside the timed region."""
    dev = L.device
    pinv = torch.empty_like(p.long())
    pinv[p.long()] = torch.arange(m, device=dev)
    qinv = torch.empty_like(q.long())
    qinv[q.long()] = torch.arange(q.numel(), device=dev)
    rows = torch.repeat_interleave(torch.arange(m, device=dev), rp[1:] - rp[:-1])
    cil = ci.long()
    normA2 = float((val * val).sum())
    inner = 0.0
    step = 1 << 19
    for s0 in range(0, val.numel(), step):
        r = pinv[rows[s0:s0 + step]]
        c = qinv[cil[s0:s0 + step]]
        inner += float((val[s0:s0 + step] * (L[r] * U[:, c].t()).sum(1)).sum())
    normLU2 = float(((L.t() @ L) * (U @ U.t())).sum())
    return max(normA2 - 2.0 * inner + normLU2, 0.0) ** 0.5 / normA2 ** 0.5


def run_sparse(args):
    """PowerLU (Alg. bpowerlu + Alg. gpowerlu) on the sparse workload, every
    pass an FP64 sparse product.  value = the passes' algorithmic flops
    (2 nnz per column) over the call time."""
    import numpy as np
    import torch
    import synth
    import paper_2002_07138_gb300 as plu

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    peaks = {"hbm_gbs": 6791.0, "bf16_tflops": 1934.6, "sm_max_mhz": 2070.0}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks.update(json.load(f))
    except OSError:
        peaks["source"] = "fallback"
    sp = SPARSE
    n, k, l, v = sp["n"], sp["k"], sp["l"], sp["v"]
    rp, ci, val = sparse_host(sp["seed"] + rank)
    nnz = int(rp[-1])
    host_arrays = (rp, ci, val) + tuple(synth.csr_transpose(n, n, rp, ci, val))
    pinned = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in host_arrays]
    dev_arrays = [t.cuda() for t in pinned]
    S = plu.CsrMatrix(n, n, *dev_arrays)
    stream = torch.cuda.current_stream()
    ctx = plu.Context(local, stream.cuda_stream)
    flops = 2.0 * nnz * (l * (v - 1) + k)

    def call(seed, A=S, vv=v):
        return plu.plu_powerlu_csr(ctx, A, k, l, vv, seed=seed)

    # the CSR arrays of A and A^T (about 74 MB) fit L2: a 256 MB write flushes
    # it before every timed call, outside the call's events
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
    for i in range(args.warmup):
        call(i)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    dist_barrier(ws)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    reps = []
    for i, (e0, e1) in enumerate(evs):
        flush.zero_()
        e0.record(stream)
        reps.append(call(1000 + i)[4])
        e1.record(stream)
    torch.cuda.synchronize()
    dist_barrier(ws)
    clk = clocks.stop()
    ms_total = sum(e0.elapsed_time(e1) for e0, e1 in evs)
    ms_max = dist_max(ws, ms_total)
    ms_step = ms_max / args.steps
    value = flops * args.steps * ws / (ms_max / 1e3) / 1e12
    launches = int(sum(r["launches"] for r in reps))
    ms_pass = statistics.mean(r["ms_passes"] / r["passes"] for r in reps)

    # v = 2 (no power iteration, the paper's left panel), one timed call
    call(0, vv=2)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    call(5, vv=2)
    t1.record(stream)
    torch.cuda.synchronize()
    ms_v2 = t0.elapsed_time(t1)

    # end to end: the CSR arrays host -> device, the call, the factors back
    dev_e = [torch.empty_like(t) for t in dev_arrays]
    Se = plu.CsrMatrix(n, n, *dev_e)
    ph = torch.empty(n, dtype=torch.int32, pin_memory=True)
    qh = torch.empty(n, dtype=torch.int32, pin_memory=True)
    Lh = torch.empty(k, n, dtype=torch.float64, pin_memory=True).t()
    Uh = torch.empty(n, k, dtype=torch.float64, pin_memory=True).t()

    def e2e_step(seed):
        for d, h in zip(dev_e, pinned):
            d.copy_(h, non_blocking=True)
        p, q, L, U, _ = call(seed, Se)
        ph.copy_(p, non_blocking=True)
        qh.copy_(q, non_blocking=True)
        Lh.copy_(L, non_blocking=True)
        Uh.copy_(U, non_blocking=True)
        torch.cuda.synchronize()

    e2e_step(0)
    ne = max(2, min(args.steps, 5))
    t0h = time.perf_counter()
    for i in range(ne):
        e2e_step(3000 + i)
    e2e_ms = dist_max(ws, 1e3 * (time.perf_counter() - t0h) / ne)
    h2d = sum(t.numel() * t.element_size() for t in pinned)
    d2h = 8 * n + 16 * n * k

    # the steps timed alone (asynchronous context: no host sync per call)
    plu.lib().plu_set_async(ctx.handle, 1)
    X = plu.colmajor_empty(n, l)
    X.normal_()
    Z = plu.colmajor_empty(n, l)
    ms0 = time_calls(torch, lambda: plu.plu_spmm(ctx, S, 0, X, out=Z), 5, stream)
    ms1 = time_calls(torch, lambda: plu.plu_spmm(ctx, S, 1, Z, out=X), 5, stream)
    ms_sp = 0.5 * (ms0 + ms1)
    Zc = Z.clone()
    ctx.set_lu_updates(1)              # as the sparse call runs its LUs
    ms_lu = time_calls(torch, lambda: (Zc.copy_(Z), plu.plu_lu_reorth(ctx, Zc)), 3, stream)
    ms_cp = time_calls(torch, lambda: Zc.copy_(Z), 3, stream)
    ms_lu = max(ms_lu - ms_cp, 1e-6)
    ctx.set_lu_updates(-1)
    plu.lib().plu_set_async(ctx.handle, 0)
    ctx.check(plu.lib().plu_check(ctx.handle))
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    # launches per call: v passes; v - 2 re-orthogonalising LUs (v > 2) and
    # the tail's two LUs of n x k panels
    share = {"spmm": ms_sp * v, "panel_lu": ms_lu * (max(v - 2, 0) + 2)}
    # the sparse pass issues one FP64 FMA per nonzero and column: at GB300's
    # FP64 rate that, not HBM (the CSR arrays and two n x l operands) or the
    # L2 gathers of X's rows, is its bound
    pbytes = sparse_pass_bytes(n, nnz, l)
    pm = measure_peaks(torch, plu, ctx, stream, local)
    fp64pk = pm["fp64_tflops"]
    rf_sp = {"bound": "alu", "achieved": 2.0 * nnz * l / ms_sp / 1e9, "peak": fp64pk,
             "unit": "TFLOP/s", "peak_source": "measured FP64 GEMM (of measured, peaks_measured)",
             "kernel": "k_spmm_csr + k_to_rowmajor", "ms_per_launch": ms_sp,
             "traffic": None, "share_of_step": share["spmm"] / ms_step,
             "hbm_gbs": pbytes / ms_sp / 1e6, "hbm_frac": pbytes / ms_sp / 1e6 / peaks["hbm_gbs"],
             "l2_gather_gbs": nnz * l * 8.0 / ms_sp / 1e6,
             "note": "the rows of X a pass gathers (nnz x l x 8 B) come from L2"}
    rf_sp["frac"] = rf_sp["achieved"] / rf_sp["peak"]
    # the leaf kernel of the tensor-core LU (one 32-column leaf, timed alone)
    # against the FP64 pipe; the whole LU's FP64-equivalent rate beside it
    Z32 = Z[:, :32].clone()
    Zc32 = Z32.clone()
    ctx.set_lu_updates(1)
    ms_leaf = time_calls(torch, lambda: (Zc32.copy_(Z32), plu.plu_lu_reorth(ctx, Zc32)), 5, stream)
    ms_leaf = max(ms_leaf - time_calls(torch, lambda: Zc32.copy_(Z32), 5, stream), 1e-6)
    ctx.set_lu_updates(-1)
    rf_lu = {"bound": "alu", "achieved": leaf_flops(n, 32) / ms_leaf / 1e9, "peak": fp64pk,
             "unit": "TFLOP/s", "peak_source": "measured FP64 GEMM (of measured, peaks_measured)",
             "kernel": "k_lu_leaf", "ms_per_launch": ms_leaf, "traffic": None,
             "share_of_step": share["panel_lu"] / ms_step, "ms_whole_lu": ms_lu,
             "fp64_equivalent_tflops_whole_lu": lu_flops(n, l) / ms_lu / 1e9}
    rf_lu["frac"] = rf_lu["achieved"] / rf_lu["peak"]
    rf = rf_sp if share["spmm"] >= share["panel_lu"] else rf_lu

    # accuracy of one call, formed from the nonzeros (outside the timed region)
    res = call(7)
    rel_err = sparse_rel_error(torch, n, dev_arrays[0], dev_arrays[1], dev_arrays[2], *res[:4])

    cpu = None
    if rank == 0 and ws == 1 and not args.skip_cpu:
        dt, sfl, desc = sparse_oracle_sample(n, rp, ci, val, seed=0)
        cpu = {"value": sfl / dt / 1e12, "unit": "TFLOP/s", "cores": os.cpu_count(),
               "kind": "oracle", "sample": "%s on the same matrix, %.1f s" % (desc, dt)}
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": sp["name"], "m": n, "n": n, "nnz": nnz,
                       "density": sp["density"], "values": "uniform [0, 1)", "k": k, "l": l,
                       "v": v, "pass_precision": "fp64 (sparse)", "between_passes": "f64",
                       "l2_flush": "256 MB write before every timed call, outside its "
                                   "events (the CSR arrays of A and A^T are %.0f MB)" % (h2d / 1e6),
                       "parallelism": "replicas" if ws > 1 else "single"},
            "ms_per_pass": ms_pass, "ms_per_step_v2": ms_v2, "rel_error": rel_err,
            "tflops_per_pass": 2.0 * nnz * l / (ms_pass / 1e3) / 1e12,
            "e2e": {"value": flops * ws / (e2e_ms / 1e3) / 1e12, "unit": "TFLOP/s",
                    "ms_per_step": e2e_ms, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches, "clocks": clk, "roofline": rf, "roofline_spmm": rf_sp,
            "roofline_panel_lu": rf_lu,
            "kernel_ms": {"spmm": {"ms_per_launch": ms_sp, "launches_per_step": v},
                          "panel_lu": {"ms_per_launch": ms_lu,
                                       "launches_per_step": max(v - 2, 0) + 2}},
            "ms_phase": {nm: statistics.mean(r["ms_phase"][nm] for r in reps)
                         for nm in reps[0]["ms_phase"]},
            "peaks_measured": pm,
            "cpu_baseline": cpu,
        }))
    ctx.close()
    return 0


def sparse_oracle_sample(n, rp, ci, val, seed):
    """The oracle's first pass of Alg. gpowerlu on the sparse A (v even:
    A^T Omega) and its LU re-orthogonalisation.  Returns (seconds, flops,
    description)."""
    import oracle
    l = SPARSE["l"]
    t0 = time.perf_counter()
    Om = oracle.gaussian_matrix(n, l, seed, oracle.STREAM_OMEGA_M)
    Y = oracle.csr_tmul(n, rp, ci, val, Om)
    oracle.lu_permuted_L(Y)
    dt = time.perf_counter() - t0
    return dt, 2.0 * int(rp[-1]) * l, ("the oracle's first pass of Alg. gpowerlu (A^T Omega "
                                       "from the CSR, FP64, on one core) and its LU "
                                       "re-orthogonalisation (numpy BLAS threads)")


def run_reference_sparse(args):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return 0
    sp = SPARSE
    rp, ci, val = sparse_host(sp["seed"])
    for i in range(args.warmup):
        sparse_oracle_sample(sp["n"], rp, ci, val, seed=i)
    times = []
    for i in range(args.steps):
        dt, flops, desc = sparse_oracle_sample(sp["n"], rp, ci, val, seed=i)
        times.append(dt)
    total = sum(times)
    value = flops * args.steps / total / 1e12
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": sp["name"], "m": sp["n"], "n": sp["n"], "nnz": int(rp[-1]),
                   "density": sp["density"], "k": sp["k"], "l": sp["l"], "v": sp["v"]},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": os.cpu_count(),
                         "kind": "oracle", "sample": desc + " per step"},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))
    return 0


def synth_colmajor(t):
    import synth
    return synth.colmajor(t)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mixed_32768", choices=sorted(workloads()))
    ap.add_argument("--prec", default="tf32", choices=["fp64", "fp32", "tf32", "bf16", "fp8",
                                                         "tf32x3"])
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--algo", default="powerlu", choices=["powerlu", "singlepass", "randlu"],
                    help="singlepass: Alg. singlepasslu (rank k, one read of A) on the workload; "
                         "randlu: RandLU with --piter power iterations against PowerLU with "
                         "as many passes")
    ap.add_argument("--piter", type=int, default=1,
                    help="power iterations of RandLU (--algo randlu): 2 piter + 2 passes")
    args = ap.parse_args()
    if args.workload == "batched_512":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the batched workload has no "
                              "reference arm; use the default workload"}))
            return 0
        return run_batched(args)
    if args.workload == "sparse_32000":
        return run_reference_sparse(args) if args.impl == "reference" else run_sparse(args)
    w = workloads()[args.workload]
    if args.impl == "reference":
        return run_reference(args, w)
    if w.eps:
        return run_fixed_precision(args, w)
    if args.algo == "singlepass":
        return run_singlepass(args, w)
    if args.algo == "randlu":
        return run_randlu(args, w)
    return run_ours(args, w)


if __name__ == "__main__":
    sys.exit(main())
