#!/usr/bin/env python3
"""OverSketch benchmark: sketched A.B effective TFLOP/s (2mnl/t) on GB300.

One step = one whole OverSketch product on the square workload
(A 16384x65536, B 65536x16384 FP32 N(0,1) + rank-64 spike; b=1024, N=8,
e=2; blocks {1,6} dropped): left sketch, right sketch (both emitting the GEMM
dtype), masked block-sum GEMM with scale 1/k.  Inputs (8.6 GB) exceed L2, so
no flush is needed between steps.  The plan (hash + bucket-CSR) is built once
before timing, as the same S is reused across products.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--dtype bf16|f32|fp8]
  python bench.py --impl reference ...   # the FP64 CPU oracle on a sample
  python bench.py --workload small|hessian|batched|autograd|lp|sec51   # the other workloads

The other workloads: the minimum slice 512x4096x512 timed with L2 flushed and
warm (small); the interior-point normal matrix A D A^T with a 1 %-dense
A (hessian); 256 uneven products in one CUDA graph (batched); a BF16 forward
and backward (autograd); the LP of Sec. 5.2 with its sketched Hessian and
100-iteration barrier runs (lp); the accuracy study of Sec. 5.1 on
A(x, y) = x + y (sec51).

Multi-GPU (torchrun): every rank runs its own independent product (weak
scaling, no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sketched A·B effective TFLOP/s (2mnl/t) vs exact GEMM at stated Frobenius error"
# DRAM bytes (read + write) of one gemm_pair_bf16_kernel launch on the square workload:
# one ncu capture of the 8192 x 8192 x 8192 product (--shape 8192,65536,8192), scaled by
# the 4x tiles of the full 16384 x 8192 x 16384 product (profiles/square_launch_list.md)
TRAFFIC_GEMM_PAIR_SQUARE = 4 * (1280785000 + 255578368)
# DRAM bytes (read + write) of sketch_left_onepass_kernel on the first 304 rows of the
# interior-point operand (--workload hessian --rows 304; profiles/sketch_left_onepass_304x1048576.md):
# the kernel streams each row once, so a launch over m rows moves m / 304 times as much
TRAFFIC_ONEPASS_304_ROWS = 1298136000 + 19260672
UNIT = "TFLOP/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _backend() -> str:
    """NCCL between GPUs; gloo where no GPU is present (the CPU tests of this logic)."""
    import torch
    return "nccl" if torch.cuda.is_available() else "gloo"


def _max_over_ranks(x: float, world: int) -> float:
    """The largest of every rank's x (the step time the whole job waits for)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if _backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _job_value(flop_per_rank: float, ms_max: float, world: int) -> float:
    """Whole-job throughput in TFLOP/s: every rank runs its own product (weak
    scaling), so the job does world x the per-rank work in the slowest rank's time."""
    return world * flop_per_rank / (ms_max * 1e-3) / 1e12


# ----------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ----------------------------------------------------------------------------

def oracle_sample_time(w, rows: int, cols: int, reps: int = 1, inputs=None):
    """Time the oracle (as it stands) on a rows x n x cols sample of the workload:
    both sketches and the masked product in FP64 (the plan is built once,
    untimed, as on the GPU).  Returns (seconds, threads used, description)."""
    import oracle
    if inputs is None:
        A = w.left_rows(range(rows)).astype(np.float64)
        B = np.ascontiguousarray(w.right_cols(range(cols)).T, dtype=np.float64)
        h, s = oracle.hash_tables(w.n, w.b, w.N, w.e, w.hash_seed)
    else:
        A, B, h, s = inputs
    oracle.oversketch(A[:4], B[:, :4], h, s, w.b, w.mask)      # load + warm
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.oversketch(A, B, h, s, w.b, w.mask)
        ts.append(time.perf_counter() - t0)
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    desc = (f"{rows} rows of A x {cols} columns of B at full n={w.n}: both sketches and the masked "
            f"product in FP64 (effective flop 2*{rows}*{w.n}*{cols}); plan built once, untimed")
    return min(ts), threads, desc


def calibrated_sample(w, target_s: float) -> int:
    """Rows (= columns) of the oracle sample that take about target_s seconds."""
    t, _, _ = oracle_sample_time(w, 128, 128)
    r = int(128 * target_s / max(t, 1e-3))
    return int(min(4096, max(64, r // 64 * 64)))


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    from paper_1811_02653_gb300 import workloads as W
    w = _workload(args)
    budget = 150.0 / max(1, args.steps + args.warmup)          # whole run within a few minutes
    rows = cols = args.ref_sample or calibrated_sample(w, budget)
    A = w.left_rows(range(rows)).astype(np.float64)
    B = np.ascontiguousarray(w.right_cols(range(cols)).T, dtype=np.float64)
    h, s = oracle.hash_tables(w.n, w.b, w.N, w.e, w.hash_seed)
    inputs = (A, B, h, s)
    for _ in range(args.warmup):
        oracle_sample_time(w, rows, cols, inputs=inputs)
    steps_t = []
    threads, desc = 1, ""
    for _ in range(args.steps):
        t, threads, desc = oracle_sample_time(w, rows, cols, inputs=inputs)
        steps_t.append(t)
    t = statistics.median(steps_t)
    value = 2.0 * rows * w.n * cols / t / 1e12
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(w, args, sample=f"{rows}x{w.n}x{cols}"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _time_plans(ops, w, runs: int):
    """Host wall times of oversketch_plan (table allocation, hash, bucket-CSR,
    synchronise) and the device time between CUDA events on its stream."""
    import torch
    host, dev = [], []
    st = torch.cuda.current_stream()
    for _ in range(runs):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0.record(st)
        q = ops.plan(w.n, w.b, w.N, w.e, w.hash_seed)
        e1.record(st)
        host.append(time.perf_counter() - t0)
        e1.synchronize()
        dev.append(e0.elapsed_time(e1))
        q.destroy()
    return host, dev


def _plan_record(host_s, dev_ms):
    return {"median": statistics.median(host_s) * 1e3, "device_median": statistics.median(dev_ms), "runs": len(host_s),
            "what": "oversketch_plan: host wall time (table allocation, hash, bucket-CSR, synchronise) and the "
                    "device time between CUDA events around it"}


def _sketch_dtype(gemm_dtype: str, b: int) -> str:
    """Sketch output dtype of a GEMM dtype: the FP32 product runs as 3xTF32 on the
    tensor cores, so its sketches emit hi/lo planes."""
    return "tf32x2" if gemm_dtype == "f32" and b % 32 == 0 else gemm_dtype


def _oracle_product_as(oracle, f, At_r, Bt_c, b, mask):
    """The oracle's masked product with the operand rounding of GEMM dtype f
    (BF16: RNE of the sketch; FP8: per-(row, 128-column) UE8M0 scale + E4M3)."""
    if f == "bf16":
        return oracle.masked_product(oracle.round_bf16(At_r), oracle.round_bf16(Bt_c), b, mask)
    if f == "fp8":
        Aq = oracle.dequantize_fp8_rows(*oracle.quantize_fp8_rows(At_r))
        Bq = oracle.dequantize_fp8_rows(*oracle.quantize_fp8_rows(Bt_c.T)).T
        return oracle.masked_product(Aq, Bq, b, mask)
    return oracle.masked_product(At_r, Bt_c, b, mask)


def _workload(args):
    from paper_1811_02653_gb300 import workloads as W
    if args.shape:
        m, n, l = (int(x) for x in args.shape.split(","))
        return W.scaled(W.SQUARE, m=m, n=n, l=l,
                        name=f"square-shaped {m}x{n}x{l} (profiling size), b=1024 N=8 e=2, blocks {{1,6}} dropped")
    return W.SQUARE


def _config(w, args, **extra):
    d = {"workload": w.name, "m": w.m, "n": w.n, "l": w.l, "b": w.b, "N": w.N, "e": w.e,
         "kept_blocks": [j for j in range(w.P) if (w.mask >> j) & 1], "gemm_dtype": args.dtype,
         "input_dtype": "f32",
         "l2": f"inputs ({(w.m * w.n + w.n * w.l) * 4 / 1e9:.1f} GB) larger than L2 (129 MB); no flush needed",
         "parallelism": f"replicas{args.gpus}"}
    d.update(extra)
    return d


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------

def run_ours(args):
    import torch

    from paper_1811_02653_gb300 import build, ops
    from paper_1811_02653_gb300 import workloads as W

    world, rank, local = _init_dist()
    build.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    w = _workload(args)
    peaks, peak_kind = _peaks()

    # ---- inputs (host, pinned) and device copies ----
    A_h = torch.from_numpy(w.left()).pin_memory()
    Bt_h = torch.from_numpy(w.right_cols(range(w.l)))            # l x n: columns of B
    A = A_h.to(dev, non_blocking=False)
    B = Bt_h.to(dev).t().contiguous()                              # n x l row-major
    B_h = B.cpu().pin_memory()
    del Bt_h
    # plan creation (hash tables + bucket-CSR; oversketch_plan synchronises), timed
    # on its own: the same S serves every product, so it is outside the step
    plan_s, plan_dev = _time_plans(ops, w, 3)
    p = ops.plan(w.n, w.b, w.N, w.e, w.hash_seed)
    gd = args.dtype
    sd = _sketch_dtype(gd, w.b)
    z = p.z
    At, a_sc = ops.sketch_left(p, A, sd)
    BtT, b_sc = ops.sketch_right(p, B, sd)
    C = torch.empty((w.m, w.l), dtype=torch.float32, device=dev)
    # one packed-strip workspace, reused by the left and then the right sketch (as oversketch_matmul does;
    # FP8 sketches also stage their FP32 sums there)
    ws_pack = torch.empty(ops.workspace_size(p, w.m, w.l, torch.float32, gd) if gd == "fp8" else
                          max(ops.sketch_workspace(p, w.m), ops.sketch_workspace(p, w.l)), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    # the same three calls oversketch_matmul makes: only kept blocks are sketched
    def step():
        ops.sketch_left(p, A, sd, out=At, scales=a_sc, workspace=ws_pack, block_mask=w.mask)
        ops.sketch_right(p, B, sd, out=BtT, scales=b_sc, block_mask=w.mask, workspace=ws_pack)
        ops.gemm_masked(p, At, BtT, w.mask, C=C, a_scales=a_sc, b_scales=b_sc, dtype=sd)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- timed region: K steps, per-phase events on the launching stream ----
    n_ev = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(n_ev)]
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    _barrier(world)
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for s in range(args.steps):
        e = ev[s]
        e[0].record(stream)
        ops.sketch_left(p, A, sd, out=At, scales=a_sc, workspace=ws_pack, block_mask=w.mask)
        e[1].record(stream)
        ops.sketch_right(p, B, sd, out=BtT, scales=b_sc, block_mask=w.mask, workspace=ws_pack)
        e[2].record(stream)
        ops.gemm_masked(p, At, BtT, w.mask, C=C, a_scales=a_sc, b_scales=b_sc, dtype=sd)
        e[3].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    _barrier(world)
    clk = clocks.stop()
    total_ms = _max_over_ranks(t_start.elapsed_time(t_end), world)
    ms = total_ms / args.steps
    t_left = statistics.mean(e[0].elapsed_time(e[1]) for e in ev)
    t_right = statistics.mean(e[1].elapsed_time(e[2]) for e in ev)
    t_gemm = statistics.mean(e[2].elapsed_time(e[3]) for e in ev)
    flop_eff = 2.0 * w.m * w.n * w.l
    value = _job_value(flop_eff, ms, world)

    # ---- end to end through the C ABI with host buffers (oversketch_matmul_host:
    # pinned A and B in, C out, the transfers overlapped with the kernels) ----
    C_h = torch.empty((w.m, w.l), dtype=torch.float32).pin_memory()
    ws_mm = torch.empty(ops.workspace_size(p, w.m, w.l, torch.float32, gd), dtype=torch.uint8, device=dev)
    ws_host = torch.empty(ops.matmul_host_workspace(p, w.m, w.l, gemm_dtype=gd), dtype=torch.uint8, device=dev)
    e2e_steps = max(3, min(args.steps, 10))

    def e2e_step():
        ops.matmul_host(p, A_h, B_h, w.mask, gd, C=C_h, workspace=ws_host)

    e2e_step()
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    s1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = _max_over_ranks(s0.elapsed_time(s1) / e2e_steps, world)
    h2d = A_h.numel() * 4 + B_h.numel() * 4
    d2h = C_h.numel() * 4

    # ---- the other GEMM dtypes on the same inputs (same three calls, own sketch buffers) ----
    forms = {}
    if not args.no_forms:
        for f in [x for x in ("f32", "fp8", "bf16") if x != gd]:
            sf = _sketch_dtype(f, w.b)
            # the workspace oversketch_matmul sizes for this dtype (FP8: room to stage the FP32 sums)
            ws_f = torch.empty(ops.workspace_size(p, w.m, w.l, torch.float32, f), dtype=torch.uint8, device=dev)
            Af, asf = ops.sketch_left(p, A, sf, workspace=ws_f)
            Bf, bsf = ops.sketch_right(p, B, sf, workspace=ws_f)
            phases_f = [("sketch_left", lambda: ops.sketch_left(p, A, sf, out=Af, scales=asf, workspace=ws_f,
                                                                 block_mask=w.mask)),
                        ("sketch_right", lambda: ops.sketch_right(p, B, sf, out=Bf, scales=bsf, block_mask=w.mask,
                                                                   workspace=ws_f)),
                        ("gemm_masked", lambda: ops.gemm_masked(p, Af, Bf, w.mask, C=C, a_scales=asf, b_scales=bsf,
                                                                dtype=sf))]
            ms_f, per_f, _ = _time_phases(phases_f, max(3, min(args.steps, 10)), 2, world, sample_clocks=False)
            forms[f] = {"ms_per_step": ms_f, "tflops": _job_value(2.0 * w.m * w.n * w.l, ms_f, world),
                        "phases_ms": {k_: round(v_, 4) for k_, v_ in per_f.items()},
                        "sketch_dtype": sf}
            del Af, Bf, asf, bsf, ws_f
        torch.cuda.synchronize()

    # ---- exact GEMM on the same GPU: the same tcgen05 kernel over K = n (all blocks kept) ----
    exact = None
    if not args.no_exact and w.n % 64 == 0 and w.n // 64 <= 4096:
        bx = 1024 if w.n % 1024 == 0 and w.n // 1024 <= 64 else None
        if bx is not None:
            A16 = A.to(torch.bfloat16)
            Bt16 = B.t().contiguous().to(torch.bfloat16)         # l x n, K-major (setup, untimed)
            pe = ops.plan(w.n, bx, w.n // bx, 0, 0)
            full = (1 << (w.n // bx)) - 1
            Cx = torch.empty((w.m, w.l), dtype=torch.float32, device=dev)
            # every block kept: alpha = k cancels the library's 1/k, giving A.B itself
            ops.gemm_masked(pe, A16, Bt16, full, alpha=float(w.n // bx), C=Cx)
            torch.cuda.synchronize()
            x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 3
            x0.record(stream)
            for _ in range(reps):
                ops.gemm_masked(pe, A16, Bt16, full, alpha=float(w.n // bx), C=Cx)
            x1.record(stream)
            torch.cuda.synchronize()
            ex_ms = x0.elapsed_time(x1) / reps
            exact = {"ms": ex_ms, "tflops": flop_eff / (ex_ms * 1e-3) / 1e12, "dtype": "bf16",
                     "kernel": "gemm_pair_bf16_kernel with every block of a width-1024 split of n kept",
                     "sketched_speedup": ex_ms / ms}
            exact_C = Cx
            del A16, Bt16

    # ---- dominant kernel and its roofline ----
    es = {"bf16": 2, "f32": 4, "fp8": 1, "tf32x2": 8}[sd]
    n_kept = w.k
    right_bytes = w.n * w.l * 4 + w.l * n_kept * w.b * es
    left_bytes = w.m * w.n * 4 + w.m * n_kept * w.b * es
    gemm_flop = 2.0 * w.m * n_kept * w.b * w.l
    # the sketches against HBM (algorithmic bytes: operand read once, kept blocks written
    # once) and as signed adds (rows * n * k); their own bound is the L2 gather (DESIGN)
    hbm = peaks.get("hbm_gbs")
    sketch_roofs = {}
    for side, nbytes, rows, t_ms in (("left", left_bytes, w.m, t_left), ("right", right_bytes, w.l, t_right)):
        gbs = nbytes / (t_ms * 1e-3) / 1e9
        sketch_roofs[side] = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                              "frac": gbs / hbm if hbm else None, "algorithmic_bytes": nbytes,
                              "signed_adds_per_s": float(rows) * w.n * n_kept / (t_ms * 1e-3)}
    phases = {"sketch_left (pack + gather)": t_left, "sketch_right (pack + gather)": t_right,
              "gemm_masked": t_gemm}
    if t_gemm >= t_right:
        ach = gemm_flop / (t_gemm * 1e-3) / 1e12
        bound, unit = "tensor", "TFLOP/s"
        if sd == "bf16":
            # CTA-pair tcgen05 kernel; it runs ~2.5 ms at a time between memory-bound
            # phases at full clock, so the burst (not the seconds-long sustained) peak
            dom = "gemm_pair_bf16_kernel (BF16, cta_group::2)"
            peak = peaks.get("bf16_tflops", peaks.get("bf16_tflops_sustained"))
        elif sd == "fp8":
            # block-scaled E4M3: nominal FP8 : BF16 tensor rate = 2 : 1
            dom = "gemm_masked_tc_kernel<Cfg<224,4,Fp8>> (E4M3, UE8M0 block scales)"
            peak = 2.0 * peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
        elif sd == "tf32x2":
            # three TF32 products per K step at half the BF16 rate: the useful FP32 rate peaks
            # at 1/6 of the BF16 figure (nominal TF32 : BF16 = 1 : 2)
            dom = "gemm_masked_tc_kernel<Cfg<128,3,2>> (3xTF32)"
            peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops")) / 6.0
        else:
            dom = "gemm_masked_f32_kernel (FFMA)"
            peak, bound = None, "alu"
        per_launch = {"flop": gemm_flop}
    else:
        dom = "sketch_gather_kernel (right sketch)"
        peak = peaks.get("hbm_gbs")
        bound, unit, ach = "hbm", "GB/s", right_bytes / (t_right * 1e-3) / 1e9
        per_launch = {"bytes": right_bytes}
    # DRAM bytes per launch from one ncu capture of this command (profiles/square_launch_list.md);
    # valid for the square workload with the kernels as they were when captured
    traffic = None
    if sd == "bf16" and dom.startswith("gemm_pair_bf16") and (w.m, w.n, w.l) == (16384, 65536, 16384):
        traffic = TRAFFIC_GEMM_PAIR_SQUARE
    roof = {"bound": bound, "achieved": ach, "peak": peak, "unit": unit,
            "frac": (ach / peak) if peak else None, "traffic": traffic, "kernel": dom,
            "peak_source": f"{peak_kind} (MEASURED_PEAKS.json)" if peak_kind == "measured" else "fallback",
            "algorithmic_per_launch": per_launch}

    # ---- the cpu_baseline leg (not timed on the GPU): the FP64 oracle on a
    # bounded sample, and sampled entries of C set beside the oracle's ----
    err = None
    cpu = None
    if _cpu_leg(args, rank, world):
        import oracle
        if not args.no_check:
            rows = sorted({0, 1, 2, 777 % w.m, w.m // 4, w.m // 2, (3 * w.m) // 4, w.m - 1})
            cols = sorted({0, 3, 4096 % w.l, 5000 % w.l, w.l // 3, (2 * w.l) // 3, w.l - 2, w.l - 1})
            h, s = oracle.hash_tables(w.n, w.b, w.N, w.e, w.hash_seed)
            Ar = w.left_rows(rows).astype(np.float64)
            Bc = np.ascontiguousarray(w.right_cols(cols).T, dtype=np.float64)
            At_r = oracle.sketch_left(Ar, h, s, w.b)
            Bt_c = oracle.sketch_right(Bc, h, s, w.b)
            C_or_exact_sketch = oracle.masked_product(At_r, Bt_c, w.b, w.mask)
            AB = Ar @ Bc

            def sampled_error(f):
                C_or = _oracle_product_as(oracle, f, At_r, Bt_c, w.b, w.mask)
                ws_f = torch.empty(ops.workspace_size(p, w.m, w.l, torch.float32, f), dtype=torch.uint8, device=dev)
                ops.matmul(p, A, B, w.mask, f, C=C, workspace=ws_f)
                C_s = C[rows][:, cols].cpu().numpy().astype(np.float64)
                del ws_f
                return oracle.rel_frob(C_s, C_or), oracle.rel_frob(C_s, AB)

            if exact is not None:
                exact["vs_exact_rel_frob"] = oracle.rel_frob(exact_C[rows][:, cols].cpu().numpy(), Ar @ Bc)
            e_or, e_ex = sampled_error(gd)
            err = {"vs_oracle_rel_frob": e_or, "vs_exact_rel_frob": e_ex,
                   "oracle_sketch_vs_exact_rel_frob": oracle.rel_frob(C_or_exact_sketch, AB),
                   "sample": f"{len(rows)}x{len(cols)} entries of C; oracle emulates {gd} operand rounding"}
            for f, d in forms.items():
                d["vs_oracle_rel_frob"], d["vs_exact_rel_frob"] = sampled_error(f)
        rs = args.ref_sample or calibrated_sample(w, 10.0)
        t_cpu, threads, desc = oracle_sample_time(w, rs, rs)
        cpu = {"value": 2.0 * rs * w.n * rs / t_cpu / 1e12, "unit": UNIT,
               "cores": threads, "kind": "oracle", "sample": desc}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": gd, "data": "synthetic (seeded; no dataset)",
            "config": _config(w, args),
            "phases_ms": {k_: round(v_, 4) for k_, v_ in phases.items()},
            "roofline": roof, "sketch_rooflines": sketch_roofs, "cpu_baseline": cpu,
            "e2e": {"value": _job_value(flop_eff, e2e_ms, world), "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
            # pack + gather (left), gather (right), GEMM; FP8 adds the two quantisation passes
            "gpu_launches": (6 if sd == "fp8" else 4) * args.steps, "clocks": clk, "error": err, "exact_gemm": exact,
            "forms": forms,
            "plan_ms": _plan_record(plan_s, plan_dev)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# ----------------------------------------------------------------------------
# the other workloads (--workload): parity cases of the suite, measured the same way
# ----------------------------------------------------------------------------

def _time_phases(phases, steps, warmup, world, sample_clocks=True):
    """W untimed warm-up steps, then K timed steps bracketed by a barrier and a
    synchronize, with one CUDA event per phase boundary on the launching stream.
    Returns (ms per step (max over ranks), {phase: mean ms}, clocks)."""
    import torch
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        for _, fn in phases:
            fn()
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(phases) + 1)] for _ in range(steps)]
    clocks = ClockSampler(torch.cuda.current_device()) if sample_clocks else None
    if clocks:
        clocks.start()
        time.sleep(0.3)
    _barrier(world)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for s in range(steps):
        ev[s][0].record(stream)
        for q, (_, fn) in enumerate(phases):
            fn()
            ev[s][q + 1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    _barrier(world)
    clk = clocks.stop() if clocks else None
    total = _max_over_ranks(t0.elapsed_time(t1), world)
    per = {name: statistics.mean(e[q].elapsed_time(e[q + 1]) for e in ev) for q, (name, _) in enumerate(phases)}
    return total / steps, per, clk


def _cpu_leg(args, rank: int, world: int) -> bool:
    """The cpu_baseline leg: rank 0 of a one-GPU run, unless --no-cpu-baseline.
    It is the one place outside --impl reference where bench.py runs the FP64
    oracle: timed on a bounded sample of the workload (cpu_baseline), and, unless
    --no-check, its outputs on that sample set beside the GPU's (error)."""
    return rank == 0 and world == 1 and not args.no_cpu_baseline


def _init_dist():
    """One process per GPU (torchrun's RANK / LOCAL_RANK / WORLD_SIZE, rendezvous at
    MASTER_ADDR); a single process needs no process group."""
    import torch
    world, rank, local = _dist()
    if torch.cuda.is_available():
        torch.cuda.set_device(local if world > 1 else 0)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(_backend())
    return world, rank, local


def _line(args, w_name, value, ms, dtype, config, phases, roof, cpu, e2e, launches, clk, err, world, **extra):
    d = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
         "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
         "vs_baseline": None, "dtype": dtype, "data": "synthetic (seeded; no dataset)", "config": config,
         "phases_ms": {k_: round(v_, 4) for k_, v_ in phases.items()}, "roofline": roof,
         "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk, "error": err}
    d.update(extra)
    return d


def _hbm_roof(peaks, peak_kind, bytes_, ms, kernel):
    ach = bytes_ / (ms * 1e-3) / 1e9
    pk = peaks.get("hbm_gbs")
    return {"bound": "hbm", "achieved": ach, "peak": pk, "unit": "GB/s", "frac": ach / pk, "traffic": None,
            "kernel": kernel, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json)",
            "algorithmic_per_launch": {"bytes": bytes_}}


def run_small(args):
    """The minimum slice (512 x 4096 x 512 FP32, b=256, N=4, e=1, block 2 dropped):
    16 MB of inputs fit in L2, so the step is timed twice -- back to back with
    the inputs warm in L2, and with a 512 MB buffer written between steps (the
    L2 flushed; only the step is inside the events).  `value` is the flushed rate."""
    import torch
    from paper_1811_02653_gb300 import build, ops
    from paper_1811_02653_gb300 import workloads as W
    world, rank, _ = _init_dist()
    build.build()
    w = W.SMALL
    dev = torch.device("cuda", torch.cuda.current_device())
    A_h = torch.from_numpy(w.left()).pin_memory()
    B_h = torch.from_numpy(w.right()).pin_memory()
    A, B = A_h.to(dev), B_h.to(dev)
    plan_s, plan_dev = _time_plans(ops, w, 5)
    p = ops.plan(w.n, w.b, w.N, w.e, w.hash_seed)
    gd = args.dtype
    sd = _sketch_dtype(gd, w.b)
    At, a_sc = ops.sketch_left(p, A, sd)
    BtT, b_sc = ops.sketch_right(p, B, sd)
    C = torch.empty((w.m, w.l), dtype=torch.float32, device=dev)
    ws = torch.empty(max(ops.sketch_workspace(p, w.m), ops.sketch_workspace(p, w.l)), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    phases = [("sketch_left", lambda: ops.sketch_left(p, A, sd, out=At, scales=a_sc, workspace=ws, block_mask=w.mask)),
              ("sketch_right", lambda: ops.sketch_right(p, B, sd, out=BtT, scales=b_sc, block_mask=w.mask,
                                                         workspace=ws)),
              ("gemm_masked", lambda: ops.gemm_masked(p, At, BtT, w.mask, C=C, a_scales=a_sc, b_scales=b_sc,
                                                      dtype=sd))]
    flop = 2.0 * w.m * w.n * w.l
    # warm L2: steps back to back
    warm_ms, warm_per, _ = _time_phases(phases, max(args.steps, 50), args.warmup, world, sample_clocks=False)
    # flushed L2: a 512 MB write between steps, outside the per-step events
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        for _, fn in phases:
            fn()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    _barrier(world)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        for q, (_, fn) in enumerate(phases):
            ev[k][q].record(stream)
            fn()
        ev[k][3].record(stream)
    torch.cuda.synchronize()
    _barrier(world)
    clk = clocks.stop()
    fl_ms = _max_over_ranks(statistics.median(e[0].elapsed_time(e[3]) for e in ev), world)
    fl_per = {name: statistics.median(e[q].elapsed_time(e[q + 1]) for e in ev) for q, (name, _) in enumerate(phases)}
    # the dominant phase of the flushed step against its roofline (algorithmic work)
    peaks, peak_kind = _peaks()
    es = {"bf16": 2, "f32": 4, "fp8": 1, "tf32x2": 8}[sd]
    dom = max(fl_per, key=fl_per.get)
    if dom == "gemm_masked":
        gflop = 2.0 * w.m * w.k * w.b * w.l
        ach = gflop / (fl_per[dom] * 1e-3) / 1e12
        pk = peaks.get("bf16_tflops") * {"bf16": 1.0, "fp8": 2.0, "tf32x2": 1.0 / 6.0}.get(sd, 1.0)
        roof = {"bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                "traffic": None, "kernel": f"masked GEMM ({sd})",
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json)", "algorithmic_per_launch": {"flop": gflop}}
    else:
        rows = w.m if dom == "sketch_left" else w.l
        roof = _hbm_roof(peaks, peak_kind, rows * w.n * 4 + rows * w.k * w.b * es, fl_per[dom],
                         f"{dom} (pack + gather)")
    # end to end through the C ABI with pinned host buffers
    C_h = torch.empty((w.m, w.l), dtype=torch.float32).pin_memory()
    ws_host = torch.empty(ops.matmul_host_workspace(p, w.m, w.l, gemm_dtype=gd), dtype=torch.uint8, device=dev)
    ops.matmul_host(p, A_h, B_h, w.mask, gd, C=C_h, workspace=ws_host)
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(10, args.steps)
    s0.record(stream)
    for _ in range(reps):
        ops.matmul_host(p, A_h, B_h, w.mask, gd, C=C_h, workspace=ws_host)
    s1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = _max_over_ranks(s0.elapsed_time(s1) / reps, world)
    err = cpu = None
    if _cpu_leg(args, rank, world):
        import oracle
        h, s_ = oracle.hash_tables(w.n, w.b, w.N, w.e, w.hash_seed)
        A64, B64 = w.left().astype(np.float64), w.right().astype(np.float64)
        t0 = time.perf_counter()
        reps_cpu = 0
        while time.perf_counter() - t0 < 10.0 or reps_cpu < 1:
            At_r = oracle.sketch_left(A64, h, s_, w.b)
            Bt_c = oracle.sketch_right(B64, h, s_, w.b)
            C_or64 = oracle.masked_product(At_r, Bt_c, w.b, w.mask)
            reps_cpu += 1
        t_cpu = (time.perf_counter() - t0) / reps_cpu
        cpu = {"value": flop / t_cpu / 1e12, "unit": UNIT,
               "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)), "kind": "oracle",
               "sample": f"the whole workload (512x4096x512: both sketches and the masked product in FP64), "
                         f"{reps_cpu} runs"}
        if not args.no_check:
            ops.matmul(p, A, B, w.mask, gd, C=C)
            Cg = C.cpu().numpy().astype(np.float64)
            err = {"vs_oracle_rel_frob": oracle.rel_frob(Cg, _oracle_product_as(oracle, gd, At_r, Bt_c, w.b, w.mask)),
                   "vs_exact_rel_frob": oracle.rel_frob(Cg, A64 @ B64),
                   "oracle_sketch_vs_exact_rel_frob": oracle.rel_frob(C_or64, A64 @ B64),
                   "sample": f"all of C; oracle emulates {gd} operand rounding"}
    cfg = {"workload": w.name, "m": w.m, "n": w.n, "l": w.l, "b": w.b, "N": w.N, "e": w.e,
           "kept_blocks": [j for j in range(w.P) if (w.mask >> j) & 1], "gemm_dtype": gd, "input_dtype": "f32",
           "l2": "inputs (16.8 MB) fit in L2: value is timed with a 512 MB buffer written between steps "
                 "(L2 flushed); warm_l2 gives the back-to-back rate",
           "parallelism": f"replicas{world}"}
    line = _line(args, w.name, _job_value(flop, fl_ms, world), fl_ms, gd, cfg, fl_per, roof, cpu,
                 {"value": _job_value(flop, e2e_ms, world), "unit": UNIT, "ms_per_step": e2e_ms,
                  "h2d_bytes_per_step": A_h.numel() * 4 + B_h.numel() * 4, "d2h_bytes_per_step": C_h.numel() * 4},
                 4 * args.steps, clk, err, world,   # transpose + gather, gather in place, GEMM
                 warm_l2={"ms_per_step": warm_ms, "tflops": _job_value(flop, warm_ms, world),
                          "phases_ms": {k_: round(v_, 4) for k_, v_ in warm_per.items()}},
                 plan_ms=_plan_record(plan_s, plan_dev))
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_hessian(args):
    """H = A D A^T (Sec. 5.2's normal matrix): left sketch with col_scale = sqrt(D),
    then the symmetric masked product (B~ = A~), BF16 operands."""
    import torch
    from paper_1811_02653_gb300 import build, ops
    from paper_1811_02653_gb300 import workloads as W
    world, rank, _ = _init_dist()
    build.build()
    peaks, peak_kind = _peaks()
    w = W.HESSIAN if not args.rows else W.scaled(W.HESSIAN, m=args.rows,
                                                 name=f"hessian rows 0..{args.rows - 1} (profiling size)")
    offs, idx, val = w.left_sparse(range(w.m))
    A = torch.zeros((w.m, w.n), dtype=torch.float32, device="cuda")
    rows_of = torch.repeat_interleave(torch.arange(w.m, device="cuda"), torch.from_numpy(np.diff(offs)).cuda())
    A[rows_of, torch.from_numpy(idx).cuda()] = torch.from_numpy(val).cuda()
    del rows_of, idx, val
    cs_h = w.col_scale()
    cs = torch.from_numpy(cs_h).cuda()
    p = ops.plan(w.n, w.b, w.N, w.e, w.hash_seed)
    if args.dense_sketch:
        ws = torch.empty(ops.sketch_workspace(p, w.m), dtype=torch.uint8, device="cuda")
        At, _ = ops.sketch_left(p, A, "bf16", col_scale=cs, workspace=ws, block_mask=w.mask)
        sk_name, sk_kernel = "sketch_left (pack + weights + gather, col_scale)", "pack_cols_kernel + entry_weights_kernel + sketch_gather_kernel"

        def sketch():
            ops.sketch_left(p, A, "bf16", col_scale=cs, out=At, workspace=ws, block_mask=w.mask)
    else:
        # A is 1% dense: route only its nonzeros (Sec. 4's O(nnz) sketch), one CTA per row
        At, _ = ops.sketch_left_sparse(p, A, "bf16", col_scale=cs, block_mask=w.mask)
        sk_name, sk_kernel = "sketch_left_sparse (col_scale)", "sketch_left_onepass_kernel + sketch_left_sparse_kernel"

        def sketch():
            ops.sketch_left_sparse(p, A, "bf16", col_scale=cs, out=At, block_mask=w.mask)
    H = torch.empty((w.m, w.m), dtype=torch.float32, device="cuda")
    phases = [(sk_name, sketch),
              ("gemm_masked (symmetric: B~ = A~)", lambda: ops.gemm_masked(p, At, At, w.mask, C=H))]
    ms, per, clk = _time_phases(phases, args.steps, args.warmup, world)
    flop_eff = 2.0 * w.m * w.n * w.m
    value = _job_value(flop_eff, ms, world)
    t_sk = per[phases[0][0]]
    sk_bytes = w.m * w.n * 4 + w.n * 4 + w.m * w.k * w.b * 2
    roof = _hbm_roof(peaks, peak_kind, sk_bytes, t_sk, f"{sk_kernel} (left sketch)")
    if not args.dense_sketch:
        roof["traffic"] = TRAFFIC_ONEPASS_304_ROWS * w.m / 304
        roof["traffic_note"] = "sketch_left_onepass_kernel, ncu capture of 304 rows scaled by rows"
    gemm_flop = 2.0 * w.m * w.k * w.b * w.m
    # the symmetric product computes the 256 x 256 tiles on and below the diagonal only
    T = -(-w.m // 256)
    done_flop = gemm_flop * (T * (T + 1) / 2) / (T * T)
    t_g = per[phases[1][0]]
    gemm = {"tflops_effective": gemm_flop / (t_g * 1e-3) / 1e12,
            "tflops_executed": done_flop / (t_g * 1e-3) / 1e12,
            "frac_of_sustained_bf16": done_flop / (t_g * 1e-3) / 1e12 / peaks.get("bf16_tflops_sustained", 1710.4),
            "note": f"lower triangle: {T * (T + 1) // 2} of {T * T} tiles of 256 x 256 computed, then mirrored"}
    err, cpu = None, None
    if _cpu_leg(args, rank, world):
        import oracle
        rows = [r for r in [0, 1, 777, 2048, 3333, 4095] if r < w.m]
        A_r = A[rows].cpu().numpy().astype(np.float64)
        h, s = oracle.hash_tables(w.n, w.b, w.N, w.e, w.hash_seed)
        if not args.no_check:
            At_r = oracle.sketch_left(A_r, h, s, w.b, cs_h.astype(np.float64))
            H_or = oracle.masked_product(oracle.round_bf16(At_r), oracle.round_bf16(At_r).T, w.b, w.mask)
            H_ex = (A_r * cs_h.astype(np.float64) ** 2) @ A_r.T
            H_s = H[rows][:, rows].cpu().numpy().astype(np.float64)
            err = {"vs_oracle_rel_frob": oracle.rel_frob(H_s, H_or), "vs_exact_rel_frob": oracle.rel_frob(H_s, H_ex),
                   "sample": f"{len(rows)}x{len(rows)} entries of H; oracle emulates bf16 operand rounding"}
        nr = 2
        t0 = time.perf_counter()
        At_c = oracle.sketch_left(A_r[:nr], h, s, w.b, cs_h.astype(np.float64))
        oracle.masked_product(At_c, At_c.T, w.b, w.mask)
        t_cpu = time.perf_counter() - t0
        cpu = {"value": 2.0 * nr * w.n * nr / t_cpu / 1e12, "unit": UNIT,
               "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)), "kind": "oracle",
               "sample": f"{nr} rows of A at full n={w.n} with sqrt(D): sketch and the {nr}x{nr} block of H in FP64"}
    cfg = {"workload": w.name, "m": w.m, "n": w.n, "l": w.m, "b": w.b, "N": w.N, "e": w.e,
           "kept_blocks": [j for j in range(w.P) if (w.mask >> j) & 1], "gemm_dtype": "bf16",
           "input_dtype": "f32", "l2": "inputs (17.2 GB) larger than L2; no flush needed",
           "sketch": "dense gather" if args.dense_sketch else "sparse rows", "parallelism": f"replicas{world}"}
    line = _line(args, w.name, value, ms, "bf16", cfg, per, roof, cpu,
                 None, (4 if args.dense_sketch else 3) * args.steps, clk, err, world, gemm=gemm)
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_batched(args):
    """256 uneven products in one CUDA graph (parallel sketch branches, one
    grouped persistent tcgen05 GEMM), autotuned."""
    import torch
    from paper_1811_02653_gb300 import build, ops
    from paper_1811_02653_gb300 import workloads as W
    world, rank, _ = _init_dist()
    build.build()
    peaks, peak_kind = _peaks()
    shapes = W.batched_shapes()
    dev = []
    for q, (m, n, l) in enumerate(shapes):
        A, B = W.batched_device_inputs(shapes, q, "cuda")
        C = torch.empty((m, l), dtype=torch.float32, device="cuda")
        dev.append((A, B, C, ops.plan(n, n // 32, 4, 1, 0), 0b11111 & ~(1 << (q % 5))))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    batch = ops.Batch(dev, tune=not args.no_tune)
    t_create = time.perf_counter() - t0
    info = batch.info()
    ms, per, clk = _time_phases([("graph (sketches + grouped GEMM)", batch.run)], args.steps, args.warmup, world)
    flop_eff = float(sum(2 * m * n * l for m, n, l in shapes))
    value = _job_value(flop_eff, ms, world)
    sk_bytes = sum((m + l) * n * 4 + (m + l) * 4 * (n // 32) * 2 for m, n, l in shapes)
    roof = _hbm_roof(peaks, peak_kind, sk_bytes, ms,
                     "whole graph (pack_cols, sketch_gather, gemm_grouped): sketch bytes / run time")
    gemm_flop = float(sum(2 * m * 4 * (n // 32) * l for m, n, l in shapes))
    err = None
    cpu = None
    if _cpu_leg(args, rank, world):
        import oracle
        sample = [0, 100, 255, max(range(256), key=lambda q: shapes[q][1])]
        worst, t_cpu, flop = 0.0, 0.0, 0.0
        for q in sample:
            A, B, C, p, mask = dev[q]
            m, n, l = shapes[q]
            rows, cols = sorted({0, m // 2, m - 1}), sorted({0, l // 3, l - 1})
            A_r = A[rows].cpu().numpy().astype(np.float64)
            B_c = B[:, cols].cpu().numpy().astype(np.float64)
            t0 = time.perf_counter()
            h, s = oracle.hash_tables(n, n // 32, 4, 1, 0)
            ref = oracle.masked_product(oracle.round_bf16(oracle.sketch_left(A_r, h, s, n // 32)),
                                        oracle.round_bf16(oracle.sketch_right(B_c, h, s, n // 32)), n // 32, mask)
            t_cpu += time.perf_counter() - t0
            flop += 2.0 * len(rows) * n * len(cols)
            worst = max(worst, oracle.rel_frob(C[rows][:, cols].cpu().numpy().astype(np.float64), ref))
        if not args.no_check:
            err = {"vs_oracle_rel_frob_max": worst,
                   "sample": f"3x3 entries of C in products {sample}; oracle emulates bf16 operand rounding"}
        cpu = {"value": flop / t_cpu / 1e12, "unit": UNIT, "cores": int(os.environ.get("OMP_NUM_THREADS",
                                                                                      os.cpu_count() or 1)),
               "kind": "oracle", "sample": f"3x3 entries of C in products {sample}, hash tables, both "
                                           f"sketches and the masked product in FP64 (effective flop 2*3*n*3)"}
    # the same products through oversketch_matmul_batched (caller workspace, masks read on
    # the device): one captured graph replayed with two straggler sets
    batch.close()
    plans = [d[3] for d in dev]
    As, Bs, Cs = [d[0] for d in dev], [d[1] for d in dev], [d[2] for d in dev]
    masks = torch.tensor([d[4] for d in dev], dtype=torch.int64, device="cuda")
    ws = torch.empty(ops.matmul_batched_workspace(plans, [m for m, _, _ in shapes], [n for _, n, _ in shapes],
                                                  [l for _, _, l in shapes]), dtype=torch.uint8, device="cuda")
    ops.matmul_batched(plans, As, Bs, Cs, masks, workspace=ws)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ops.matmul_batched(plans, As, Bs, Cs, masks, workspace=ws)
    shifted = torch.tensor([0b11111 & ~(1 << ((q + 2) % 5)) for q in range(len(dev))], dtype=torch.int64,
                           device="cuda")
    ms_mb, per_mb, _ = _time_phases([("masks p mod 5", lambda: (masks.copy_(torch.tensor([d[4] for d in dev],
                                                                                            dtype=torch.int64)),
                                                                 g.replay())),
                                     ("masks p+2 mod 5", lambda: (masks.copy_(shifted), g.replay()))],
                                    max(2, args.steps // 2), 1, world, sample_clocks=False)
    batched_entry = {"ms_per_run": ms_mb / 2, "phases_ms": {k_: round(v_, 3) for k_, v_ in per_mb.items()},
                     "tflops": _job_value(flop_eff, ms_mb / 2, world), "workspace_bytes": ws.numel(),
                     "what": "oversketch_matmul_batched captured once in a CUDA graph and replayed with two "
                             "device-resident straggler sets (every block sketched, dropped blocks' CTAs return at once)"}
    del ws
    cfg = {"workload": "batched: 256 uneven products, m,l ~ U[256,4096], n log-U[8192,131072], b=n/32, N=4, e=1, "
                       "product p drops block p mod 5", "count": 256,
           "input_bytes": sum((m + l) * n * 4 for m, n, l in shapes), "gemm_dtype": "bf16", "input_dtype": "f32",
           "l2": "inputs (182 GB) larger than L2; no flush needed", "parallelism": f"replicas{world}",
           "graph": {k_: v_ for k_, v_ in info.items()}, "create_s": round(t_create, 2)}
    line = _line(args, cfg["workload"], value, ms, "bf16", cfg, per, roof, cpu, None,
                 info["kernel_launches"] * args.steps, clk, err, world,
                 gemm={"flop_per_run": gemm_flop}, matmul_batched=batched_entry)
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_autograd(args):
    """Forward C = (X S)(S^T G)/k and backward dX, dG through the autograd Function."""
    import torch
    from paper_1811_02653_gb300 import build, ops
    from paper_1811_02653_gb300 import autograd as AG
    from paper_1811_02653_gb300 import workloads as W
    world, rank, _ = _init_dist()
    build.build()
    peaks, peak_kind = _peaks()
    w = W.AUTOGRAD
    X = torch.from_numpy(w.left()).to(torch.bfloat16).cuda().requires_grad_(True)
    G = torch.from_numpy(w.right_cols(range(w.l))).to(torch.bfloat16).cuda().t().contiguous().requires_grad_(True)
    dC = torch.from_numpy(w.upstream_grad()).cuda()
    p = ops.plan(w.n, w.b, w.N, w.e, w.hash_seed)
    state = {}

    def fwd():
        state["C"] = AG.oversketch_matmul(X, G, p, w.mask, args.recompute)

    def bwd():
        X.grad = None
        G.grad = None
        state["C"].backward(dC)

    ms, per, clk = _time_phases([("forward", fwd), ("backward", bwd)], args.steps, args.warmup, world)
    flop_eff = 6.0 * w.m * w.n * w.l          # exact forward + the two exact gradient GEMMs
    value = _job_value(flop_eff, ms, world)
    t_f = per["forward"]
    fwd_bytes = (w.m * w.n + w.n * w.l) * 2 + (w.m + w.l) * w.k * w.b * 2 + w.m * w.l * 4
    roof = _hbm_roof(peaks, peak_kind, fwd_bytes, t_f, "forward: left + right sketch + masked GEMM")
    err, cpu = None, None
    if _cpu_leg(args, rank, world):
        import oracle
        rows, cols = [0, 2048, 4095], [0, 1024, 4095]
        X_r = X.detach()[rows].float().cpu().numpy().astype(np.float64)
        G_c = G.detach()[:, cols].float().cpu().numpy().astype(np.float64)
        t0 = time.perf_counter()
        h, s = oracle.hash_tables(w.n, w.b, w.N, w.e, w.hash_seed)
        ref = oracle.masked_product(oracle.round_bf16(oracle.sketch_left(X_r, h, s, w.b)),
                                    oracle.round_bf16(oracle.sketch_right(G_c, h, s, w.b)), w.b, w.mask)
        t_cpu = time.perf_counter() - t0
        if not args.no_check:
            err = {"forward_vs_oracle_rel_frob": oracle.rel_frob(
                state["C"].detach()[rows][:, cols].cpu().numpy().astype(np.float64), ref),
                "sample": "3x3 entries of C (gradients: tests/test_gpu_autograd.py)"}
        cpu = {"value": 2.0 * len(rows) * w.n * len(cols) / t_cpu / 1e12, "unit": UNIT,
               "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)), "kind": "oracle",
               "sample": "3x3 entries of the forward product at full n: hash tables, both sketches and the "
                         "masked product in FP64 (effective flop 2*3*n*3)"}
    cfg = {"workload": w.name, "m": w.m, "n": w.n, "l": w.l, "b": w.b, "N": w.N, "e": w.e,
           "kept_blocks": [j for j in range(w.P) if (w.mask >> j) & 1], "gemm_dtype": "bf16",
           "input_dtype": "bf16", "recompute": bool(args.recompute),
           "metric_note": "effective flop = 6mnl (forward + dX + dG as exact GEMMs)",
           "l2": "inputs (1.07 GB) larger than L2; no flush needed", "parallelism": f"replicas{world}"}
    # per step: forward pack + gather of X, the in-place gather of G and the masked GEMM
    # (4); backward: dC cast to BF16, two GEMMs reading the sketches and dC MN-major,
    # two unsketch kernels (5); plus the two sketches again (3) with --recompute
    launches = (9 + (3 if args.recompute else 0)) * args.steps
    line = _line(args, w.name, value, ms, "bf16", cfg, per, roof, cpu, None, launches, clk, err, world)
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_lp(args):
    """Sec. 5.2's LP at the paper's proportions: n = 40b constraints, m = 5b
    variables, sketch dimension z = 20b (P = 20 blocks of width b = 1024), Hessian
    blocks b x b.  The timed step is the sketched Hessian A^T D A of one Newton
    iteration (right sketch of A with row scale 1/s, then the per-block masked GEMM
    with one straggler ignored per block); the 100-iteration barrier runs
    (unsketched BF16 Hessian, e = 0, e = 1 per block, e = 1 shared) follow."""
    import torch
    from paper_1811_02653_gb300 import build, lp, ops
    from paper_1811_02653_gb300 import workloads as W
    world, rank, _ = _init_dist()
    build.build()
    peaks, peak_kind = _peaks()
    blk, P = 1024, 20
    NC, MV = 40 * blk, 5 * blk
    nb = MV // blk
    A, bvec, c = W.lp_instance(NC, MV, 1006)
    solver = lp.SketchedBarrierLP(A, bvec, c, blk=blk, N=P - 1, e=1, seed=0)
    del A
    per_block = lambda t: W.straggler_block_masks(P, 1, nb, nb, 11, t)
    shared = lambda t: W.straggler_block_masks(P, 1, nb, nb, 11, t, shared=True)
    runs, x_end = {}, None
    if args.lp_iters > 0:
        solver.solve(iters=3)                  # cuSOLVER / cuBLAS handles and workspaces
    for name, exact, masks in ([("exact_bf16_hessian", True, None), ("e0", False, None),
                                ("e1_per_block", False, per_block), ("e1_shared", False, shared)]
                               if args.lp_iters > 0 else []):
        solver.exact = exact
        x, h = solver.solve(iters=args.lp_iters, block_masks=masks, timing=True)
        if name == "e0":
            x_end = x
        runs[name] = {"final_objective": h.objective[-1], "iter_ms_mean": statistics.mean(h.iter_ms),
                      "hessian_ms_mean": statistics.mean(h.hessian_ms), "shifted_systems": h.shifts,
                      "objective_at_stage_ends": [h.objective[k] for k in range(9, len(h.objective), 10)]}
    if runs:
        f_ref = runs["exact_bf16_hessian"]["final_objective"]
        for r in runs.values():
            r["rel_diff_vs_exact_hessian"] = abs(r["final_objective"] - f_ref) / abs(f_ref)
    if x_end is None:                          # no barrier runs: time the Hessian at x = 0
        x_end = torch.zeros(MV, dtype=torch.float64, device="cuda")
    solver.exact = False
    s = (solver.b - solver.A64 @ x_end)
    d = (1.0 / s).float()
    masks = torch.from_numpy(per_block(0)).cuda()

    def sketch():
        ops.sketch_right(solver.plan, solver.A, "bf16", out=solver.Ask, workspace=solver.ws, row_scale=d)

    def gemm():
        ops.gemm_masked_blocks(solver.plan, solver.Ask, solver.Ask, masks, blk, blk, C=solver.H)

    ms, per, clk = _time_phases([("sketch", sketch), ("gemm", gemm)], args.steps, args.warmup, world)
    value = _job_value(2.0 * MV * MV * NC, ms, world)
    kept = P - 1
    flop = 2.0 * MV * MV * kept * blk
    ach = flop / (per["gemm"] * 1e-3) / 1e12
    pk = peaks.get("bf16_tflops")
    roof_gemm = {"bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                 "frac": ach / pk if pk else None, "traffic": None,
                 "kernel": "gemm_pair_bf16_kernel (BF16, cta_group::2, per-block masks)",
                 "peak_source": f"bf16_tflops burst, {peak_kind} (MEASURED_PEAKS.json)",
                 "algorithmic_per_launch": {"flop": flop, "note": "2 m^2 k b, k = 19 kept blocks per block of H"}}
    # the dominant kernel is the gather: A read once (FP32) and A~ written once (BF16)
    gbytes = NC * MV * 4 + MV * P * blk * 2
    roof = _hbm_roof(peaks, peak_kind, gbytes, per["sketch"],
                     "sketch_gather_kernel (right sketch of A in place, row scale 1/s, BF16 out)")
    roof["l2_gather_tbs"] = P * NC * MV * 4 / (per["sketch"] * 1e-3) / 1e12
    roof["note"] = "every element of A reaches P = 20 buckets, one per sketch block: P |A| leaves the L2"
    cfg = {"workload": f"lp hessian A^T D A, A {NC}x{MV} (n = 40b constraints, m = 5b variables), "
                       f"b={blk}, P={P} (z = 20b), one straggler per Hessian block",
           "n": NC, "m": MV, "b": blk, "P": P, "e_per_block": 1, "gemm_dtype": "bf16", "input_dtype": "f32",
           "metric_note": "effective flop = 2 m^2 n (the exact Hessian)",
           "l2": "A (839 MB FP32) larger than L2; no flush needed", "parallelism": f"replicas{world}",
           "lp_iterations": args.lp_iters, "tau": "1, doubled every 10 iterations"}
    # per step: entry weights + gather (the scaled right sketch), the masked GEMM
    line = _line(args, cfg["workload"], value, ms, "bf16", cfg, per, roof, None, None, 3 * args.steps, clk, None,
                 world, roofline_gemm=roof_gemm, lp_runs=runs)
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_sec51(args):
    """Sec. 5.1's matrix A(x, y) = x + y with B = A^T at the paper's sizes
    (b = 2048, m = l = 10b, n = 60b, sketch dimension z = 30b), e sketch blocks
    ignored per b x b block of C.  The timed step is one product at e = 4 (both
    sketches and the per-block masked GEMM); the mean relative error over ten
    sketch seeds is reported for e = 0 .. 10."""
    import torch
    from paper_1811_02653_gb300 import build, ops
    from paper_1811_02653_gb300 import workloads as W
    world, rank, _ = _init_dist()
    build.build()
    peaks, peak_kind = _peaks()
    blk, P = 2048, 30
    m = l = 10 * blk
    n = 60 * blk
    nb = m // blk
    A, B, AB = W.sec51_device(m, n, "cuda")
    ws = torch.empty(ops.sketch_workspace(ops.plan(n, blk, P - 4, 4, 0), m), dtype=torch.uint8, device="cuda")
    wsr = torch.empty(ops.sketch_workspace(ops.plan(n, blk, P - 4, 4, 0), 0), dtype=torch.uint8, device="cuda")
    state = {}

    def sketches(seed):
        p = ops.plan(n, blk, P - 4, 4, seed)
        state["p"] = p
        state["At"], _ = ops.sketch_left(p, A, "bf16", out=state.get("At"), workspace=ws)
        state["Bt"], _ = ops.sketch_right(p, B, "bf16", out=state.get("Bt"), workspace=wsr)

    ab2 = float(ops.frob(AB, AB)[1])
    rel = {e: [] for e in range(11)}
    for seed in range(10):
        sketches(seed)
        for e in range(11):
            masks = torch.from_numpy(W.straggler_block_masks(P, e, nb, nb, seed, 0)).cuda()
            state["C"] = ops.gemm_masked_blocks(state["p"], state["At"], state["Bt"], masks, blk, blk,
                                                C=state.get("C"))
            rel[e].append(math.sqrt(float(ops.frob(state["C"], AB)[0]) / ab2))
    masks4 = torch.from_numpy(W.straggler_block_masks(P, 4, nb, nb, 0, 0)).cuda()
    sketches(0)
    p = state["p"]

    def left():
        ops.sketch_left(p, A, "bf16", out=state["At"], workspace=ws)

    def right():
        ops.sketch_right(p, B, "bf16", out=state["Bt"], workspace=wsr)

    def gemm():
        ops.gemm_masked_blocks(p, state["At"], state["Bt"], masks4, blk, blk, C=state["C"])

    ms, per, clk = _time_phases([("sketch_left (pack + gather)", left), ("sketch_right (gather in place)", right),
                                 ("gemm_masked_blocks", gemm)], args.steps, args.warmup, world)
    value = _job_value(2.0 * m * n * l, ms, world)
    flop = 2.0 * m * (P - 4) * blk * l
    ach = flop / (per["gemm_masked_blocks"] * 1e-3) / 1e12
    pk = peaks.get("bf16_tflops")
    roof = {"bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk if pk else None,
            "traffic": None, "kernel": "gemm_pair_bf16_kernel (BF16, cta_group::2, per-block masks)",
            "peak_source": f"bf16_tflops burst, {peak_kind} (MEASURED_PEAKS.json)",
            "algorithmic_per_launch": {"flop": flop, "note": "2 m k b l, k = 26 kept blocks per block of C"}}
    err = {"mean_rel_frob_by_e": {e: statistics.mean(v) for e, v in rel.items()},
           "max_rel_frob_by_e": {e: max(v) for e, v in rel.items()},
           "instances": 10, "paper_context": "Fig. 5b: 0.8 % average error with 4 of 30 workers ignored"}
    cpu = None
    if _cpu_leg(args, rank, world):
        import oracle
        U, V = W.sec51_factors(m, n)
        err["expected_rms_rel_by_e"] = {e: math.sqrt(oracle.expected_sq_error_factored(U, V, V, U, P - e, blk)
                                                     / ab2) for e in range(11)}
        rows = [0, m // 2, m - 1]
        A_r = A[rows].cpu().numpy().astype(np.float64)
        t0 = time.perf_counter()
        h, s = oracle.hash_tables(n, blk, P - 4, 4, 0)
        At_r = oracle.sketch_left(A_r, h, s, blk)
        oracle.masked_product(At_r, np.ascontiguousarray(At_r.T), blk, (1 << P) - 1 - 0b1111)
        t_cpu = time.perf_counter() - t0
        cpu = {"value": 2.0 * len(rows) * n * len(rows) / t_cpu / 1e12, "unit": UNIT,
               "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)), "kind": "oracle",
               "sample": "3 rows of A (B = A^T: the same 3 columns of B) at full n: hash tables, sketch and the "
                         "3x3 masked product in FP64 (effective flop 2*3*n*3)"}
    cfg = {"workload": f"sec 5.1: A(x,y) = x+y {m}x{n}, B = A^T; b={blk}, P={P} (z = 30b); "
                       f"4 of 30 blocks ignored per {blk}x{blk} block of C",
           "m": m, "n": n, "l": l, "b": blk, "P": P, "e_per_block": 4, "gemm_dtype": "bf16", "input_dtype": "f32",
           "l2": "A and B (10 GB each) larger than L2; no flush needed", "parallelism": f"replicas{world}"}
    # transpose + gather (left), gather in place (right), per-block GEMM
    line = _line(args, cfg["workload"], value, ms, "bf16", cfg, per, roof, cpu, None, 4 * args.steps, clk, err,
                 world)
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dtype", default="bf16", choices=["bf16", "f32", "fp8"])
    ap.add_argument("--ref-sample", type=int, default=0, help="oracle sample rows (0: calibrate)")
    ap.add_argument("--shape", default="", help="m,n,l override for profiling captures")
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-exact", action="store_true", help="skip the exact-GEMM comparison")
    ap.add_argument("--no-forms", action="store_true", help="square: skip timing the other GEMM dtypes")
    ap.add_argument("--workload", default="square",
                    choices=["square", "small", "hessian", "batched", "autograd", "lp", "sec51"],
                    help="square (default: the headline line), or another workload of the suite")
    ap.add_argument("--no-tune", action="store_true", help="batched: skip the autotuner")
    ap.add_argument("--recompute", action="store_true", help="autograd: recompute the sketches in backward")
    ap.add_argument("--dense-sketch", action="store_true", help="hessian: sketch A with the dense gather path")
    ap.add_argument("--rows", type=int, default=0, help="hessian: the first ROWS rows of A only (profiling size)")
    ap.add_argument("--lp-iters", type=int, default=100,
                    help="lp: barrier iterations per run (0: time the Hessian at x = 0 only)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "small":
        return run_small(args)
    if args.workload == "hessian":
        return run_hessian(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "autograd":
        return run_autograd(args)
    if args.workload == "lp":
        return run_lp(args)
    if args.workload == "sec51":
        return run_sec51(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
