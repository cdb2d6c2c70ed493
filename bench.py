#!/usr/bin/env python
"""Benchmark of the sliced tensor-network contraction on GB300.

Workload (default "c3"): the 42-qubit 6x7-grid circuit with 16 cycles, its
tree sliced into 2^12 slices with intermediates <= 2^28 complex64, all 4096
slices contracted per step, 12 open qubits (4096 correlated amplitudes), XEB of
the batch.  One step = tn_contract_slices over every slice + tn_xeb.

value  : slices/s over the whole job, device-timed (CUDA events), inputs resident.
e2e    : the same through the public API with host buffers: the batch's
         bitstrings from pinned host memory in, amplitudes + XEB back to host.
Also reported: complex TFLOP/s, the FP32 SIMT path on the same plan, relative
amplitude and XEB error against the oracle's stored amplitudes, the roofline of
the dominant kernel, SM clocks sampled during the timed region, and the oracle
timed on the host cores (cpu_baseline).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Multi-GPU (one process per GPU via torchrun): each rank contracts every slice
for its own bitstring batch (independent problems, weak scaling), no collective
on the data path; a barrier and a max over ranks bracket the timing.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import rqcgen  # noqa: E402

L2_FLUSH_BYTES = 512 << 20          # larger than the 129 MB L2

# per workload: slices contracted per step (None: all) and slices per chunk (0: planner's choice)
WORKLOAD_RUN = {
    "c1": dict(step_slices=None, log2_batch=0),
    "c2": dict(step_slices=None, log2_batch=0),
    "c3": dict(step_slices=None, log2_batch=0, trials=128),
    # 2^20+ slices: one seeded aligned block of 1024 slices per step; every slice
    # has the same cost, so the full task's time is T_block * 2^S / 1024
    "c5": dict(step_slices=1024, log2_batch=10, trials=128, arena_gib=160),
}


# ------------------------------------------------------------------ multi-process helpers
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def batch_bits_for_rank(name: str, rank: int) -> int:
    """Closed bits of the batch a rank contracts: rank 0 takes the workload's own
    bitstring, rank r > 0 an independent one drawn from (seed, stream r + 1)."""
    circ, om, cb = rqcgen.config_circuit(name)
    if rank == 0:
        return cb
    return rqcgen.random_bits(circ.n_qubits, rqcgen.CONFIGS[name]["seed"], stream=rank + 1) & ~om


def max_over_ranks(value: float, world: int, device=None) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((float(r[3]) for r in rows if r[3].replace(".", "").isdigit()), default=None)}


# ------------------------------------------------------------------ oracle (CPU) timing
ORACLE_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import rqcgen
from oracle import tensornet
circ, om, cb = rqcgen.config_circuit({name!r})
net = tensornet.CircuitNetwork(circ, cb, om)
t0 = time.time()
merges, extra = net.plan([], max_log2={maxlog!r}, method="bisect", trials={trials!r})
plan_s = time.time() - t0
budget = {budget!r}
steps = []
done = 0
for s in range({n_steps!r}):
    # one step: at least one sub-network, then more until the step's budget is spent
    cnt, t_run = 0, 0.0
    while (cnt == 0 or t_run < budget):
        values = {{leg: ((done % (1 << len(extra))) >> j) & 1 for j, leg in enumerate(extra)}}
        t1 = time.time()
        net._run(merges, values)
        t_run += time.time() - t1
        done += 1
        cnt += 1
    steps.append([t_run, cnt])
print(json.dumps({{"sub_networks": 1 << len(extra), "steps": steps, "plan_s": plan_s}}))
"""


def oracle_timing(name: str, budget_s: float, n_steps: int = 1) -> dict:
    """Time the FP64 oracle on bounded samples: the oracle contracts the whole
    batch as 2^E sub-networks of its own (its sub-slicing); each of n_steps
    samples runs at least one of them and more within budget_s, and its
    full-batch time is extrapolated from the sample."""
    code = ORACLE_SNIPPET.format(root=ROOT, name=name, maxlog=26, trials=4, budget=budget_s, n_steps=n_steps)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=3600)
    if r.returncode != 0:
        return {"error": r.stderr.strip()[-400:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    per_step = [sec / cnt * d["sub_networks"] for sec, cnt in d["steps"]]
    return {"full_batch_seconds": per_step[-1], "step_full_batch_seconds": per_step,
            "timed_sub_networks": sum(cnt for _, cnt in d["steps"]), "sub_networks": d["sub_networks"],
            "seconds": sum(sec for sec, _ in d["steps"])}


def cores_used() -> int:
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(var, "").isdigit():
            return int(os.environ[var])
    return os.cpu_count() or 1


# ------------------------------------------------------------------ rooflines
FP32_SIMT_TFLOPS = 152 * 128 * 2 * 1.92 / 1e3   # SMs x FP32 lanes x 2 flops x GHz under load

# DRAM bytes (read + write) per launch from ncu captures of the current kernels,
# keyed by (kernel, log2 m,k,n,batch); see profiles/ for the command and scaling.
MEASURED_TRAFFIC = {
    # 4 x the 8-instance proxy capture (profiles/tc_bf16x3_12x12x8_batch8.md: 1320.1 MB)
    ("tc_bf16x3", (12, 12, 8, 5)): 5.2804e9,
}


def load_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        d["source"] = "measured"
        return d
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


def complex_peak_tflops(kernel: str, peaks: dict) -> float:
    """Peak in algorithmic complex flops (8 per complex multiply-add) of a kernel:
    a real tensor peak P runs a complex MAC as R real MACs, so P_eff = P * 8 / (2 R)."""
    bf16 = peaks["bf16_tflops"]
    real = {"tc_tf32": (bf16 / 2, 4),          # TF32 dense = half the BF16 rate, 4M
            "tc_tf32_3m": (bf16 / 2, 3),
            "tc_bf16x3": (bf16, 12),           # 3 bf16 products per real product, 4M
            "tc_bf16x3_3m": (bf16, 9),
            "tc_fp16x3": (bf16, 12),           # FP16 dense runs at the BF16 rate
            "tc_fp16x3_3m": (bf16, 9)}
    if kernel in real:
        p, r = real[kernel]
        return p * 8 / (2 * r)
    return FP32_SIMT_TFLOPS


def step_roofline(shape, ms: float, kernel: str, peaks: dict) -> dict:
    m, k, n, b = shape
    flops = 8.0 * 2 ** (m + k + n + b)
    nbytes = 8.0 * (2 ** (m + k) + 2 ** (k + n) + 2 ** (m + n)) * 2 ** b
    p_tf = complex_peak_tflops(kernel, peaks)
    bw = peaks["hbm_gbs"]
    t_c = flops / (p_tf * 1e12) * 1e3
    t_m = nbytes / (bw * 1e9) * 1e3
    if t_c >= t_m:
        bound = "tensor" if kernel.startswith("tc") else "alu"
        ach = flops / (ms / 1e3) / 1e12
        r = {"bound": bound, "achieved": ach, "peak": p_tf, "unit": "TFLOP/s", "frac": ach / p_tf}
    else:
        ach = nbytes / (ms / 1e3) / 1e9
        r = {"bound": "hbm", "achieved": ach, "peak": bw, "unit": "GB/s", "frac": ach / bw}
    r.update({"traffic": MEASURED_TRAFFIC.get((kernel, (m, k, n, b))), "kernel": kernel,
              "shape_log2_mknb": [m, k, n, b], "ms": ms,
              "t_roof_ms": max(t_c, t_m), "peak_source": peaks.get("source", "measured")})
    return r


# ------------------------------------------------------------------ one pairwise contraction
def pair_bench(args) -> int:
    """Time tn_contract_pair on random operands of shape (m, k, n) with a
    seeded random storage order of every operand (the permutation is folded
    into the kernel's loads)."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2111_01066_gb300 import tn
    vals = [int(x) for x in args.pair.split(",")]
    m, k, n = vals[:3]
    batch = vals[3] if len(vals) > 3 else 1
    prec = args.precision if args.precision != "auto" else "bf16x3"
    rng = np.random.default_rng(m * 10000 + k * 100 + n)
    wires = list(range(m + k + n))
    mw, kw, nw = wires[:m], wires[m:m + k], wires[m + k:]
    a_w = {"random": list(rng.permutation(mw + kw)), "kfast": kw + mw, "mfast": mw + kw}[args.layout]
    b_w = list(rng.permutation(kw + nw)) if args.layout == "random" else kw + nw
    c_w = mw + nw
    dev = torch.device("cuda", 0)
    a = torch.randn(batch, 2 ** (m + k), dtype=torch.complex64, device=dev)
    b = torch.randn(batch, 2 ** (k + n), dtype=torch.complex64, device=dev)
    c = torch.empty(batch, 2 ** (m + n), dtype=torch.complex64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 1)):
        tn.contract_pair(a, a_w, b, b_w, c, c_w, batch=batch, precision=prec, stream=stream)
    torch.cuda.synchronize()
    times = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tn.contract_pair(a, a_w, b, b_w, c, c_w, batch=batch, precision=prec, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = statistics.mean(times)
    peaks = load_peaks()
    kernel = {"fp32": "simt", "tf32": "tc_tf32", "bf16x3": "tc_bf16x3"}[prec]
    if prec != "fp32" and (m + k + n + int(math.log2(batch)) < 20 or m < 4):
        kernel = "simt"
    r = step_roofline((m, k, n, int(round(math.log2(batch)))), ms, kernel, peaks)
    print(json.dumps({"metric": "pair_contraction", "shape_log2_mkn": [m, k, n], "batch": batch,
                      "layout": args.layout,
                      "precision": prec, "ms": ms, "complex_tflops": 8.0 * 2 ** (m + k + n) * batch / ms / 1e9,
                      "roofline": r, "note": "includes the B' image pre-pass for tensor-core kernels"}))
    return 0


# ------------------------------------------------------------------ kernel sweep
def _event_ms(fn, reps, flush, stream):
    import torch
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def sweep_bench(args) -> int:
    """Kernel sweep: every (m, k, n) in {2^4, 2^6, ..., 2^14}^3 whose operands stay
    within 2^30 complex elements, in FP32, TF32, BF16x3, FP16x3 and BF16x3 3M (A
    stored [k, m] so tensor-core runs fetch it by TMA), plus every distinct step
    shape of the C2, C3 and C5 plans (BF16x3), or random permutations of rank 20..30
    (8 seeded permutations per rank plus the full reversal).  One JSON line per
    case goes to --sweep-out; stdout gets a summary line."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2111_01066_gb300 import tn
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    peaks = load_peaks()
    rows = []
    if args.sweep == "gemm":
        modes = [("fp32", 4), ("tf32", 4), ("bf16x3", 4), ("fp16x3", 4), ("bf16x3", 3)]
        kname = {("fp32", 4): "simt", ("tf32", 4): "tc_tf32", ("bf16x3", 4): "tc_bf16x3",
                 ("fp16x3", 4): "tc_fp16x3", ("bf16x3", 3): "tc_bf16x3_3m"}

        def run_case(m, k, n, b, modes_here, source):
            mw, kw, nw = list(range(m)), list(range(m, m + k)), list(range(m + k, m + k + n))
            batch = 1 << b
            a = torch.randn(batch, 2 ** (m + k), dtype=torch.complex64, device=dev)
            bb = torch.randn(batch, 2 ** (k + n), dtype=torch.complex64, device=dev)
            cc = torch.empty(batch, 2 ** (m + n), dtype=torch.complex64, device=dev)
            for prec, cm in modes_here:
                fn = lambda: tn.contract_pair(a, kw + mw, bb, kw + nw, cc, mw + nw, batch=batch, precision=prec,
                                              complex_mult=cm, stream=stream)
                ms = _event_ms(fn, 2, flush, stream)
                kern = kname[(prec, cm)]
                if prec != "fp32" and (m + k + n + b < 20 or m < 4):
                    kern = "simt"
                r = step_roofline((m, k, n, b), ms, kern, peaks)
                rows.append({"case": "gemm", "source": source, "mknb_log2": [m, k, n, b], "precision": prec,
                             "complex_mult": cm, "ms": ms,
                             "complex_tflops": 8.0 * 2 ** (m + k + n + b) / ms / 1e9, "bound": r["bound"],
                             "frac": r["frac"], "kernel": kern})
            del a, bb, cc

        sizes = [4, 6, 8, 10, 12, 14]
        for m in sizes:
            for k in sizes:
                for n in sizes:
                    if m + k > 30 or k + n > 30 or m + n > 30:
                        continue
                    run_case(m, k, n, 0, modes, "grid")
        # every distinct step shape of the C2, C3 and C5 plans the benchmark uses (batched as in
        # the plan), in the default BF16x3 4M mode
        shapes = set()
        for name in ("c2", "c3", "c5"):
            cfg = rqcgen.CONFIGS[name]
            run = WORKLOAD_RUN[name]
            circ, om, _ = rqcgen.config_circuit(name)
            pl = tn.Plan(tn.Network(circ), open_mask=om, max_log2_intermediate=cfg["log2_bound"],
                         min_log2_slices=cfg.get("log2_slices", 0), log2_batch_slices=run["log2_batch"],
                         trials=run.get("trials", 64), max_arena_bytes=int(run.get("arena_gib", 96)) << 30,
                         precision="bf16x3")
            shapes |= {s for s in pl.step_shapes() if sum(s) >= 20 and s[0] >= 4}
        for (m, k, n, b) in sorted(shapes):
            if 2 ** (m + k + b) > 2 ** 31 or 2 ** (m + n + b) > 2 ** 31:
                continue
            run_case(m, k, n, b, [("bf16x3", 4)], "plans")
    else:
        rng = np.random.default_rng(4)
        for rank in (20, 22, 24, 26, 28, 30):
            x = torch.randn(2 ** rank, dtype=torch.complex64, device=dev)
            y = torch.empty_like(x)
            perms = [list(rng.permutation(rank)) for _ in range(8)] + [list(range(rank - 1, -1, -1))]
            for i, perm in enumerate(perms):
                ms = _event_ms(lambda: tn.permute(x, y, rank, perm, 1, stream), 3, flush, stream)
                gbs = 16.0 * 2 ** rank / ms / 1e6
                rows.append({"case": "permute", "rank": rank, "perm": i if i < 8 else "reverse", "ms": ms,
                             "gbs": gbs, "frac": gbs / peaks["hbm_gbs"]})
            del x, y
    if args.sweep_out:
        with open(args.sweep_out, "w") as f:
            for r in rows:
                f.write(json.dumps(r) + "\n")
    fr = [r["frac"] for r in rows]
    summ = {"metric": f"{args.sweep}_sweep", "cases": len(rows), "frac_median": statistics.median(fr),
            "frac_min": min(fr), "frac_max": max(fr)}
    if args.sweep == "gemm":
        for prec, cm in (("fp32", 4), ("tf32", 4), ("bf16x3", 4), ("fp16x3", 4), ("bf16x3", 3)):
            tag = prec if cm == 4 else prec + "_3m"
            big = [r for r in rows if r["precision"] == prec and r["complex_mult"] == cm and r["source"] == "grid"
                   and sum(r["mknb_log2"]) >= 30]
            if big:
                summ[f"{tag}_median_frac_large"] = statistics.median(r["frac"] for r in big)
                summ[f"{tag}_max_tflops"] = max(r["complex_tflops"] for r in big)
        pl_rows = [r for r in rows if r["source"] == "plans"]
        if pl_rows:
            summ["plan_shapes"] = len(pl_rows)
            summ["plan_shapes_median_frac"] = statistics.median(r["frac"] for r in pl_rows)
    print(json.dumps(summ))
    return 0


# ------------------------------------------------------------------ main
def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=sorted(rqcgen.CONFIGS))
    ap.add_argument("--precision", default="auto")
    ap.add_argument("--select", type=int, default=6,
                    help="candidate plans timed by tn_plan_select before the run (<= 1: one plan)")
    ap.add_argument("--complex-mult", type=int, default=4, choices=[3, 4],
                    help="4M or 3M complex products on the tensor cores")
    ap.add_argument("--compare-fp32", type=int, default=1)
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--autotune", type=int, default=1, help="tune kernels per step before timing")
    ap.add_argument("--pair", default=None,
                    help="log2 m,k,n[,batch]: time one pairwise contraction (tn_contract_pair) instead")
    ap.add_argument("--sweep", default=None, choices=["gemm", "permute"],
                    help="kernel sweep: complex GEMMs m,k,n in 2^4..2^14 (3 precisions) or rank-20..30 permutations")
    ap.add_argument("--sweep-out", default=None, help="file for the sweep's per-case JSON lines")
    ap.add_argument("--layout", default="random", choices=["random", "kfast", "mfast"],
                    help="storage order of A in --pair mode: seeded random, contracted wires lowest, "
                         "free wires lowest")
    args = ap.parse_args()
    if args.pair:
        return pair_bench(args)
    if args.sweep:
        return sweep_bench(args)
    rank, world, local = dist_env()
    name = args.workload
    cfg = rqcgen.CONFIGS[name]
    circ, om, _ = rqcgen.config_circuit(name)
    n_slices = None

    if args.impl == "reference":
        if rank != 0:
            return 0
        # W warm-up + K timed bounded samples, each at least one oracle sub-network,
        # the whole run sized to a few minutes
        n_all = args.warmup + args.steps
        t = oracle_timing(name, max(1.0, min(args.cpu_budget, 180.0 / max(1, n_all))), n_all)
        total_slices = 1 << cfg["log2_slices"]
        steps = []
        if "error" not in t:
            steps = t["step_full_batch_seconds"][args.warmup:]
        mean_s = statistics.mean(steps) if steps else None
        value = total_slices / mean_s if steps else None
        # n_gpus is the launch's N (the line pairs with this arm's own line at
        # that N); the oracle itself runs on the host cores of rank 0 only
        line = {"impl": "reference", "metric": "slices/s", "value": value, "unit": "slices/s", "n_gpus": args.gpus,
                "device": "host cores (FP64 oracle)",
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": (mean_s * 1e3 if steps else None),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": f"{name}: {circ.n_qubits}-qubit {cfg['rows']}x{cfg['cols']} grid, "
                                       f"{cfg['cycles']} cycles, 2^{cfg['log2_slices']} slices (<=2^"
                                       f"{cfg['log2_bound']} per slice), {cfg['k_open']} open qubits"},
                "cpu_baseline": {"value": value, "unit": "slices/s", "cores": cores_used(), "kind": "oracle",
                                 "sample": f"{args.warmup} + {args.steps} samples, {t.get('timed_sub_networks')} of "
                                           f"{t.get('sub_networks')} oracle sub-networks of the full {total_slices}-slice "
                                           f"batch in all ({t.get('seconds', 0):.1f} s), each extrapolated"},
                "e2e": {"value": value, "unit": "slices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        if "error" in t:
            line["unavailable"] = "oracle failed: " + t["error"]
        print(json.dumps(line))
        return 0

    import numpy as np
    import torch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    barrier(world)
    from paper_2111_01066_gb300 import tn
    tn.load()

    prec = args.precision if args.precision != "auto" else "bf16x3"
    bits = batch_bits_for_rank(name, rank)
    net = tn.Network(circ)
    run = WORKLOAD_RUN[name]
    plan_kw = dict(open_mask=om, max_log2_intermediate=cfg["log2_bound"], min_log2_slices=cfg["log2_slices"],
                   log2_batch_slices=run["log2_batch"], trials=run.get("trials", 64),
                   max_arena_bytes=int(run.get("arena_gib", 96)) << 30)
    t_plan = time.time()
    selection = None
    if args.select > 1:
        # plan selection by measured time over candidate orders (untimed)
        plan, est = tn.select_plan(net, args.select, bits, precision=prec, complex_mult=args.complex_mult,
                                   **plan_kw)
        ch = int(min(range(len(est)), key=lambda i: est[i] if est[i] > 0 else float("inf")))
        selection = {"candidates": args.select, "estimated_seconds_all_slices": est, "chosen": ch}
        # the chosen candidate's options (seed + i, memory weight 32 x (1, 1/4, 4)[i % 3]), so
        # that the comparison paths below contract the same order
        plan_kw = dict(plan_kw, seed=1 + ch, mem_weight=32.0 * (1.0, 0.25, 4.0)[ch % 3])
    else:
        plan = tn.Plan(net, precision=prec, complex_mult=args.complex_mult, **plan_kw)
    t_plan = time.time() - t_plan
    info = plan.info()
    all_slices = 1 << info["log2_slices"]
    n_slices = all_slices if run["step_slices"] is None else min(all_slices, run["step_slices"])
    first = 0
    if n_slices < all_slices:
        import numpy as _np
        blocks = all_slices // n_slices
        first = int(_np.random.default_rng([cfg["seed"], 13]).integers(blocks)) * n_slices
    k_open = info["n_open"]
    n_chunks = max(1, n_slices >> info["log2_batch_slices"])
    out = torch.zeros(2 << k_open, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step(p, o):
        o.zero_()
        p.contract_slices(first, n_slices, [bits], o, stream)
        return tn.xeb(o.view(torch.complex128), circ.n_qubits, stream)

    def timed(p, o, k, w, mark=False):
        for _ in range(w):
            step(p, o)
        torch.cuda.synchronize()
        times = []
        for _ in range(k):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            if mark:   # NVTX range of the timed steps (a profiler can capture just these)
                torch.cuda.nvtx.range_push("timed_step")
            e0.record(stream)
            step(p, o)
            e1.record(stream)
            if mark:
                torch.cuda.nvtx.range_pop()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        return times

    # untimed first call: device state + warm-up; then the per-step autotuner
    step(plan, out)
    torch.cuda.synchronize()
    t_tune = time.time()
    if args.autotune:
        plan.autotune(reps=2, stream=stream)
        step(plan, out)
        torch.cuda.synchronize()
    t_tune = time.time() - t_tune
    barrier(world)
    clocks = ClockSampler(local)
    clocks.start()
    times = timed(plan, out, args.steps, args.warmup, mark=True)
    clk = clocks.stop()
    barrier(world)
    ms = statistics.mean(times)
    ms_max = max_over_ranks(ms, world, dev)
    total_units = n_slices * world
    value = total_units / (ms_max / 1e3)
    amps = out.cpu().numpy().view(np.complex128).copy()
    f_xeb = tn.xeb(out.view(torch.complex128), circ.n_qubits)

    # e2e: host bitstrings in, host amplitudes + XEB out, wall clock
    host_amps = torch.empty(2 << k_open, dtype=torch.float64, pin_memory=True)
    e2e_times = []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out.zero_()
        plan.contract_slices(first, n_slices, [bits], out, stream)
        host_amps.copy_(out, non_blocking=True)
        tn.xeb(out.view(torch.complex128), circ.n_qubits, stream)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_times.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(statistics.mean(e2e_times), world, dev)

    # the other paths on the same workload: FP32 SIMT (the plain path) and TF32
    others = {}
    gold = None
    # stored oracle results (text files written by tests/golden/make_golden.py):
    # the batch's amplitudes and their linear XEB
    gold_path = os.path.join(ROOT, "tests", "golden", f"{name}_amplitudes.txt")
    gold_xeb_path = os.path.join(ROOT, "tests", "golden", f"{name}_xeb.txt")
    gold_xeb = None
    if rank == 0 and os.path.exists(gold_path) and os.path.exists(gold_xeb_path):
        g = np.loadtxt(gold_path, comments="#")
        gold = g[:, 0] + 1j * g[:, 1]
        gold_xeb = float(np.loadtxt(gold_xeb_path, comments="#"))

    def amp_error(o):
        if gold is None or gold.size != (o.numel() // 2) or n_slices != all_slices:
            return None
        got = o.cpu().numpy().view(np.complex128)
        f = tn.xeb(o.view(torch.complex128), circ.n_qubits)
        return {"rel_amp_err": float(np.linalg.norm(got - gold) / np.linalg.norm(gold)),
                "xeb_err": abs(f - gold_xeb)}

    if args.compare_fp32:
        # the plain FP32 path, TF32, and the other complex product (4M / 3M) of this precision
        alts = [("fp32", 4), ("tf32", 4)]
        if prec in ("tf32", "bf16x3", "fp16x3"):
            alts.append((prec, 7 - args.complex_mult))
        for other, ocm in alts:
            if (other, ocm) == (prec, args.complex_mult):
                continue
            p2 = tn.Plan(net, precision=other, complex_mult=ocm, **plan_kw)
            o2 = torch.zeros_like(out)
            step(p2, o2)
            if args.autotune:
                p2.autotune(reps=1, stream=stream)
                o2.zero_()
                step(p2, o2)
            t2 = timed(p2, o2, min(3, args.steps), 1)
            ms2 = max_over_ranks(statistics.mean(t2), world, dev)
            others[other if ocm == 4 else other + "_3m"] = {"precision": other, "complex_mult": ocm,
                                                             "value": total_units / (ms2 / 1e3), "ms_per_step": ms2,
                             "error_vs_oracle": amp_error(o2)}
            del p2, o2
    fp32 = others.get("fp32")

    # roofline of the dominant kernel: per-step device times on the same stream
    st = plan.step_times(reps=3, stream=stream)
    shapes = plan.step_shapes()
    peaks = load_peaks()
    rows = [step_roofline(shapes[i], st[i][0], st[i][1], peaks) for i in range(len(st))]
    i_dom = max(range(len(rows)), key=lambda i: rows[i]["ms"])
    roof = dict(rows[i_dom])
    roof["share_of_step_time"] = rows[i_dom]["ms"] / sum(r["ms"] for r in rows)
    roof["step"] = i_dom
    # whole-path roofline: sum over steps of max(flops / peak, bytes / bandwidth)
    t_roof = sum(r["t_roof_ms"] for r in rows)
    path_roof = {"t_roof_ms": t_roof, "t_steps_ms": sum(r["ms"] for r in rows),
                 "frac": t_roof / sum(r["ms"] for r in rows)}
    top = sorted(rows, key=lambda r: -r["ms"])[:8]

    err = amp_error(out) if rank == 0 else None

    # frugal sampling within the batch (main text, section III): with the whole
    # slice sum in hand, draw 2^k samples (128 uniform proposals each, M = 10)
    # and take the linear XEB of the samples (1 for an ideal sampler)
    frugal = None
    if rank == 0 and n_slices == all_slices:
        m_bound, draws, n_samp = 10.0, 128, 1 << k_open
        rs = np.random.default_rng([cfg["seed"], 17])
        cand = torch.from_numpy(rs.integers(0, 1 << k_open, size=(n_samp, draws))).to(dev)
        unif = torch.from_numpy(rs.random((n_samp, draws))).to(dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        first_draw = tn.frugal_sample(out.view(torch.complex128), circ.n_qubits, m_bound, cand, unif, stream)
        t_samp = time.perf_counter() - t0
        idx = [int(cand[s, t]) for s, t in enumerate(first_draw) if t >= 0]
        picked = out.view(torch.complex128)[torch.tensor(idx, device=dev)]
        # what an exact sampler of this batch gives: E[N p] under min(1, N p / M)
        x = np.ldexp(np.abs(amps) ** 2, circ.n_qubits)
        w = np.minimum(1.0, x / m_bound)
        frugal = {"samples": len(idx), "proposals_per_sample": draws, "m_bound": m_bound,
                  "sampled_xeb": tn.xeb(picked, circ.n_qubits),
                  "expected_sampled_xeb": float(np.sum(w * x) / np.sum(w) - 1.0), "ms": t_samp * 1e3}
    # time per perfect sample (main text, section III): one batch of 2^6
    # amplitudes over all slices yields a sample with probability
    # 1 - (1 - E[min(1, x / M)])^64, x ~ Exp(1) (Porter-Thomas), M = 10
    per_sample = None
    if k_open == 6:
        p_accept = (1 - math.exp(-10.0)) / 10.0
        p_batch = 1 - (1 - p_accept) ** 64
        t_batch = all_slices / value * world
        per_sample = {"batch_seconds": t_batch, "p_sample_per_batch": p_batch,
                      "seconds_per_perfect_sample": t_batch / p_batch,
                      "days_for_1M_samples_at_xeb_0.002": 2000 * t_batch / p_batch / 86400,
                      "note": "extrapolated from the timed slice block; 1M samples at fidelity 0.002 "
                              "cost as much as 2000 perfect samples (main text, section III)"}

    cpu = None
    if rank == 0 and world == 1 and args.cpu_budget > 0:
        t = oracle_timing(name, args.cpu_budget)
        if "error" not in t:
            cpu = {"value": n_slices / t["full_batch_seconds"], "unit": "slices/s", "cores": cores_used(),
                   "kind": "oracle",
                   "sample": f"{t['timed_sub_networks']} of {t['sub_networks']} oracle sub-networks of the "
                             f"full {n_slices}-slice batch ({t['seconds']:.1f} s), extrapolated"}
        else:
            cpu = {"value": None, "unit": "slices/s", "cores": cores_used(), "kind": "oracle",
                   "sample": "oracle failed: " + t["error"][-200:]}

    if rank == 0:
        line = {
            "metric": "slices/s", "value": value, "unit": "slices/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp32": "f32", "tf32": "tf32", "bf16x3": "bf16x3",
                                           "fp16x3": "fp16x3"}[prec],
            "data": "synthetic",
            "config": {"workload": f"{name}: {circ.n_qubits}-qubit {cfg['rows']}x{cfg['cols']} grid, "
                                   f"{cfg['cycles']} cycles, 2^{info['log2_slices']} slices (<=2^"
                                   f"{cfg['log2_bound']} per slice), {k_open} open qubits",
                       "precision": prec, "complex_mult": info["complex_mult"],
                       "slices_per_step": n_slices, "chunks_per_step": n_chunks, "slice_first": first,
                       "slices_total": all_slices,
                       "log2_batch_slices": info["log2_batch_slices"], "l2": "flushed between steps "
                       "(512 MiB write); intermediates also exceed L2"},
            "complex_tflops": info["flops_per_chunk"] * n_chunks * world / (ms_max / 1e3) / 1e12,
            "complex_tflops_per_slice_basis": info["flops_per_slice"] * total_units / (ms_max / 1e3) / 1e12,
            "plan": {"flops_per_slice": info["flops_per_slice"], "flops_per_chunk": info["flops_per_chunk"],
                     "bytes_per_chunk": info["bytes_per_chunk"], "n_steps": info["n_steps"],
                     "log2_max_intermediate": info["log2_max_intermediate"], "arena_gib": info["arena_bytes"] / 2**30,
                     "plan_seconds": t_plan, "autotune_seconds": t_tune if args.autotune else None},
            "extrapolated_full_task_s": all_slices / value * world if n_slices < all_slices else None,
            "fp32_path": fp32,
            "tf32_path": others.get("tf32"),
            "other_complex_mult_path": others.get(prec + "_3m") if args.complex_mult == 4 else others.get(prec),
            "speedup_vs_fp32_path": (value / fp32["value"]) if fp32 else None,
            "error_vs_oracle": err,
            "xeb": f_xeb,
            "plan_selection": selection,
            "frugal_sampling": frugal,
            "perfect_sample": per_sample,
            "roofline": roof,
            "path_roofline": path_roof,
            "top_steps": top,
            "clocks": clk,
            "e2e": {"value": total_units / e2e_s, "unit": "slices/s", "h2d_bytes_per_step": 8 + 40 * n_chunks,
                    "d2h_bytes_per_step": (16 << k_open) + 8},
            "gpu_launches": args.steps * (n_chunks * plan.chunk_launches() + 1),   # + the XEB kernel
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
