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
    "c3": dict(step_slices=None, log2_batch=0, trials=128, select=8),
    # 2^20+ slices: one seeded aligned block of 1024 slices per step; every slice
    # has the same cost, so the full task's time is T_block * 2^S / 1024
    "c5": dict(step_slices=1024, log2_batch=10, trials=128, arena_gib=160, select=6),
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


def step_bits_for_rank(name: str, rank: int, count: int) -> list:
    """One seeded closed bitstring per step (stream 1000 (rank + 1) + i): every
    step is a new batch, so the steps that depend on the closed output bits
    (run once per batch) run inside every timed step."""
    circ, om, _ = rqcgen.config_circuit(name)
    seed = rqcgen.CONFIGS[name]["seed"]
    return [rqcgen.random_bits(circ.n_qubits, seed, stream=1000 * (rank + 1) + i) & ~om for i in range(count)]


def elementwise_error(got, want, n_qubits: int) -> dict:
    """The paper's Table 2 relative error per amplitude, |a - a_ref| / |a_ref|,
    as max and median over the amplitudes with 2^n |a_ref|^2 >= 0.01."""
    import numpy as np
    sel = np.ldexp(np.abs(want) ** 2, n_qubits) >= 0.01
    r = np.abs(got[sel] - want[sel]) / np.abs(want[sel])
    return {"max": float(r.max()), "median": float(np.median(r)), "count": int(sel.sum())}


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
# The oracle runs in a child process (its own BLAS threads and memory).  Its
# contraction order is data, computed beforehand by the oracle itself
# (tests/golden/make_golden.py c3order: the order its stored amplitudes were
# computed with) or built by the oracle from a candidate plan's tree shape
# (tests/golden/<name>_plans.json), so the timed samples hold
# contractions only.  A sample is a whole number of the oracle's sub-networks
# (the batch, or one slice, split by the extra wires the oracle slices itself).
ORACLE_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import rqcgen
from oracle import tensornet
circ, om, cb = rqcgen.config_circuit({name!r})
net = tensornet.CircuitNetwork(circ, cb, om)
src = json.load(open({src!r}))
if {cand!r} is None:
    merges = [tuple(m) for m in src["merges"]]
    extra = [tuple(w) for w in src["extra"]]
    sliced = []
else:
    c = [c for c in src["candidates"] if (c["seed"], c["mem_weight"]) == tuple({cand!r})][0]
    sliced = [tuple(w) for w in c["sliced_wires"]]
    merges, extra = net.plan_along_tree(sliced, c["leaf_of_gate"], [tuple(p) for p in c["step_nodes"]], max_log2=27)
budget = {budget!r}
steps = []
done = 0
for s in range({n_steps!r}):
    # one step: at least one sub-network, then more until the step's budget is spent
    cnt, t_run = 0, 0.0
    while (cnt == 0 or t_run < budget):
        sub = done % (1 << len(extra))
        values = {{leg: (sub >> j) & 1 for j, leg in enumerate(extra)}}
        values.update({{leg: 0 for leg in sliced}})
        t1 = time.time()
        net._run(merges, values)
        t_run += time.time() - t1
        done += 1
        cnt += 1
    steps.append([t_run, cnt])
print(json.dumps({{"sub_networks": 1 << len(extra), "steps": steps}}))
"""


def oracle_timing(name: str, budget_s: float, n_steps: int = 1, cand=None) -> dict:
    """Time the FP64 oracle on bounded samples.  Without `cand`: the whole batch
    of `name` along the oracle's stored order, split into 2^E sub-networks by its
    own extra sliced wires; each of n_steps samples runs at least one of them and
    more within budget_s, and the full-batch time is extrapolated from it.  With
    cand = (seed, mem_weight): one slice of that candidate plan (its stored tree
    shape and sliced wires), extrapolated the same way to a whole slice."""
    if cand is None:
        src = os.path.join(ROOT, "tests", "golden", f"{name}_oracle_order.json")
    else:
        src = os.path.join(ROOT, "tests", "golden", f"{name}_plans.json")
    if not os.path.exists(src):
        return {"error": f"no stored oracle order for {name} ({os.path.basename(src)})"}
    code = ORACLE_SNIPPET.format(root=ROOT, name=name, src=src, cand=list(cand) if cand else None,
                                 budget=budget_s, n_steps=n_steps)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=3600)
    if r.returncode != 0:
        return {"error": r.stderr.strip()[-400:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    per_step = [sec / cnt * d["sub_networks"] for sec, cnt in d["steps"]]
    return {"unit_seconds": per_step[-1], "step_unit_seconds": per_step,
            "step_seconds": [sec for sec, _ in d["steps"]], "step_sub_networks": [cnt for _, cnt in d["steps"]],
            "timed_sub_networks": sum(cnt for _, cnt in d["steps"]), "sub_networks": d["sub_networks"],
            "seconds": sum(sec for sec, _ in d["steps"])}


def cores_used() -> int:
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(var, "").isdigit():
            return int(os.environ[var])
    return os.cpu_count() or 1


# ------------------------------------------------------------------ rooflines
FP32_SIMT_TFLOPS = 152 * 128 * 2 * 1.92 / 1e3   # SMs x FP32 lanes x 2 flops x GHz under load

# DRAM bytes (read + write) per launch of the tensor-core GEMM at full size,
# keyed by (kernel, log2 m,k,n,batch): one ncu launch list (time and DRAM bytes,
# a single pass per launch) of one timed step of each benchmark plan with the
# kernels an unprofiled run's autotuner chose (one SM or SM pairs; replayed in
# the profiled run), matched to the steps in launch order (profiles/c3_bf16x3_launch_list.md,
# profiles/c5_bf16x3_launch_list.md)
MEASURED_TRAFFIC = {
    ("tc_bf16x3", (21, 8, 8, 0)): 8.7789e+09,   # c3
    ("tc_bf16x3", (21, 7, 8, 0)): 6.4022e+09,   # c3
    ("tc_bf16x3", (12, 10, 7, 7)): 5.1233e+09,   # c3
    ("tc_bf16x3", (11, 10, 9, 5)): 1.1190e+09,   # c3
    ("tc_bf16x3", (22, 4, 6, 0)): 2.6199e+09,   # c3
    ("tc_bf16x3", (15, 7, 12, 0)): 1.0543e+09,   # c3
    ("tc_bf16x3", (19, 8, 5, 0)): 1.1935e+09,   # c3
    ("tc_bf16x3", (16, 6, 10, 0)): 5.0618e+08,   # c3
    ("tc_bf16x3", (13, 9, 11, 0)): 1.3029e+08,   # c3
    ("tc_bf16x3", (20, 5, 4, 0)): 3.6322e+08,   # c3
    ("tc_bf16x3", (13, 8, 11, 0)): 9.5713e+07,   # c3
    ("tc_bf16x3", (18, 6, 4, 0)): 1.4450e+08,   # c3
    ("tc_bf16x3", (20, 8, 8, 0)): 4.3654e+09,   # c5
    ("tc_bf16x3", (18, 8, 9, 1)): 3.3820e+09,   # c5
    ("tc_bf16x3", (14, 9, 8, 5)): 3.8655e+09,   # c5
    ("tc_bf16x3", (21, 7, 7, 0)): 4.2418e+09,   # c5
    ("tc_bf16x3", (19, 8, 8, 0)): 2.1476e+09,   # c5
    ("tc_bf16x3", (13, 10, 11, 0)): 2.3925e+08,   # c5
    ("tc_bf16x3", (18, 6, 9, 0)): 1.1464e+09,   # c5
    ("tc_bf16x3", (13, 14, 3, 0)): 1.0961e+09,   # c5
    ("tc_bf16x3", (12, 9, 9, 3)): 2.6187e+08,   # c5
    ("tc_bf16x3", (12, 11, 9, 1)): 2.0207e+08,   # c5
    ("tc_bf16x3", (18, 6, 8, 0)): 6.0673e+08,   # c5
    ("tc_bf16x3", (19, 7, 5, 0)): 6.4703e+08,   # c5
    ("tc_bf16x3", (11, 11, 8, 0)): 5.2409e+07,   # c5
    ("tc_bf16x3", (12, 5, 12, 0)): 7.2190e+07,   # c5
    ("tc_bf16x3", (13, 3, 10, 0)): 4.4308e+06,   # c5
    ("tc_bf16x3", (11, 8, 10, 0)): 8.4800e+06,   # c5
    ("tc_bf16x3", (16, 6, 6, 0)): 3.3713e+07,   # c5
}


_PEAKS = None


def measure_matmul_peaks() -> dict:
    """Dense matmul rates of the other precisions, measured like the BF16 one of
    MEASURED_PEAKS.json (torch.matmul, 8192^3, 2 N^3 flops, best of 10, CUDA
    events): FP16, TF32 (FP32 inputs with TF32 tensor cores allowed) and plain
    FP32 on the CUDA cores (TF32 disallowed: cuBLAS SGEMM, the roof of an FP32
    SIMT GEMM)."""
    import torch
    n = 8192
    out = {}
    old = torch.backends.cuda.matmul.allow_tf32
    try:
        for key, dtype, tf32 in (("fp16_tflops", torch.float16, False), ("tf32_tflops", torch.float32, True),
                                 ("fp32_simt_tflops", torch.float32, False)):
            torch.backends.cuda.matmul.allow_tf32 = tf32
            a = torch.randn(n, n, device="cuda", dtype=dtype)
            b = torch.randn(n, n, device="cuda", dtype=dtype)
            c = torch.empty(n, n, device="cuda", dtype=dtype)
            torch.matmul(a, b, out=c)
            torch.cuda.synchronize()
            best = None
            for _ in range(10 if key != "fp32_simt_tflops" else 4):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b, out=c)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
            out[key] = 2.0 * n ** 3 / (best / 1e3) / 1e12
            del a, b, c
    finally:
        torch.backends.cuda.matmul.allow_tf32 = old
    torch.cuda.empty_cache()
    return out


def load_peaks() -> dict:
    """MEASURED_PEAKS.json (HBM copy, BF16 matmul), plus the other precisions'
    matmul rates measured in this process when a GPU is present (once)."""
    global _PEAKS
    if _PEAKS is not None:
        return _PEAKS
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        d["source"] = "measured"
    else:
        d = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}
    try:
        import torch
        if torch.cuda.is_available():
            d.update(measure_matmul_peaks())
            d["other_precisions"] = "measured here: torch.matmul 8192^3, best of 10 (FP32 SIMT: of 4)"
    except Exception as e:  # pragma: no cover - reported, the nominal ratios are used instead
        d["other_precisions"] = f"not measured ({e}); nominal ratios to BF16"
    _PEAKS = d
    return d


def complex_peak_tflops(kernel: str, peaks: dict) -> float:
    """Peak in algorithmic complex flops (8 per complex multiply-add) of a kernel:
    a real tensor peak P runs a complex MAC as R real MACs, so P_eff = P * 8 / (2 R).
    Each precision takes its own measured matmul rate when present, else the
    nominal ratio to BF16 (TF32 half, FP16 equal)."""
    bf16 = peaks["bf16_tflops"]
    tf32 = peaks.get("tf32_tflops", bf16 / 2)
    fp16 = peaks.get("fp16_tflops", bf16)
    real = {"tc_tf32": (tf32, 4),              # 4M: four real products per complex one
            "tc_tf32_3m": (tf32, 3),
            "tc_bf16x3": (bf16, 12),           # 3 bf16 products per real product, 4M
            "tc_bf16x3_3m": (bf16, 9),
            "tc_fp16x3": (fp16, 12),
            "tc_fp16x3_3m": (fp16, 9)}
    if kernel in real:
        p, r = real[kernel]
        return p * 8 / (2 * r)
    # CUDA-core complex GEMM: 4 real FMAs (8 flops) per complex multiply-add
    return peaks.get("fp32_simt_tflops", FP32_SIMT_TFLOPS)


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


# ------------------------------------------------------------------ one workload
def golden_amplitudes(name: str):
    """The oracle's stored amplitudes and XEB of the whole batch of `name` (text
    files written by tests/golden/make_golden.py), or (None, None)."""
    import numpy as np
    gold_path = os.path.join(ROOT, "tests", "golden", f"{name}_amplitudes.txt")
    gold_xeb_path = os.path.join(ROOT, "tests", "golden", f"{name}_xeb.txt")
    if not (os.path.exists(gold_path) and os.path.exists(gold_xeb_path)):
        return None, None
    g = np.loadtxt(gold_path, comments="#")
    return g[:, 0] + 1j * g[:, 1], float(np.loadtxt(gold_xeb_path, comments="#"))


def golden_block(name: str, cand):
    """The oracle's stored partial sums for candidate cand = (seed, mem_weight)
    (tests/golden/<name>_block_amplitudes.txt): {"block": the first slices of
    its timed block, "sample": a seeded slice sample}, each {"slices", "wires",
    "amps"}; None if absent."""
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", f"{name}_block_amplitudes.txt")
    if not os.path.exists(path):
        return None
    found, cur = {}, None
    with open(path) as f:   # sections: "# candidate seed=.. mem_weight=.. kind=.. slices=a,b,..", "# wires", values
        for line in f:
            if line.startswith("# candidate"):
                kv = dict(tok.split("=", 1) for tok in line.split() if "=" in tok)
                cur = {"slices": [int(x) for x in kv["slices"].split(",")], "amps": [], "wires": []}
                found.setdefault((int(kv["seed"]), float(kv["mem_weight"])), {})[kv["kind"]] = cur
            elif line.startswith("# wires") and cur is not None:
                cur["wires"] = [tuple(int(x) for x in w.split(",")) for w in line.split()[2:]]
            elif line.strip() and not line.startswith("#") and cur is not None:
                re_, im_ = line.split()
                cur["amps"].append(complex(float(re_), float(im_)))
    got = found.get((int(cand[0]), float(cand[1])))
    if got is not None:
        for sec in got.values():
            sec["amps"] = np.array(sec["amps"])
    return got


def run_workload(name: str, args, ctx: dict, prec: str, cm: int, pool_n: int, n_select: int, compare: bool,
                 cpu_budget: float, steps: int, warmup: int) -> dict:
    """Plan (pool ranked by model, best few timed), autotune, then time `steps`
    steps of the workload (one step = every slice of the batch, or the timed
    block of slices, + the XEB); error against the oracle's stored values; e2e;
    rooflines; sampling; CPU baseline."""
    import numpy as np
    import torch
    from paper_2111_01066_gb300 import pool
    tn, rank, world, dev, stream, flush = (ctx[k] for k in ("tn", "rank", "world", "dev", "stream", "flush"))
    from paper_2111_01066_gb300 import shard
    sharded = ctx.get("shard") == "slices" and world > 1
    cfg = rqcgen.CONFIGS[name]
    circ, om, cb = rqcgen.config_circuit(name)
    # weak scaling: every rank its own batch; sharded: one batch, its slices split across ranks
    bits = batch_bits_for_rank(name, 0 if sharded else rank)
    net = tn.Network(circ)
    run = WORKLOAD_RUN[name]
    log2_batch = run["log2_batch"]
    if sharded:
        # chunks small enough that every rank gets whole chunks of the step's slices
        step_log2 = cfg["log2_slices"] if run["step_slices"] is None else int(math.log2(run["step_slices"]))
        log2_batch = max(0, step_log2 - max(0, (world - 1).bit_length()))
    plan_kw = dict(open_mask=om, max_log2_intermediate=cfg["log2_bound"], min_log2_slices=cfg["log2_slices"],
                   log2_batch_slices=log2_batch, trials=run.get("trials", 64),
                   max_arena_bytes=int(run.get("arena_gib", 96)) << 30)
    t_plan = time.time()
    selection = None
    cand = (1, 32.0)
    plan = None
    if ctx.get("plan_choice"):   # a given candidate (seed, memory weight): no pool
        cand = ctx["plan_choice"]
    elif pool_n > 1 and n_select >= 1:
        if rank == 0:
            # host: rank the pool by modeled time; GPU: time the best few, keep the fastest
            t0 = time.time()
            ranked = pool.rank_pool(net, pool_n, prec, cm, **plan_kw)
            t_rank = time.time() - t0
            cands = ranked[:n_select]
            t0 = time.time()
            plan, ch, est = pool.select_from(net, cands, bits, prec, cm, stream=stream, **plan_kw)
            cand = (cands[ch]["seed"], cands[ch]["mem_weight"])
            selection = {"pool": pool_n, "planned": len(ranked), "ranked_by": "modeled time for all slices "
                         "(tn_plan_rank: per-step roofline max(flops / peak, bytes / bandwidth))",
                         "rank_seconds": t_rank, "select_seconds": time.time() - t0,
                         "model_best_seconds": ranked[0]["model_seconds"],
                         "model_median_seconds": statistics.median(r["model_seconds"] for r in ranked),
                         "timed": [dict(c, measured_seconds=e) for c, e in zip(cands, est)],
                         "chosen": ch, "chosen_seed": cand[0], "chosen_mem_weight": cand[1]}
        if world > 1:   # every rank runs rank 0's choice
            import torch.distributed as dist
            t = torch.tensor([float(cand[0]), cand[1]], dtype=torch.float64, device=dev)
            dist.broadcast(t, 0)
            cand = (int(t[0].item()), float(t[1].item()))
    plan_kw = dict(plan_kw, seed=cand[0], mem_weight=cand[1])
    if plan is None:
        plan = tn.Plan(net, precision=prec, complex_mult=cm, **plan_kw)
    t_plan = time.time() - t_plan
    info = plan.info()
    all_slices = 1 << info["log2_slices"]
    n_slices = all_slices if run["step_slices"] is None else min(all_slices, run["step_slices"])
    first = rqcgen.timed_block_first(info["log2_slices"], n_slices, cfg["seed"]) if n_slices < all_slices else 0
    k_open = info["n_open"]
    # this rank's slices of the step: all of them, or its chunk-aligned share of one batch
    my_first, my_count = (shard.slice_ranges(first, n_slices, info["log2_batch_slices"], world)[rank] if sharded
                          else (first, n_slices))
    n_chunks = max(1, -(-my_count >> info["log2_batch_slices"])) if my_count else 0
    out = torch.zeros(2 << k_open, dtype=torch.float64, device=dev)
    # a new batch (closed bitstring) every step: the per-batch prologue is part of each step
    sbits = step_bits_for_rank(name, 0 if sharded else rank, warmup + steps)

    def step(p, o, b=bits):
        o.zero_()
        if my_count:
            p.contract_slices(my_first, my_count, [b], o, stream)
        if sharded:   # the batch's amplitudes: one FP64 sum over the ranks' slice ranges
            shard.allreduce_amplitudes(o)
        return tn.xeb(o.view(torch.complex128), circ.n_qubits, stream)

    def timed(p, o, k, w, mark=False):
        for i in range(w):
            step(p, o, sbits[i % len(sbits)])
        torch.cuda.synchronize()
        times = []
        for i in range(k):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            if mark:   # NVTX range of the timed steps (a profiler can capture just these)
                torch.cuda.nvtx.range_push("timed_step")
            e0.record(stream)
            step(p, o, sbits[(w + i) % len(sbits)])
            e1.record(stream)
            if mark:
                torch.cuda.nvtx.range_pop()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        return times

    gold, gold_xeb = golden_amplitudes(name) if rank == 0 else (None, None)
    gblock = golden_block(name, cand) if rank == 0 and n_slices < all_slices else None

    def amp_error(p, o):
        """Error of plan p against the oracle: the whole batch (workload
        bitstring) when every slice is contracted, else the oracle's partial sum
        over the first slices of this candidate's timed block."""
        if n_slices == all_slices:
            step(p, o)   # every rank runs it: with sharded slices the step holds the all-reduce
            torch.cuda.synchronize()
            if gold is None or gold.size != (o.numel() // 2):
                return None
            got = o.cpu().numpy().view(np.complex128)
            f = tn.xeb(o.view(torch.complex128), circ.n_qubits)
            return {"rel_amp_err": float(np.linalg.norm(got - gold) / np.linalg.norm(gold)),
                    "elementwise_rel_err": elementwise_error(got, gold, circ.n_qubits),
                    "xeb_err": abs(f - gold_xeb), "against": "oracle amplitudes of the whole batch"}
        if gblock is not None and gblock["block"]["slices"][0] == first and \
                [tuple(w) for w in p.sliced_wires()] == gblock["block"]["wires"]:
            def slice_sum(ids):
                o.zero_()
                ids = sorted(ids)
                i = 0
                while i < len(ids):
                    j = i + 1
                    while j < len(ids) and ids[j] == ids[j - 1] + 1:
                        j += 1
                    p.contract_slices(ids[i], j - i, [cb], o, stream)
                    i = j
                p.sync(stream)
                return o.cpu().numpy().view(np.complex128).copy()

            def rel(got, want, scale):
                pw = np.abs(want) ** 2
                sel = pw >= 0.01 * np.mean(pw)
                r = np.abs(got[sel] - want[sel]) / np.abs(want[sel])
                return {"rel_amp_err": float(np.linalg.norm(got - want) / scale),
                        "elementwise_rel_err": {"max": float(r.max()), "median": float(np.median(r)),
                                                "count": int(sel.sum()), "cut": "|a|^2 >= 0.01 mean |a|^2"}}
            smp, blk = gblock["sample"], gblock["block"]
            res = {"sample": dict(rel(slice_sum(smp["slices"]), smp["amps"], np.linalg.norm(smp["amps"])),
                                  against=f"oracle partial sum over a seeded sample of {len(smp['slices'])} "
                                          f"slice ids")}
            scale = max(np.linalg.norm(blk["amps"]), np.linalg.norm(smp["amps"]))
            b = rel(slice_sum(blk["slices"]), blk["amps"], scale)
            b["near_zero_block"] = bool(np.linalg.norm(blk["amps"]) < 1e-6 * np.linalg.norm(smp["amps"]))
            b["against"] = (f"oracle partial sum over slices {blk['slices'][0]}..{blk['slices'][-1]} of the timed "
                            f"block; norm-wise error on the scale of a 16-slice sum")
            res["timed_block"] = b
            res["rel_amp_err"] = max(res["sample"]["rel_amp_err"], b["rel_amp_err"])
            return res
        return None

    # untimed first call: device state + warm-up; then the per-step autotuner,
    # or the per-step kernel choices of an earlier run (a profiled run replays
    # those of its unprofiled twin: under a profiler the autotuner's own timing
    # is distorted and would pick other kernels)
    step(plan, out)
    torch.cuda.synchronize()
    t_tune = time.time()
    if ctx.get("tuning_in"):
        with open(ctx["tuning_in"]) as f:
            plan.set_tuning(json.load(f))
        step(plan, out)
        torch.cuda.synchronize()
    elif args.autotune:
        plan.autotune(reps=2, stream=stream)
        step(plan, out)
        torch.cuda.synchronize()
    if ctx.get("tuning_out") and rank == 0:
        with open(ctx["tuning_out"], "w") as f:
            json.dump(plan.get_tuning(), f)
    t_tune = time.time() - t_tune
    barrier(world)
    clocks = ClockSampler(ctx["local"])
    clocks.start()
    times = timed(plan, out, steps, warmup, mark=True)
    clk = clocks.stop()
    barrier(world)
    ms = statistics.mean(times)
    ms_max = max_over_ranks(ms, world, dev)
    total_units = n_slices if sharded else n_slices * world
    value = total_units / (ms_max / 1e3)
    err = amp_error(plan, out)
    step(plan, out)   # the rank's own batch
    torch.cuda.synchronize()
    amps = out.cpu().numpy().view(np.complex128).copy()
    f_xeb = tn.xeb(out.view(torch.complex128), circ.n_qubits)

    # e2e: host bitstrings in, host amplitudes + XEB out, wall clock
    host_amps = torch.empty(2 << k_open, dtype=torch.float64, pin_memory=True)
    e2e_times = []
    for i in range(warmup + steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out.zero_()
        if my_count:
            plan.contract_slices(my_first, my_count, [sbits[i]], out, stream)
        if sharded:
            shard.allreduce_amplitudes(out)
        host_amps.copy_(out, non_blocking=True)
        tn.xeb(out.view(torch.complex128), circ.n_qubits, stream)
        torch.cuda.synchronize()
        if i >= warmup:
            e2e_times.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(statistics.mean(e2e_times), world, dev)

    # the other paths on the same plan and slices: FP32 SIMT (the plain path),
    # TF32, and the other complex product (4M / 3M) of this precision
    others = {}
    if compare:
        alts = [("fp32", 4), ("tf32", 4)]
        if prec in ("tf32", "bf16x3", "fp16x3"):
            alts.append((prec, 7 - cm))
        for other, ocm in alts:
            if (other, ocm) == (prec, cm):
                continue
            p2 = tn.Plan(net, precision=other, complex_mult=ocm, **plan_kw)
            o2 = torch.zeros_like(out)
            step(p2, o2)
            if args.autotune:
                p2.autotune(reps=1, stream=stream)
                o2.zero_()
                step(p2, o2)
            t2 = timed(p2, o2, min(3, steps), 1)
            ms2 = max_over_ranks(statistics.mean(t2), world, dev)
            others[other if ocm == 4 else other + "_3m"] = {
                "precision": other, "complex_mult": ocm, "value": total_units / (ms2 / 1e3), "ms_per_step": ms2,
                "error_vs_oracle": amp_error(p2, o2)}
            del p2, o2

    # roofline of every step: per-step device times on the same stream
    st = plan.step_times(reps=3, stream=stream)
    shapes = plan.step_shapes()
    peaks = load_peaks()
    rows = [step_roofline(shapes[i], st[i][0], st[i][1], peaks) for i in range(len(st))]
    i_dom = max(range(len(rows)), key=lambda i: rows[i]["ms"])
    roof = dict(rows[i_dom])
    roof["share_of_step_time"] = rows[i_dom]["ms"] / sum(r["ms"] for r in rows)
    roof["step"] = i_dom
    t_roof = sum(r["t_roof_ms"] for r in rows)
    path_roof = {"t_roof_ms": t_roof, "t_steps_ms": sum(r["ms"] for r in rows),
                 "frac": t_roof / sum(r["ms"] for r in rows)}
    top = sorted(rows, key=lambda r: -r["ms"])[:8]
    if ctx.get("step_report") and rank == 0:
        with open(ctx["step_report"], "w") as f:
            for i, row in enumerate(rows):
                f.write(json.dumps(dict(row, step=i, dep_flags=plan.step_layout(i)["dep_flags"])) + "\n")

    # frugal sampling within the batch (main text, section III): with the whole
    # slice sum in hand, draw 2^k samples (128 uniform proposals each, M = 10)
    # and take the linear XEB of the samples (1 for an ideal sampler)
    frugal = None
    if n_slices == all_slices:
        step(plan, out)   # the workload's own batch again (every rank: the step may hold the all-reduce)
        torch.cuda.synchronize()
    if rank == 0 and n_slices == all_slices:
        m_bound, draws, n_samp = 10.0, 128, 1 << k_open
        rs = np.random.default_rng([cfg["seed"], 17])
        cand_t = torch.from_numpy(rs.integers(0, 1 << k_open, size=(n_samp, draws))).to(dev)
        unif = torch.from_numpy(rs.random((n_samp, draws))).to(dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        first_draw = tn.frugal_sample(out.view(torch.complex128), circ.n_qubits, m_bound, cand_t, unif, stream)
        t_samp = time.perf_counter() - t0
        idx = [int(cand_t[s_, t_]) for s_, t_ in enumerate(first_draw) if t_ >= 0]
        picked = out.view(torch.complex128)[torch.tensor(idx, device=dev)]
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
        t_batch = all_slices / value * (1 if sharded else world)
        per_sample = {"batch_seconds": t_batch, "p_sample_per_batch": p_batch,
                      "seconds_per_perfect_sample": t_batch / p_batch,
                      "days_for_1M_samples_at_xeb_0.002": 2000 * t_batch / p_batch / 86400,
                      "note": "extrapolated from the timed slice block; 1M samples at fidelity 0.002 "
                              "cost as much as 2000 perfect samples (main text, section III)"}

    cpu = None
    if rank == 0 and world == 1 and cpu_budget > 0:
        if n_slices == all_slices:
            t = oracle_timing(name, cpu_budget)
            unit = n_slices
            what = f"oracle sub-networks of the full {n_slices}-slice batch along its stored order"
        else:
            t = oracle_timing(name, cpu_budget, cand=cand)
            unit = 1
            what = (f"oracle sub-networks of one slice of the chosen plan (seed {cand[0]}, weight {cand[1]}), "
                    f"along an order the oracle builds from the plan's tree shape")
        if "error" not in t:
            cpu = {"value": unit / t["unit_seconds"], "unit": "slices/s", "cores": cores_used(), "kind": "oracle",
                   "sample": f"{t['timed_sub_networks']} of {t['sub_networks']} {what} ({t['seconds']:.1f} s), "
                             f"extrapolated"}
        else:
            cpu = {"value": None, "unit": "slices/s", "cores": cores_used(), "kind": "oracle",
                   "sample": "oracle unavailable: " + t["error"][-200:]}

    launches = n_chunks * plan.chunk_launches() + (plan.batch_launches() if my_count else 0) + 1   # + XEB
    return {"sharded": sharded, "my_range": [my_first, my_count],"name": name, "circ": circ, "cfg": cfg, "info": info, "value": value, "ms": ms_max, "times": times,
            "e2e_s": e2e_s, "n_slices": n_slices, "all_slices": all_slices, "first": first, "n_chunks": n_chunks,
            "k_open": k_open, "total_units": total_units, "err": err, "xeb": f_xeb, "others": others,
            "roof": roof, "path_roof": path_roof, "top": top, "frugal": frugal, "per_sample": per_sample,
            "cpu": cpu, "clocks": clk, "selection": selection, "cand": cand, "t_plan": t_plan, "t_tune": t_tune,
            "launches_per_step": launches, "plan": plan}


def workload_string(name: str, circ, cfg, log2_slices: int, k_open: int) -> str:
    return (f"{name}: {circ.n_qubits}-qubit {cfg['rows']}x{cfg['cols']} grid, {cfg['cycles']} cycles, "
            f"2^{log2_slices} slices (<=2^{cfg['log2_bound']} per slice), {k_open} open qubits")


# ------------------------------------------------------------------ reference arm
def reference_arm(args, name: str, rank: int) -> int:
    """The oracle as it stands, on the host cores of rank 0: one step = one of
    the oracle's own sub-networks of the batch (the batch is the sum of
    2^E of them along its stored order), so the step time is measured, not
    extrapolated; value = the batch's slices / 2^E per step time."""
    if rank != 0:
        return 0
    cfg = rqcgen.CONFIGS[name]
    circ, _, _ = rqcgen.config_circuit(name)
    total_slices = 1 << cfg["log2_slices"]
    n_all = args.warmup + args.steps
    t = oracle_timing(name, 0.0, n_all)          # budget 0: exactly one sub-network per step
    line = {"impl": "reference", "metric": "slices/s", "unit": "slices/s", "n_gpus": args.gpus,
            "device": "host cores (FP64 oracle)", "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_string(name, circ, cfg, cfg["log2_slices"], cfg["k_open"])}}
    if "error" in t:
        line.update({"value": None, "ms_per_step": None, "unavailable": "oracle failed: " + t["error"]})
        print(json.dumps(line))
        return 0
    secs = t["step_seconds"][args.warmup:]
    per_step_slices = total_slices / t["sub_networks"]
    mean_s = statistics.mean(secs)
    value = per_step_slices / mean_s
    line.update({"value": value, "ms_per_step": mean_s * 1e3,
                 "cpu_baseline": {"value": value, "unit": "slices/s", "cores": cores_used(), "kind": "oracle",
                                  "sample": f"{args.warmup} + {args.steps} steps, each one of the oracle's "
                                            f"{t['sub_networks']} sub-networks of the full {total_slices}-slice "
                                            f"batch (= {per_step_slices:g} slices of work), along its stored order"},
                 "e2e": {"value": value, "unit": "slices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})
    print(json.dumps(line))
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
    ap.add_argument("--pool", type=int, default=102,
                    help="candidate plans (seeds x memory weights 8, 32, 128) ranked by modeled time on the host "
                         "(<= 1: one plan, seed 1, weight 32)")
    ap.add_argument("--plan", default=None,
                    help="seed,mem_weight: use this candidate plan (no pool ranking or selection)")
    ap.add_argument("--step-report", default=None, help="file for every step's timing and roofline (JSON lines)")
    ap.add_argument("--select", type=int, default=None,
                    help="best-modeled candidates timed on the GPU (default: per workload)")
    ap.add_argument("--complex-mult", type=int, default=4, choices=[3, 4],
                    help="4M or 3M complex products on the tensor cores")
    ap.add_argument("--compare-fp32", type=int, default=1)
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--c5", type=int, default=1,
                    help="with the default workload on one GPU, also time the 53-qubit block (c5 sub-object)")
    ap.add_argument("--c5-steps", type=int, default=5)
    ap.add_argument("--autotune", type=int, default=1, help="tune kernels per step before timing")
    ap.add_argument("--tuning-out", default=None, help="write the per-step kernel choices (JSON) after tuning")
    ap.add_argument("--tuning-in", default=None,
                    help="use the per-step kernel choices of an earlier run (JSON from --tuning-out) instead of "
                         "tuning: the same plan then runs the same kernels, e.g. under a profiler")
    ap.add_argument("--shard", default="batches", choices=["batches", "slices"],
                    help="N > 1: every rank its own batch (weak scaling), or one batch whose slices are split "
                         "across the ranks and summed by one FP64 all-reduce (strong scaling)")
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
    if args.impl == "reference":
        return reference_arm(args, name, rank)

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
    plan_choice = None
    if args.plan:
        sd, wt = args.plan.split(",")
        plan_choice = (int(sd), float(wt))
    ctx = {"tn": tn, "rank": rank, "world": world, "local": local, "dev": dev, "shard": args.shard,
           "plan_choice": plan_choice, "step_report": args.step_report,
           "tuning_in": args.tuning_in, "tuning_out": args.tuning_out,
           "stream": torch.cuda.current_stream(),
           "flush": torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)}
    n_select = args.select if args.select is not None else WORKLOAD_RUN[name].get("select", 6)
    r = run_workload(name, args, ctx, prec, args.complex_mult, args.pool, n_select, bool(args.compare_fp32),
                     args.cpu_budget, args.steps, args.warmup)
    info, circ, cfg = r["info"], r["circ"], r["cfg"]

    # the 53-qubit workload beside the default one: its timed block, plan
    # selection and time per perfect sample (one GPU only)
    c5 = None
    if args.c5 and name == "c3" and world == 1:
        del r["plan"]
        torch.cuda.empty_cache()
        r5 = run_workload("c5", args, dict(ctx, plan_choice=None, step_report=None, tuning_in=None, tuning_out=None), prec, args.complex_mult, args.pool, WORKLOAD_RUN["c5"]["select"], False,
                          min(args.cpu_budget, 10.0), args.c5_steps, args.warmup)
        c5 = {"workload": workload_string("c5", r5["circ"], r5["cfg"], r5["info"]["log2_slices"], r5["k_open"]),
              "metric": "slices/s", "value": r5["value"], "ms_per_block": r5["ms"], "steps": args.c5_steps,
              "slices_per_step": r5["n_slices"], "slice_first": r5["first"], "slices_total": r5["all_slices"],
              "extrapolated_full_task_s": r5["all_slices"] / r5["value"],
              "complex_tflops": r5["info"]["flops_per_chunk"] * r5["n_chunks"] / (r5["ms"] / 1e3) / 1e12,
              "perfect_sample": r5["per_sample"], "error_vs_oracle": r5["err"], "plan_selection": r5["selection"],
              "roofline": r5["roof"], "path_roofline": r5["path_roof"], "top_steps": r5["top"][:4],
              "clocks": r5["clocks"], "cpu_baseline": r5["cpu"],
              "plan": {"seed": r5["cand"][0], "mem_weight": r5["cand"][1], "n_steps": r5["info"]["n_steps"],
                       "flops_per_chunk": r5["info"]["flops_per_chunk"],
                       "arena_gib": r5["info"]["arena_bytes"] / 2 ** 30, "plan_seconds": r5["t_plan"]},
              "e2e": {"value": r5["n_slices"] / r5["e2e_s"], "unit": "slices/s"},
              "gpu_launches": args.c5_steps * r5["launches_per_step"]}

    if rank == 0:
        fp32 = r["others"].get("fp32")
        value, ms_max, n_chunks, k_open = r["value"], r["ms"], r["n_chunks"], r["k_open"]
        line = {
            "metric": "slices/s", "value": value, "unit": "slices/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
            "scaling": "strong" if r["sharded"] else "weak",
            "vs_baseline": None, "dtype": {"fp32": "f32", "tf32": "tf32", "bf16x3": "bf16x3",
                                           "fp16x3": "fp16x3"}[prec],
            "data": "synthetic",
            "config": {"workload": workload_string(name, circ, cfg, info["log2_slices"], k_open),
                       "precision": prec, "complex_mult": info["complex_mult"],
                       "parallelism": (f"slices of one batch split over {world} GPUs + FP64 all-reduce"
                                       if r["sharded"] else f"{world} GPU(s), one batch each"),
                       "slices_per_step": r["n_slices"], "chunks_per_step": n_chunks, "slice_first": r["first"],
                       "slices_total": r["all_slices"],
                       "log2_batch_slices": info["log2_batch_slices"], "l2": "flushed between steps "
                       "(512 MiB write); intermediates also exceed L2",
                       "batches": "a new seeded closed bitstring every step: the per-batch prologue (steps "
                                  "that depend on the closed output bits) runs inside every timed step"},
            "complex_tflops": info["flops_per_chunk"] * n_chunks * world / (ms_max / 1e3) / 1e12,   # whole job
            "complex_tflops_per_slice_basis": info["flops_per_slice"] * r["total_units"] / (ms_max / 1e3) / 1e12,
            "plan": {"seed": r["cand"][0], "mem_weight": r["cand"][1], "flops_per_slice": info["flops_per_slice"],
                     "flops_per_chunk": info["flops_per_chunk"], "bytes_per_chunk": info["bytes_per_chunk"],
                     "n_steps": info["n_steps"], "log2_max_intermediate": info["log2_max_intermediate"],
                     "arena_gib": info["arena_bytes"] / 2**30, "plan_seconds": r["t_plan"],
                     "autotune_seconds": r["t_tune"] if args.autotune else None},
            "extrapolated_full_task_s": r["all_slices"] / value * world if r["n_slices"] < r["all_slices"] else None,
            "fp32_path": fp32,
            "tf32_path": r["others"].get("tf32"),
            "other_complex_mult_path": r["others"].get(prec + "_3m") if args.complex_mult == 4
            else r["others"].get(prec),
            "speedup_vs_fp32_path": (value / fp32["value"]) if fp32 else None,
            "error_vs_oracle": r["err"],
            "xeb": r["xeb"],
            "plan_selection": r["selection"],
            "frugal_sampling": r["frugal"],
            "perfect_sample": r["per_sample"],
            "roofline": r["roof"],
            "path_roofline": r["path_roof"],
            "top_steps": r["top"],
            "clocks": r["clocks"],
            "peaks": {k: v for k, v in load_peaks().items() if k in ("hbm_gbs", "bf16_tflops", "fp16_tflops",
                                                                     "tf32_tflops", "fp32_simt_tflops",
                                                                     "other_precisions", "source")},
            "e2e": {"value": r["total_units"] / r["e2e_s"], "unit": "slices/s", "h2d_bytes_per_step": 8 + 40 * n_chunks,
                    "d2h_bytes_per_step": (16 << k_open) + 8},
            "gpu_launches": args.steps * r["launches_per_step"],
            "cpu_baseline": r["cpu"],
            "c5": c5,
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
