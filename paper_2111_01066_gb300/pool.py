"""Plan pools: many candidate contraction orders, ranked on the host by a
roofline model, the best few measured on the GPU (SI, TN section: the paper
generates many orders and keeps the one whose measured slice time is smallest,
because the order with the fewest flops is not the fastest).

A candidate is a (seed, memory weight) pair of tn_plan_opts; the planner is
deterministic for a given candidate (its trials are seeded and the best tree
does not depend on the thread count), so a ranked pool can be stored and
rebuilt.  The ranking uses fixed reference peaks, so the same pool always
yields the same candidates to time, whatever the measured peaks of the GPU at
hand: only the ratio of the two peaks matters for the order of the ranking.

Argument marshalling and bookkeeping only; planning and timing run in the
library (tn_plan_rank, tn_plan_select_list).
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

from . import tn

# reference peaks of the ranking model (a GB300: HBM copy 6786.9 GB/s, dense
# BF16 1894.8 TFLOP/s); each precision's algorithmic complex peak follows from
# the real products it issues per complex multiply-add (TF32: 4M at half the
# BF16 rate; BF16X3 / FP16X3: three split products per real product)
REF_HBM_BYTES = 6786.9e9
REF_BF16_FLOPS = 1894.8e12
MEM_WEIGHTS = (8.0, 32.0, 128.0)


def ranking_peaks(precision: str, complex_mult: int = 4) -> Tuple[float, float]:
    """(algorithmic complex flop/s, bytes/s) the ranking model uses."""
    real_products = {("fp32", 4): None, ("tf32", 4): 4, ("tf32", 3): 3, ("bf16x3", 4): 12,
                     ("bf16x3", 3): 9, ("fp16x3", 4): 12, ("fp16x3", 3): 9}[(precision, complex_mult)]
    if real_products is None:   # CUDA-core FP32: 152 SMs x 128 lanes x 2 flops x ~1.9 GHz
        return 152 * 128 * 2 * 1.9e9, REF_HBM_BYTES
    rate = REF_BF16_FLOPS / 2 if precision == "tf32" else REF_BF16_FLOPS
    return rate * 8 / (2 * real_products), REF_HBM_BYTES


def candidate_grid(n: int) -> List[Tuple[int, float]]:
    """The first n candidates of the grid seeds 1, 2, ... x memory weights
    (8, 32, 128), seed-major."""
    return [(1 + i // len(MEM_WEIGHTS), MEM_WEIGHTS[i % len(MEM_WEIGHTS)]) for i in range(n)]


def rank_pool(network, n: int, precision: str, complex_mult: int = 4, **plan_kw) -> List[Dict]:
    """Plan the first n grid candidates (tn_plan_rank) and return them sorted by
    modeled time for all slices, fastest first; unplannable ones are dropped.
    plan_kw: the tn_plan_opts of every candidate (open_mask, bounds, trials ...)."""
    grid = candidate_grid(n)
    pf, pb = ranking_peaks(precision, complex_mult)
    secs = tn.rank_plans(network, [s for s, _ in grid], [w for _, w in grid], pf, pb, precision=precision,
                         complex_mult=complex_mult, **plan_kw)
    rows = [{"seed": s, "mem_weight": w, "model_seconds": t} for (s, w), t in zip(grid, secs) if t > 0]
    rows.sort(key=lambda r: (r["model_seconds"], r["seed"], r["mem_weight"]))
    return rows


def select_from(network, candidates: Sequence[Dict], bitstring: int, precision: str, complex_mult: int = 4,
                stream=None, **plan_kw):
    """Time the given candidates on the GPU (tn_plan_select_list) and return
    (fastest plan, its index in candidates, measured estimates for all slices)."""
    plan, est = tn.select_plan_list(network, [c["seed"] for c in candidates], [c["mem_weight"] for c in candidates],
                                    bitstring, stream=stream, precision=precision, complex_mult=complex_mult,
                                    **plan_kw)
    ok = [i for i, e in enumerate(est) if e > 0]
    chosen = min(ok, key=lambda i: est[i])
    return plan, chosen, est
