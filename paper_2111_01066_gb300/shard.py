"""Sharding one batch's slices across GPUs (main text, section II: the outer
level of the two-level scheme hands independent slices of one network to
different processors; the slices' contributions are summed into the batch's
amplitudes).

One process per GPU.  Rank r contracts a contiguous range of the batch's slice
ids with tn_contract_slices into its own FP64 amplitude buffer; one all-reduce
(sum, float64) of the 2^k complex128 amplitudes then gives every rank the
batch's amplitudes.  Ranges are cut at chunk boundaries (the plan contracts
2^b slices per chunk), so no chunk is split between ranks.  No data-path
exchange other than that sum; no peer loads.

Host logic and the collective call only; the contraction runs in the library.
"""
from __future__ import annotations

from typing import List, Tuple


def slice_ranges(first: int, count: int, log2_chunk: int, world: int) -> List[Tuple[int, int]]:
    """Per-rank (first, count) covering [first, first + count) in order, cut at
    multiples of 2^log2_chunk: the chunks the range touches are dealt out as
    evenly as possible (the first ranks take one more when they do not divide),
    and the ends of the range are clipped.  Ranks without a chunk get (x, 0)."""
    if world < 1 or count < 0 or first < 0 or log2_chunk < 0:
        raise ValueError("world >= 1, count >= 0, first >= 0, log2_chunk >= 0")
    step = 1 << log2_chunk
    lo_chunk = first >> log2_chunk
    hi_chunk = (first + count + step - 1) >> log2_chunk if count > 0 else lo_chunk
    n_chunks = hi_chunk - lo_chunk
    out = []
    c = lo_chunk
    for r in range(world):
        take = n_chunks // world + (1 if r < n_chunks % world else 0)
        a = max(first, c * step)
        b = min(first + count, (c + take) * step)
        out.append((a, max(0, b - a)) if take > 0 else (min(first + count, c * step), 0))
        c += take
    return out


def allreduce_amplitudes(out, group=None) -> None:
    """Sum the ranks' FP64 amplitude buffers in place (torch.distributed
    all-reduce, SUM, float64; NCCL on GPUs, gloo on the CPU)."""
    import torch.distributed as dist
    dist.all_reduce(out, op=dist.ReduceOp.SUM, group=group)
