"""Multi-process paths on the CPU (gloo, world size 2).

* bench.py's N > 1 logic: every rank contracts its own bitstring batch (distinct
  problems, weak scaling), takes a barrier and the max of the step times.
* Sharding one batch's slices across ranks (main text, section II: slices are
  independent and summed): each rank sums its own slice subset with the FP64
  oracle and one all-reduce sum gives the unsliced amplitudes.
* A lost rank is detected on the host: the survivor's collective times out with
  an error instead of hanging.
"""
import datetime
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import rqcgen


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port, timeout_s=60):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=timeout_s))


def _bench_logic(rank, world, port, q):
    import bench
    _init(rank, world, port)
    bits = bench.batch_bits_for_rank("c3", rank)
    t = bench.max_over_ranks(float(rank + 1), world, device=None)
    bench.barrier(world)
    gathered = [None] * world
    dist.all_gather_object(gathered, bits)
    if rank == 0:
        q.put((t, gathered))
    dist.destroy_process_group()


def test_bench_ranks_take_distinct_batches_and_max_time():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    mp.start_processes(_bench_logic, args=(world, port, q), nprocs=world, start_method="spawn")
    t, bits = q.get()
    assert t == 2.0
    assert len(set(bits)) == world
    _, om, cb = rqcgen.config_circuit("c3")
    assert bits[0] == cb and all(b & om == 0 for b in bits)


def _shard_slices(rank, world, port, q, first, count, log2_chunk):
    from oracle import tensornet
    from paper_2111_01066_gb300 import shard
    _init(rank, world, port)
    circ, _, _ = rqcgen.config_circuit("c1")
    open_mask, closed = 0b111100001111, 0b000010100000
    net = tensornet.CircuitNetwork(circ, closed, open_mask)
    sliced = [(0, 3), (4, 5), (7, 2), (9, 4), (11, 6)]
    a, n = shard.slice_ranges(first, count, log2_chunk, world)[rank]
    part = net.contract(sliced, range(a, a + n))          # this rank's contiguous slice range
    buf = torch.from_numpy(np.ascontiguousarray(part.view(np.float64)))
    shard.allreduce_amplitudes(buf)
    q.put((rank, buf.numpy().view(np.complex128).copy()))
    dist.destroy_process_group()


def test_slice_sharding_sum_equals_unsliced():
    """Ranks contract contiguous chunk-aligned slice ranges of one batch and
    one FP64 all-reduce gives every rank the unsliced amplitudes (all 32
    slices), or the partial sum of a ragged sub-range."""
    from oracle import tensornet
    world = 2
    circ, _, _ = rqcgen.config_circuit("c1")
    net = tensornet.CircuitNetwork(circ, 0b000010100000, 0b111100001111)
    sliced = [(0, 3), (4, 5), (7, 2), (9, 4), (11, 6)]
    for first, count, log2_chunk in ((0, 32, 2), (3, 21, 3)):
        port = _free_port()
        ctx = mp.get_context("spawn")
        q = ctx.SimpleQueue()
        mp.start_processes(_shard_slices, args=(world, port, q, first, count, log2_chunk), nprocs=world,
                           start_method="spawn")
        got = dict(q.get() for _ in range(world))
        want = net.contract(sliced, range(first, first + count))
        for r in range(world):
            assert np.linalg.norm(got[r] - want) <= 1e-12 * np.linalg.norm(want)
    want = tensornet.batch_amplitudes(circ, 0b000010100000, 0b111100001111)
    assert np.linalg.norm(net.contract(sliced) - want) <= 1e-12 * np.linalg.norm(want)


def test_slice_ranges_partition_at_chunk_boundaries():
    from paper_2111_01066_gb300 import shard
    for first, count, lc, world in ((0, 4096, 10, 4), (0, 4096, 12, 2), (100, 1000, 6, 3), (0, 0, 4, 2),
                                    (772096, 1024, 8, 8), (5, 7, 0, 16)):
        rs = shard.slice_ranges(first, count, lc, world)
        assert len(rs) == world
        pos = first
        for a, n in rs:
            if n:
                assert a == pos
                pos = a + n
                assert a == first or a % (1 << lc) == 0           # starts on a chunk boundary
        assert pos == first + count                                 # covers the range in order
        chunks = [len(range((a >> lc), ((a + n - 1) >> lc) + 1)) if n else 0 for a, n in rs]
        assert max(chunks) - min(chunks) <= 1                       # chunks dealt out evenly
    # one chunk cannot be split: the second rank idles
    assert shard.slice_ranges(0, 4096, 12, 2) == [(0, 4096), (4096, 0)]


def _lost_rank(rank, world, port, q):
    _init(rank, world, port, timeout_s=3)
    if rank == 1:
        return                      # leaves without joining the collective
    try:
        t = torch.ones(1)
        dist.all_reduce(t)
        q.put("completed")
    except Exception as e:          # the survivor learns of it on the host
        q.put("error:" + type(e).__name__)


def test_lost_rank_is_detected_without_hanging():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    mp.start_processes(_lost_rank, args=(world, port, q), nprocs=world, start_method="spawn", join=True)
    msg = q.get()
    assert msg.startswith("error:")
