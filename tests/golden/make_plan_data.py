"""Write the parameters of the candidate plans the benchmark may time.

The benchmark's workloads use a plan chosen from a ranked pool
(paper_2111_01066_gb300.pool): the library's host planner ranks the candidates
by modeled time and the GPU times the best few.  Which candidate wins depends
on the GPU's timing, so the parity tests cover every candidate the benchmark
may time.  For each, this script records the candidate (seed, memory weight),
what defines its partial sums -- the sliced wires (slice id s sets wire j to
bit j of s) and the first slice id of its timed block (53 qubits: one seeded
block of 1024 slices) -- and the shape of its contraction tree (which circuit
gates each leaf holds and the pairwise merges), which the oracle uses only to
choose its own contraction order (any complete tree gives the same sum; the
oracle checks completeness).

This script calls the library's host planner only (no GPU, no kernel) and no
oracle code; tests/golden/make_golden.py then computes the expected partial
sums with the oracle alone.

    python tests/golden/make_plan_data.py c3 c5
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import rqcgen  # noqa: E402

# the benchmark's pools: pool size, candidates timed, plan options (bench.py
# WORKLOAD_RUN), timed block (None: every slice) and slices the oracle checks
RUNS = {"c3": dict(pool=102, timed=8, trials=128, log2_batch=0, arena_gib=96, precision="bf16x3", complex_mult=4,
                   block=None, check_slices=0),
        "c5": dict(pool=102, timed=6, trials=128, log2_batch=10, arena_gib=160, precision="bf16x3", complex_mult=4,
                   block=1024, check_slices=16)}


def plan_kw(name: str, run: dict) -> dict:
    cfg = rqcgen.CONFIGS[name]
    _, om, _ = rqcgen.config_circuit(name)
    return dict(open_mask=om, max_log2_intermediate=cfg["log2_bound"], min_log2_slices=cfg["log2_slices"],
                log2_batch_slices=run["log2_batch"], trials=run["trials"], max_arena_bytes=run["arena_gib"] << 30)


def write(name: str) -> None:
    import __graft_entry__
    __graft_entry__.build()
    from paper_2111_01066_gb300 import pool, tn
    run = RUNS[name]
    circ, om, cb = rqcgen.config_circuit(name)
    net = tn.Network(circ)
    kw = plan_kw(name, run)
    ranked = pool.rank_pool(net, run["pool"], run["precision"], run["complex_mult"], **kw)
    out = {"workload": name, "pool": run["pool"], "timed": run["timed"], "options": {k: v for k, v in run.items()},
           "closed_bits": cb, "open_mask": om, "candidates": []}
    for c in ranked[:run["timed"]]:
        p = tn.Plan(net, precision=run["precision"], complex_mult=run["complex_mult"], seed=c["seed"],
                    mem_weight=c["mem_weight"], **kw)
        info = p.info()
        leaf_of_gate, step_nodes = p.tree(circ.n_gates)
        first = (rqcgen.timed_block_first(info["log2_slices"], run["block"], rqcgen.CONFIGS[name]["seed"])
                 if run["block"] else 0)
        out["candidates"].append(dict(seed=c["seed"], mem_weight=c["mem_weight"], model_seconds=c["model_seconds"],
                                      log2_slices=info["log2_slices"], sliced_wires=p.sliced_wires(),
                                      block_first=first, check_slices=run["check_slices"],
                                      leaf_of_gate=leaf_of_gate, step_nodes=step_nodes))
        print(f"seed {c['seed']} w {c['mem_weight']}: model {c['model_seconds']:.3f} s, S {info['log2_slices']}, "
              f"block {first}")
    path = os.path.join(HERE, f"{name}_plans.json")
    with open(path, "w") as f:
        json.dump(out, f, separators=(",", ":"))
    print(path)


def read(name: str) -> dict:
    with open(os.path.join(HERE, f"{name}_plans.json")) as f:
        return json.load(f)


if __name__ == "__main__":
    for n in sys.argv[1:] or ["c3", "c5"]:
        write(n)
