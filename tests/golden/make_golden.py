"""Write the oracle's expected amplitudes for the larger synthetic workloads.

Calls only `oracle/` (and the seeded generator `rqcgen`).  Output: one text file
per workload, `<name>_amplitudes.txt`, with a header line and one amplitude per
line ("re im", 17 significant digits), in the batch order sum_j b(open_j) 2^j.

    python tests/golden/make_golden.py c2 c3 c5 c5block c3order

With the amplitudes of c2 and c3 it also writes `<name>_xeb.txt`, their linear
XEB computed by the oracle.  "c5block" writes the partial sums over the first
slices of each candidate plan's timed block (the plan parameters are read as
data from `c5_plans.json`, written by make_plan_data.py); "c3order"
stores the oracle's own contraction order for the 42-qubit batch, so that the
oracle can be timed without re-planning.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import rqcgen  # noqa: E402
from oracle import tensornet  # noqa: E402


# the oracle's order for each workload: its own greedy, or its recursive
# bisection (best of `trials` seeded trials) where greedy is far too costly
ORDER = {"c2": dict(method="greedy"), "c3": dict(method="bisect", trials=60, seed=100)}


def write(name: str) -> None:
    circ, open_mask, closed = rqcgen.config_circuit(name)
    t0 = time.time()
    amps = tensornet.batch_amplitudes(circ, closed, open_mask, max_log2=27, **ORDER[name])
    dt = time.time() - t0
    path = os.path.join(HERE, f"{name}_amplitudes.txt")
    with open(path, "w") as f:
        f.write(f"# {name}: n={circ.n_qubits} open_mask={open_mask:#x} closed={closed:#x} "
                f"count={amps.size} oracle=tensornet complex128 order={ORDER[name]} ({dt:.1f} s)\n")
        for a in amps:
            f.write(f"{a.real:.17e} {a.imag:.17e}\n")
    print(path, f"{dt:.1f} s")


def write_sliced(name: str, n_slices: int) -> None:
    """A partial sum over slices for networks too large for the whole batch: the
    oracle slices the wires of its own choice (the extra wires its bisection
    order needs under a 2^25 bound) and sums slice ids 0..n_slices-1, slice id s
    setting the j-th wire to bit j of s.  The wire list is written with it so
    that a test can hand the same slice set to the library."""
    circ, open_mask, closed = rqcgen.config_circuit(name)
    net = tensornet.CircuitNetwork(circ, closed, open_mask)
    t0 = time.time()
    merges, wires = net.plan([], max_log2=25, method="bisect", trials=12, seed=100)
    amps = net.contract_in_order(merges, wires, range(n_slices))
    dt = time.time() - t0
    path = os.path.join(HERE, f"{name}_slices_amplitudes.txt")
    with open(path, "w") as f:
        f.write(f"# {name}: n={circ.n_qubits} open_mask={open_mask:#x} closed={closed:#x} count={amps.size} "
                f"slices=0..{n_slices - 1} oracle=tensornet complex128 ({dt:.1f} s)\n")
        f.write("# wires " + " ".join(f"{q},{t}" for q, t in wires) + "\n")
        for a in amps:
            f.write(f"{a.real:.17e} {a.imag:.17e}\n")
    print(path, f"{dt:.1f} s")


def read_sliced(name: str):
    path = os.path.join(HERE, f"{name}_slices_amplitudes.txt")
    with open(path) as f:
        head = [f.readline(), f.readline()]
    wires = [tuple(int(x) for x in w.split(",")) for w in head[1].split()[2:]]
    n = int(head[0].split("slices=0..")[1].split()[0]) + 1
    data = np.loadtxt(path, comments="#")
    return wires, n, data[:, 0] + 1j * data[:, 1]


def write_block(name: str) -> None:
    """For every candidate plan in <name>_plans.json, two FP64 partial sums of
    the network with the candidate's sliced wires fixed (slice id s sets wire j
    to bit j of s), contracted by the oracle along an order it builds from the
    candidate's tree shape (tensornet.CircuitNetwork.tree_order), sub-sliced by
    the oracle itself under 2^27 entries: over slice ids block_first ..
    block_first + check_slices - 1 (the start of the benchmark's timed block),
    and over a seeded sample of as many slice ids spread over all 2^S
    (rqcgen.slice_sample, seed of the workload).  The second is the scale of a
    typical partial sum: a block whose fixed slice bits route every path
    through the fSim entries cos(pi/2) ~ 6e-17 sums to almost nothing, and is
    then compared on that scale."""
    with open(os.path.join(HERE, f"{name}_plans.json")) as f:
        data = json.load(f)
    circ, open_mask, closed = rqcgen.config_circuit(name)
    assert data["closed_bits"] == closed and data["open_mask"] == open_mask
    net = tensornet.CircuitNetwork(circ, closed, open_mask)
    path = os.path.join(HERE, f"{name}_block_amplitudes.txt")
    with open(path, "w") as f:
        f.write(f"# {name}: n={circ.n_qubits} open_mask={open_mask:#x} closed={closed:#x} oracle=tensornet complex128; "
                f"per candidate plan: partial sums over its first timed slices and over a seeded slice sample\n")
        for c in data["candidates"]:
            wires = [tuple(w) for w in c["sliced_wires"]]
            t0 = time.time()
            merges, extra = net.plan_along_tree(wires, c["leaf_of_gate"], [tuple(p) for p in c["step_nodes"]],
                                                max_log2=27)
            ids = range(c["block_first"], c["block_first"] + c["check_slices"])
            sample = [int(x) for x in rqcgen.slice_sample(c["log2_slices"], c["check_slices"],
                                                         rqcgen.CONFIGS[name]["seed"])]
            for kind, sl in (("block", list(ids)), ("sample", sample)):
                amps = net.contract_in_order(merges, wires, sl, extra)
                f.write(f"# candidate seed={c['seed']} mem_weight={c['mem_weight']} kind={kind} "
                        f"slices={','.join(str(x) for x in sl)} count={amps.size} extra={len(extra)}\n")
                f.write("# wires " + " ".join(f"{q},{t}" for q, t in wires) + "\n")
                for a in amps:
                    f.write(f"{a.real:.17e} {a.imag:.17e}\n")
            print(f"seed {c['seed']} w {c['mem_weight']}: {time.time() - t0:.1f} s", flush=True)
    print(path)


def read_block(name: str) -> dict:
    """{(seed, mem_weight): {"block": section, "sample": section}}, a section
    being {"slices": [ids], "wires": [(q, t)], "amps": array}."""
    path = os.path.join(HERE, f"{name}_block_amplitudes.txt")
    out = {}
    cur = None
    with open(path) as f:
        for line in f:
            if line.startswith("# candidate"):
                kv = dict(tok.split("=", 1) for tok in line.split() if "=" in tok)
                cur = {"slices": [int(x) for x in kv["slices"].split(",")], "amps": []}
                out.setdefault((int(kv["seed"]), float(kv["mem_weight"])), {})[kv["kind"]] = cur
            elif line.startswith("# wires") and cur is not None:
                cur["wires"] = [tuple(int(x) for x in w.split(",")) for w in line.split()[2:]]
            elif not line.startswith("#") and line.strip() and cur is not None:
                re_, im_ = line.split()
                cur["amps"].append(float(re_) + 1j * float(im_))
    for v in out.values():
        for sec in v.values():
            sec["amps"] = np.array(sec["amps"])
    return out


def write_order(name: str) -> None:
    """The oracle's own order for the whole batch of `name` (recursive
    bisection, the same options as write()) and the extra wires it slices
    itself under 2^27 entries, stored as data."""
    circ, open_mask, closed = rqcgen.config_circuit(name)
    net = tensornet.CircuitNetwork(circ, closed, open_mask)
    t0 = time.time()
    opts = ORDER[name]
    merges, extra = net.plan([], max_log2=27, method=opts["method"], trials=opts.get("trials", 8),
                             seed=opts.get("seed", 0))
    path = os.path.join(HERE, f"{name}_oracle_order.json")
    with open(path, "w") as f:
        json.dump({"workload": name, "order": opts, "max_log2": 27, "n_tensors": len(net.legs),
                   "merges": merges, "extra": extra, "plan_seconds": time.time() - t0}, f, separators=(",", ":"))
    print(path, f"{len(extra)} extra wires")


def read(name: str) -> np.ndarray:
    path = os.path.join(HERE, f"{name}_amplitudes.txt")
    data = np.loadtxt(path, comments="#")
    return data[:, 0] + 1j * data[:, 1]


def write_xeb(name: str) -> None:
    """The oracle's linear XEB (main text, Eq. (1) with F = N<p> - 1) of the
    stored amplitudes of `name`, so that a reader of the amplitudes needs no
    oracle import to compare an XEB with it."""
    from oracle import xeb
    circ, _, _ = rqcgen.config_circuit(name)
    f_xeb = xeb.linear_xeb(read(name), circ.n_qubits)
    path = os.path.join(HERE, f"{name}_xeb.txt")
    with open(path, "w") as f:
        f.write(f"# {name}: n={circ.n_qubits} linear XEB of {name}_amplitudes.txt (oracle.xeb.linear_xeb)\n")
        f.write(f"{f_xeb:.17e}\n")
    print(path, f_xeb)


def read_xeb(name: str) -> float:
    return float(np.loadtxt(os.path.join(HERE, f"{name}_xeb.txt"), comments="#"))


if __name__ == "__main__":
    for n in sys.argv[1:] or ["c2"]:
        if n == "c5":
            write_sliced("c5", 2)
        elif n == "c5block":
            write_block("c5")
        elif n == "c3order":
            write_order("c3")
        else:
            write(n)
            write_xeb(n)
