"""Write the oracle's expected amplitudes for the larger synthetic workloads.

Calls only `oracle/` (and the seeded generator `rqcgen`).  Output: one text file
per workload, `<name>_amplitudes.txt`, with a header line and one amplitude per
line ("re im", 17 significant digits), in the batch order sum_j b(open_j) 2^j.

    python tests/golden/make_golden.py c2 c3 c5

With the amplitudes of c2 and c3 it also writes `<name>_xeb.txt`, their linear
XEB computed by the oracle.
"""
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
        else:
            write(n)
            write_xeb(n)
