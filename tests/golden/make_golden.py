"""Write the oracle's expected amplitudes for the larger synthetic workloads.

Calls only `oracle/` (and the seeded generator `rqcgen`).  Output: one text file
per workload, `<name>_amplitudes.txt`, with a header line and one amplitude per
line ("re im", 17 significant digits), in the batch order sum_j b(open_j) 2^j.

    python tests/golden/make_golden.py c2
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


def read(name: str) -> np.ndarray:
    path = os.path.join(HERE, f"{name}_amplitudes.txt")
    data = np.loadtxt(path, comments="#")
    return data[:, 0] + 1j * data[:, 1]


if __name__ == "__main__":
    for n in sys.argv[1:] or ["c2"]:
        write(n)
