"""Seeded synthetic random-quantum-circuit (RQC) inputs.

This module is the one piece shared by the library side and the FP64 oracle: it
draws circuits and bitstrings from a seed and holds none of the contraction
method's arithmetic (no tensor network, no amplitudes, no XEB).

Circuit structure (paper, SI section "Random quantum circuits"):

* qubits sit on a rectangular R x C grid, optionally with sites removed;
* a circuit of d cycles interlaces d + 1 layers of single-qubit gates drawn from
  {sqrt(X), sqrt(Y), sqrt(W)} with d layers of two-qubit fSim gates, one layer per
  cycle, in the patterns A, B, C, D;
* within every block of four cycles that contains A, B, C and D each
  nearest-neighbour pair receives exactly one two-qubit gate; the 8-cycle
  sequence is ABCDCDAB and the 12-cycle one ABCDCDABABCD.

Readings where the paper is silent (figure S1 carries no data):

* pattern geometry on the grid: A = horizontal pairs (r,c)-(r,c+1) with r+c
  even, B = vertical pairs (r,c)-(r+1,c) with r+c even, C = horizontal with r+c
  odd, D = vertical with r+c odd.  Each is a matching and A+B+C+D covers every
  nearest-neighbour pair exactly once;
* d not divisible by 4: the first d letters of the periodic string ABCDCDAB;
* single-qubit layers: layer 0 uniform over the three gates, later layers uniform
  over the two gates that differ from the previous gate on that qubit;
* fSim: the (2,2) entry is exp(i(D+ - D-)) cos(theta) (as printed it repeats the
  (1,1) entry, which is not unitary for D- != 0); all Delta are 0 here;
* two-qubit matrix convention: row/column index = 2*b(q0) + b(q1), row = output,
  column = input, q0 = the first listed qubit (left or upper site);
* qubit index = row-major order of the sites present; the state-vector index of a
  bitstring is sum_q b_q 2^q.
"""
from __future__ import annotations

import dataclasses
import json
import math
from typing import List, Optional, Tuple

import numpy as np

__all__ = [
    "sqrt_x", "sqrt_y", "sqrt_w", "fsim", "Circuit", "sycamore_style",
    "PATTERN_SEQUENCE", "pattern_pairs", "cycle_patterns", "CONFIGS",
    "config_circuit", "random_bits", "slice_sample", "timed_block_first",
]

_S = math.sqrt(2.0) / 2.0


def sqrt_x() -> np.ndarray:
    """sqrt(X) of the SI gate set: (sqrt2/2) [[1, -i], [-i, 1]]."""
    return _S * np.array([[1.0, -1.0j], [-1.0j, 1.0]], dtype=np.complex128)


def sqrt_y() -> np.ndarray:
    """sqrt(Y) of the SI gate set: (sqrt2/2) [[1, -1], [1, 1]]."""
    return _S * np.array([[1.0, -1.0], [1.0, 1.0]], dtype=np.complex128)


def sqrt_w() -> np.ndarray:
    """sqrt(W) of the SI gate set: (sqrt2/2) [[1, -(sqrt2/2)(1+i)], [(sqrt2/2)(1-i), 1]]."""
    return _S * np.array([[1.0, -_S * (1.0 + 1.0j)], [_S * (1.0 - 1.0j), 1.0]],
                         dtype=np.complex128)


def fsim(theta: float, phi: float, d_plus: float = 0.0, d_minus: float = 0.0,
         d_minus_off: float = 0.0) -> np.ndarray:
    """Five-parameter fSim gate of the SI, with the (2,2) entry read as
    exp(i(D+ - D-)) cos(theta) so that the matrix is unitary."""
    u = np.zeros((4, 4), dtype=np.complex128)
    u[0, 0] = 1.0
    u[1, 1] = np.exp(1j * (d_plus + d_minus)) * math.cos(theta)
    u[1, 2] = -1j * np.exp(1j * (d_plus - d_minus_off)) * math.sin(theta)
    u[2, 1] = -1j * np.exp(1j * (d_plus + d_minus_off)) * math.sin(theta)
    u[2, 2] = np.exp(1j * (d_plus - d_minus)) * math.cos(theta)
    u[3, 3] = np.exp(1j * (2.0 * d_plus - phi))
    return u


SINGLE_QUBIT_GATES = (sqrt_x, sqrt_y, sqrt_w)
SINGLE_QUBIT_NAMES = ("sqrt_x", "sqrt_y", "sqrt_w")
PATTERN_SEQUENCE = "ABCDCDAB"


def cycle_patterns(cycles: int) -> str:
    """Pattern letters of a d-cycle circuit: the first d letters of ABCDCDAB..."""
    reps = cycles // len(PATTERN_SEQUENCE) + 1
    return (PATTERN_SEQUENCE * reps)[:cycles]


def pattern_pairs(rows: int, cols: int, letter: str,
                  present: Optional[set] = None) -> List[Tuple[Tuple[int, int], Tuple[int, int]]]:
    """Nearest-neighbour site pairs of one two-qubit pattern, in row-major order of
    their first site.  Pairs touching a removed site are dropped."""
    horizontal = letter in "AC"
    parity = 0 if letter in "AB" else 1
    out = []
    for r in range(rows):
        for c in range(cols):
            if (r + c) % 2 != parity:
                continue
            other = (r, c + 1) if horizontal else (r + 1, c)
            if other[0] >= rows or other[1] >= cols:
                continue
            if present is not None and ((r, c) not in present or other not in present):
                continue
            out.append(((r, c), other))
    return out


@dataclasses.dataclass
class Circuit:
    """A gate list in time order.  gate_qubits[g] = (q0, q1) with q1 = -1 for a
    single-qubit gate; gate_matrices[g] is 2x2 or 4x4 complex128 (row = output);
    gate_layer[g] is the layer index (2*cycle for the single-qubit layer before a
    cycle, 2*cycle+1 for the two-qubit layer, 2*d for the final single-qubit layer)."""
    n_qubits: int
    gate_qubits: np.ndarray          # int32 [G, 2]
    gate_matrices: List[np.ndarray]  # complex128, 2x2 or 4x4
    gate_layer: np.ndarray           # int32 [G]
    rows: int = 0
    cols: int = 0
    cycles: int = 0
    seed: int = 0
    sites: Optional[List[Tuple[int, int]]] = None
    gate_names: Optional[List[str]] = None

    @property
    def n_gates(self) -> int:
        return int(self.gate_qubits.shape[0])

    def n_two_qubit(self) -> int:
        return int(np.sum(self.gate_qubits[:, 1] >= 0))

    def flat_matrices(self) -> np.ndarray:
        """All gate matrices concatenated, row-major, as interleaved complex128
        (float64 [sum of 4 or 16 entries, 2])."""
        parts = [m.reshape(-1) for m in self.gate_matrices]
        flat = np.concatenate(parts).astype(np.complex128)
        return np.ascontiguousarray(flat.view(np.float64))

    def to_json(self) -> str:
        return json.dumps({
            "n_qubits": self.n_qubits, "rows": self.rows, "cols": self.cols,
            "cycles": self.cycles, "seed": self.seed,
            "sites": self.sites,
            "gates": [
                {"qubits": [int(q) for q in self.gate_qubits[g] if q >= 0],
                 "layer": int(self.gate_layer[g]),
                 "name": (self.gate_names[g] if self.gate_names else None),
                 "re": np.real(self.gate_matrices[g]).reshape(-1).tolist(),
                 "im": np.imag(self.gate_matrices[g]).reshape(-1).tolist()}
                for g in range(self.n_gates)],
        })

    @staticmethod
    def from_json(text: str) -> "Circuit":
        d = json.loads(text)
        qs, mats, layers, names = [], [], [], []
        for g in d["gates"]:
            q = list(g["qubits"]) + ([-1] if len(g["qubits"]) == 1 else [])
            qs.append(q)
            dim = 2 if len(g["qubits"]) == 1 else 4
            mats.append((np.array(g["re"]) + 1j * np.array(g["im"])).reshape(dim, dim))
            layers.append(g["layer"])
            names.append(g.get("name"))
        return Circuit(d["n_qubits"], np.array(qs, dtype=np.int32), mats,
                       np.array(layers, dtype=np.int32), d.get("rows", 0), d.get("cols", 0),
                       d.get("cycles", 0), d.get("seed", 0),
                       [tuple(s) for s in d["sites"]] if d.get("sites") else None, names)


def _connected(sites: set) -> bool:
    if not sites:
        return True
    start = next(iter(sites))
    seen = {start}
    stack = [start]
    while stack:
        r, c = stack.pop()
        for nb in ((r + 1, c), (r - 1, c), (r, c + 1), (r, c - 1)):
            if nb in sites and nb not in seen:
                seen.add(nb)
                stack.append(nb)
    return len(seen) == len(sites)


def sycamore_style(rows: int, cols: int, cycles: int, seed: int, missing_sites: int = 0,
                   theta: float = math.pi / 2, phi: float = math.pi / 6) -> Circuit:
    """Draw a Sycamore-style RQC on a rows x cols grid (seeded numpy PCG64).

    Draw order from the one generator: the removed sites (each uniform over the
    sites whose removal keeps the grid connected), then the single-qubit gate
    indices layer by layer, qubit by qubit."""
    rng = np.random.default_rng(seed)
    present = {(r, c) for r in range(rows) for c in range(cols)}
    for _ in range(missing_sites):
        cands = sorted(s for s in present if _connected(present - {s}))
        pick = cands[int(rng.integers(len(cands)))]
        present.remove(pick)
    sites = sorted(present)
    index = {s: i for i, s in enumerate(sites)}
    n = len(sites)
    u2 = fsim(theta, phi)
    one_q = [f() for f in SINGLE_QUBIT_GATES]

    qubits, mats, layers, names = [], [], [], []
    prev = np.full(n, -1, dtype=np.int64)

    def single_layer(layer: int) -> None:
        for q in range(n):
            if prev[q] < 0:
                choice = int(rng.integers(3))
            else:
                choice = int((prev[q] + 1 + rng.integers(2)) % 3)
            prev[q] = choice
            qubits.append((q, -1))
            mats.append(one_q[choice])
            layers.append(layer)
            names.append(SINGLE_QUBIT_NAMES[choice])

    letters = cycle_patterns(cycles)
    for cyc, letter in enumerate(letters):
        single_layer(2 * cyc)
        for a, b in pattern_pairs(rows, cols, letter, present):
            qubits.append((index[a], index[b]))
            mats.append(u2)
            layers.append(2 * cyc + 1)
            names.append("fsim_" + letter)
    single_layer(2 * cycles)
    return Circuit(n, np.array(qubits, dtype=np.int32), mats, np.array(layers, dtype=np.int32),
                   rows, cols, cycles, seed, sites, names)


def random_bits(n_qubits: int, seed: int, stream: int = 1) -> int:
    """A uniformly random closed-bit assignment packed as an int (bit q = qubit q),
    drawn from a generator keyed by (seed, stream)."""
    rng = np.random.default_rng([seed, stream])
    bits = rng.integers(0, 2, size=n_qubits)
    return int(sum(int(b) << q for q, b in enumerate(bits)))


def slice_sample(n_slices_log2: int, count: int, seed: int) -> np.ndarray:
    """`count` distinct slice ids drawn uniformly without replacement from
    [0, 2^n_slices_log2), keyed by seed; returned sorted ascending (uint64)."""
    total = 1 << n_slices_log2
    count = min(count, total)
    rng = np.random.default_rng([seed, 7])
    if total <= (1 << 24):
        ids = rng.choice(total, size=count, replace=False)
    else:
        got: set = set()
        while len(got) < count:
            got.update(int(x) for x in rng.integers(0, total, size=count - len(got)))
        ids = np.array(sorted(got)[:count])
    return np.sort(np.asarray(ids, dtype=np.uint64))


def timed_block_first(n_slices_log2: int, block: int, seed: int) -> int:
    """First slice id of a seeded aligned block of `block` consecutive slice ids
    (block a power of two) in [0, 2^n_slices_log2): block index uniform,
    drawn from a generator keyed by (seed, 13); 0 when the block covers all."""
    total = 1 << n_slices_log2
    if block >= total:
        return 0
    return int(np.random.default_rng([seed, 13]).integers(total // block)) * block


# The synthetic workloads: grid, cycles, seed, removed sites, open qubits, bound.
CONFIGS = {
    "c1": dict(rows=3, cols=4, cycles=8, seed=1, missing=0, k_open=12, log2_bound=30,
               log2_slices=0),
    "c2": dict(rows=5, cols=6, cycles=14, seed=2, missing=0, k_open=10, log2_bound=26,
               log2_slices=0),
    "c3": dict(rows=6, cols=7, cycles=16, seed=3, missing=0, k_open=12, log2_bound=28,
               log2_slices=12),
    "c5": dict(rows=6, cols=9, cycles=20, seed=5, missing=1, k_open=6, log2_bound=30,
               log2_slices=20),
}


def config_circuit(name: str) -> Tuple[Circuit, int, int]:
    """(circuit, open_mask, closed_bits) of a named synthetic workload.  The open
    qubits are the last k_open qubits in row-major order; the closed bits are
    uniform random from the config's seed (bits at open positions are zero)."""
    cfg = CONFIGS[name]
    circ = sycamore_style(cfg["rows"], cfg["cols"], cfg["cycles"], cfg["seed"], cfg["missing"])
    n = circ.n_qubits
    k = cfg["k_open"]
    open_mask = 0
    for q in range(n - k, n):
        open_mask |= 1 << q
    closed = random_bits(n, cfg["seed"]) & ~open_mask
    return circ, open_mask, closed
