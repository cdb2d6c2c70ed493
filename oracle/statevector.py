"""Schroedinger (state-vector) simulation in complex128.

Main text, section II: an n-qubit state is a rank-n tensor with 2^n complex
entries; applying a gate contracts the gate's input indices with the state's
indices of the qubits it acts on.  Time O(m 2^n), memory O(2^n).

Conventions: the state-vector index of a computational basis state is
sum_q b_q 2^q.  A numpy array of shape (2,)*n in C order puts the most
significant bit first, so qubit q lives on axis n-1-q.  A two-qubit matrix has
row/column index 2*b(q0) + b(q1) (row = output), q0 the first listed qubit.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

from typing import Sequence

import numpy as np


def _axis(n: int, q: int) -> int:
    return n - 1 - q


def apply_gate(state: np.ndarray, n: int, qubits: Sequence[int], u: np.ndarray) -> np.ndarray:
    """Apply one gate to a (2,)*n state and return the new state."""
    if len(qubits) == 1:
        ax = _axis(n, qubits[0])
        out = np.tensordot(u, state, axes=([1], [ax]))
        return np.moveaxis(out, 0, ax)
    q0, q1 = qubits
    a0, a1 = _axis(n, q0), _axis(n, q1)
    u4 = u.reshape(2, 2, 2, 2)          # [out0, out1, in0, in1]
    out = np.tensordot(u4, state, axes=([2, 3], [a0, a1]))
    return np.moveaxis(out, [0, 1], [a0, a1])


def simulate(circuit) -> np.ndarray:
    """Final state U|0...0> as a flat complex128 vector indexed by sum_q b_q 2^q."""
    n = circuit.n_qubits
    state = np.zeros((2,) * n, dtype=np.complex128)
    state[(0,) * n] = 1.0
    for g in range(circuit.n_gates):
        q0, q1 = int(circuit.gate_qubits[g, 0]), int(circuit.gate_qubits[g, 1])
        qs = (q0,) if q1 < 0 else (q0, q1)
        state = apply_gate(state, n, qs, np.asarray(circuit.gate_matrices[g], dtype=np.complex128))
    # C-order flattening of axes (b_{n-1}, ..., b_0) gives index sum_q b_q 2^q.
    return state.reshape(-1)


def batch_indices(n: int, closed_bits: int, open_mask: int) -> np.ndarray:
    """State-vector indices of one correlated batch: the closed bits are fixed and
    the open qubits (ascending) run through all 2^k values, the j-th open qubit
    carrying bit j of the batch position."""
    open_q = [q for q in range(n) if (open_mask >> q) & 1]
    base = closed_bits & ~open_mask
    idx = np.empty(1 << len(open_q), dtype=np.int64)
    for j in range(idx.size):
        x = base
        for i, q in enumerate(open_q):
            if (j >> i) & 1:
                x |= 1 << q
        idx[j] = x
    return idx


def batch_amplitudes(psi: np.ndarray, n: int, closed_bits: int, open_mask: int) -> np.ndarray:
    """Amplitudes <x_c y|psi> of one batch, ordered by the open-qubit assignment y."""
    return psi[batch_indices(n, closed_bits, open_mask)]
