"""Frugal rejection sampling from a batch of correlated amplitudes (main text,
section III: a batch of 2^k amplitudes from one contraction with k qubits left
open, then frugal sampling, yields one sample with probability close to 1).

The sampler walks a caller-given sequence of draws; draw t proposes the batch
member c_t and carries a uniform u_t in [0, 1).  It accepts the first draw with

    u_t * M < N p(c_t),     N = 2^n, p = |a|^2,

i.e. with probability min(1, N p / M).  An accepted member is distributed as
min(1, N p / M) normalised over the batch, which is p normalised whenever no
member has N p > M (rare under the Porter-Thomas law of Eq. (1) for M of ~10),
so the output is a sample of the batch's conditional distribution.  The
products are formed as written (no fused multiply-add) so that another FP64
implementation takes the same accept decisions.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np


def accept_mask(amplitudes: np.ndarray, n_qubits: int, m_bound: float, candidates: np.ndarray,
                uniforms: np.ndarray) -> np.ndarray:
    """Per draw: whether u_t * M < 2^n |a_{c_t}|^2."""
    a = np.asarray(amplitudes, dtype=np.complex128).reshape(-1)
    c = np.asarray(candidates, dtype=np.int64)
    u = np.asarray(uniforms, dtype=np.float64)
    re, im = a.real[c], a.imag[c]
    p = re * re + im * im
    return u * np.float64(m_bound) < np.ldexp(p, n_qubits)


def frugal_sample(amplitudes: np.ndarray, n_qubits: int, m_bound: float, candidates: np.ndarray,
                  uniforms: np.ndarray) -> int:
    """Index (into the draws) of the first accepted draw, or -1 if none is."""
    acc = accept_mask(amplitudes, n_qubits, m_bound, candidates, uniforms)
    hits = np.flatnonzero(acc)
    return int(hits[0]) if hits.size else -1


def acceptance_law(amplitudes: np.ndarray, n_qubits: int, m_bound: float) -> np.ndarray:
    """Probability that one uniformly proposed member is accepted, per member:
    min(1, N p / M) / (batch size)."""
    a = np.asarray(amplitudes, dtype=np.complex128).reshape(-1)
    p = a.real * a.real + a.imag * a.imag
    return np.minimum(1.0, np.ldexp(p, n_qubits) / m_bound) / a.size
