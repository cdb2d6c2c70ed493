"""Linear cross-entropy benchmarking (main text, section IV, Eq. (1)).

Eq. (1) gives the density of x = N p (N = 2^n, p = |amplitude|^2 of a sampled
bitstring) for a sampler of XEB fidelity F:  P(x | F) = (F x + 1 - F) e^{-x}.
Its mean is E[x] = F * 2 + (1 - F) * 1 = 1 + F, so the fidelity estimated from a
set of bitstrings is the linear XEB  F = N <p> - 1.  With F = 1 the density is
x e^{-x} (ideal sampling); with F = 0 it is e^{-x}, the Porter-Thomas law of the
probabilities of uniformly chosen bitstrings.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np


def linear_xeb(amplitudes: np.ndarray, n_qubits: int) -> float:
    """F = 2^n * mean_i |a_i|^2 - 1 over the given amplitudes."""
    a = np.asarray(amplitudes, dtype=np.complex128).reshape(-1)
    if a.size == 0:
        raise ValueError("linear_xeb needs at least one amplitude")
    p = a.real * a.real + a.imag * a.imag
    return float(np.ldexp(np.mean(p), n_qubits) - 1.0)


def fxeb_density(x: np.ndarray, fidelity: float) -> np.ndarray:
    """Eq. (1): P(x | F) = (F x + 1 - F) exp(-x)."""
    x = np.asarray(x, dtype=np.float64)
    return (fidelity * x + (1.0 - fidelity)) * np.exp(-x)


def fxeb_moment(k: int, fidelity: float) -> float:
    """k-th raw moment of Eq. (1): F (k+1)! + (1 - F) k!  (closed form of the
    integral of x^k (F x + 1 - F) e^{-x} over x >= 0)."""
    import math
    return fidelity * math.factorial(k + 1) + (1.0 - fidelity) * math.factorial(k)


def sample_bitstrings(probs: np.ndarray, count: int, seed: int) -> np.ndarray:
    """Draw `count` indices from a probability vector (ideal sampler), seeded."""
    p = np.asarray(probs, dtype=np.float64)
    p = p / p.sum()
    rng = np.random.default_rng([seed, 11])
    return rng.choice(p.size, size=count, p=p)
