"""One pairwise contraction and one index permutation, complex128 (SI, Eq. (2)).

For tensors whose every index has dimension 2, stored with index 0 fastest
(column-major, SI figure S7 caption), C = sum over the shared wires of A * B.
Written as numpy.einsum over one axis per wire: the plain definition, with no
reshaping into matrices.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

from typing import Sequence

import numpy as np


def to_axes(flat: np.ndarray, rank: int) -> np.ndarray:
    """Column-major flat tensor -> numpy array whose axis i is wire position i."""
    return np.asarray(flat).reshape((2,) * rank, order="F") if rank else np.asarray(flat).reshape(())


def from_axes(arr: np.ndarray) -> np.ndarray:
    return np.asarray(arr).reshape(-1, order="F")


def contract_pair(a: np.ndarray, a_wires: Sequence[int], b: np.ndarray, b_wires: Sequence[int],
                  c_wires: Sequence[int]) -> np.ndarray:
    """C[c_wires] = sum over wires shared by A and B of A[a_wires] B[b_wires];
    flat column-major arrays in and out."""
    letters = {}
    for w in list(a_wires) + list(b_wires):
        if w not in letters:
            letters[w] = chr(ord("a") + len(letters)) if len(letters) < 26 else chr(ord("A") + len(letters) - 26)
    spec = "".join(letters[w] for w in a_wires) + "," + "".join(letters[w] for w in b_wires) + "->" + \
        "".join(letters[w] for w in c_wires)
    out = np.einsum(spec, to_axes(np.asarray(a, dtype=np.complex128), len(a_wires)),
                    to_axes(np.asarray(b, dtype=np.complex128), len(b_wires)))
    return from_axes(out)


def permute(t: np.ndarray, rank: int, perm: Sequence[int]) -> np.ndarray:
    """Output position p carries the input index at position perm[p]."""
    return from_axes(np.transpose(to_axes(t, rank), list(perm)))
