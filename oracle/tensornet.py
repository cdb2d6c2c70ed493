"""Tensor-network contraction of a circuit amplitude batch, complex128 on the CPU.

What it computes (SI, TN section and figure S2; main text, section II):

* every gate is a tensor whose legs are wires: a single-qubit gate U has legs
  (out, in) with entries U[out, in]; a two-qubit gate has legs
  (out0, out1, in0, in1) with entries U[2 out0 + out1, 2 in0 + in1];
* wires carry the canonical label (q, t) = "qubit q after its t-th gate", so
  (q, 0) is the input wire and (q, T_q) the output wire of qubit q;
* the initial state |0> is a rank-1 tensor [1, 0] on every input wire; a closed
  output qubit with bit b gets the rank-1 tensor e_b on its output wire; the
  output wires of open qubits stay free, so contracting the network yields the
  2^k amplitudes of a correlated batch (main text, section III);
* slicing (main text, section II): fixing a set of wires to values turns the
  network into one of 2^S smaller networks; the sum over all assignments equals
  the unsliced contraction.  Slice id s sets the j-th sliced wire to bit j of s.

How: the oracle's own greedy pairwise order (at each step merge the pair of
connected tensors whose merge removes the most memory, size(C) - size(A) -
size(B) smallest, ties to the lowest tensor ids), executed with numpy.tensordot.
Larger networks use the recursive bisection order of oracle.order instead.
When the order would create a tensor larger than 2^max_log2 entries the
oracle slices extra wires of its own choosing and sums the sub-networks, which
changes nothing but memory.  No blocking, fusion or reordering beyond that.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import heapq
from typing import Dict, Iterable, List, Optional, Sequence, Tuple

import numpy as np

Label = Tuple[int, int]


class CircuitNetwork:
    """The tensor network of one circuit and one batch (closed bits + open mask)."""

    def __init__(self, circuit, closed_bits: int, open_mask: int):
        n = circuit.n_qubits
        self.n_qubits = n
        t = [0] * n
        legs: List[Tuple[Label, ...]] = []
        data: List[np.ndarray] = []
        for q in range(n):                       # |0> on every input wire
            legs.append(((q, 0),))
            data.append(np.array([1.0, 0.0], dtype=np.complex128))
        for g in range(circuit.n_gates):
            q0, q1 = int(circuit.gate_qubits[g, 0]), int(circuit.gate_qubits[g, 1])
            u = np.asarray(circuit.gate_matrices[g], dtype=np.complex128)
            if q1 < 0:
                legs.append(((q0, t[q0] + 1), (q0, t[q0])))
                data.append(u.copy())
                t[q0] += 1
            else:
                legs.append(((q0, t[q0] + 1), (q1, t[q1] + 1), (q0, t[q0]), (q1, t[q1])))
                data.append(u.reshape(2, 2, 2, 2).copy())
                t[q0] += 1
                t[q1] += 1
        self.open_legs: List[Label] = []
        for q in range(n):
            out = (q, t[q])
            if (open_mask >> q) & 1:
                self.open_legs.append(out)
            else:
                b = (closed_bits >> q) & 1
                legs.append((out,))
                data.append(np.array([1.0 - b, float(b)], dtype=np.complex128))
        self.legs = legs
        self.data = data
        self.wire_count = t

    # -- planning ---------------------------------------------------------------
    @staticmethod
    def greedy_order(leg_sets: Sequence[frozenset]) -> Tuple[List[Tuple[int, int]], List[frozenset]]:
        """Greedy pairwise order over leg sets.  Returns the merge list (ids into
        a growing list: the i-th merge creates id len(leg_sets) + i) and the leg
        set of every id."""
        sets: List[frozenset] = list(leg_sets)
        alive = set(range(len(sets)))
        owner: Dict[Label, set] = {}
        for i, s in enumerate(sets):
            for leg in s:
                owner.setdefault(leg, set()).add(i)
        heap: List[Tuple[int, int, int]] = []

        def push(i: int, j: int) -> None:
            a, b = (i, j) if i < j else (j, i)
            c = sets[a] ^ sets[b]
            score = (1 << len(c)) - (1 << len(sets[a])) - (1 << len(sets[b]))
            heapq.heappush(heap, (score, a, b))

        for leg, ids in owner.items():
            if len(ids) == 2:
                i, j = sorted(ids)
                push(i, j)
        merges: List[Tuple[int, int]] = []
        while heap:
            _, a, b = heapq.heappop(heap)
            if a not in alive or b not in alive:
                continue
            c = sets[a] ^ sets[b]
            cid = len(sets)
            sets.append(c)
            alive.discard(a)
            alive.discard(b)
            alive.add(cid)
            merges.append((a, b))
            nbrs = set()
            for leg in sets[a] | sets[b]:
                ids = owner.get(leg)
                if ids is None:
                    continue
                ids.discard(a)
                ids.discard(b)
                if leg in c:
                    ids.add(cid)
                    nbrs.update(x for x in ids if x != cid)
            for x in sorted(nbrs):
                push(x, cid)
        # disconnected components: outer products, smallest first
        rest = sorted(alive, key=lambda i: (len(sets[i]), i))
        while len(rest) > 1:
            a, b = rest[0], rest[1]
            cid = len(sets)
            sets.append(sets[a] ^ sets[b])
            merges.append((a, b))
            rest = sorted(rest[2:] + [cid], key=lambda i: (len(sets[i]), i))
        return merges, sets

    def plan(self, fixed_legs: Iterable[Label], max_log2: int = 27, method: str = "greedy",
             trials: int = 8, seed: int = 0) -> Tuple[List[Tuple[int, int]], List[Label]]:
        """Pairwise order for the network with `fixed_legs` removed ("greedy", or
        "bisect" for the recursive bisection of oracle.order), plus the extra
        wires the oracle itself slices so that no tensor of that order exceeds
        2^max_log2 entries (the order is kept; only legs are removed)."""
        fixed = set(fixed_legs)
        base = [frozenset(l for l in legs if l not in fixed) for legs in self.legs]
        if method == "greedy":
            merges, sets = self.greedy_order(base)
        elif method == "bisect":
            from . import order as _order
            merges, sets = _order.best_bisection_order(base, trials=trials, seed=seed)
        else:
            raise ValueError(f"unknown order method {method!r}")
        return merges, self._extra_slices(sets, max_log2)

    def tree_order(self, leaf_of_gate: Sequence[int],
                   step_nodes: Sequence[Tuple[int, int]]) -> List[Tuple[int, int]]:
        """A pairwise order given by its tree shape (SI, TN section: the order is
        a list of two-tuples): gate g belongs to group leaf_of_gate[g]; every
        rank-1 tensor (initial state, output projector) joins the group of the
        gate that shares its wire; each group is first contracted to one tensor
        with the oracle's own greedy order, then the groups are merged pairwise
        as step_nodes says (ids: groups 0..L-1, the j-th pair creates L + j).
        Returns the merge list over this network's tensors.  Any complete
        binary tree gives the same contraction (only rounding differs), so the
        tree only decides speed and memory; it is checked to be complete."""
        n, n_gates = self.n_qubits, len(leaf_of_gate)
        n_t = len(self.legs)
        if n + n_gates > n_t:
            raise ValueError("more gates than the network holds")
        group: List[Optional[int]] = [None] * n_t
        owner: Dict[Label, List[int]] = {}
        for g in range(n_gates):
            group[n + g] = int(leaf_of_gate[g])
            for leg in self.legs[n + g]:
                owner.setdefault(leg, []).append(n + g)
        for i in range(n_t):
            if group[i] is None:
                if len(self.legs[i]) != 1 or len(owner.get(self.legs[i][0], [])) != 1:
                    raise ValueError(f"tensor {i} touches no single gate")
                group[i] = group[owner[self.legs[i][0]][0]]
        n_groups = max(group) + 1
        if min(group) < 0 or set(group) != set(range(n_groups)):
            raise ValueError("groups must be numbered 0..L-1 without gaps")
        merges: List[Tuple[int, int]] = []
        node_id: Dict[int, int] = {}
        for grp in range(n_groups):
            members = [i for i in range(n_t) if group[i] == grp]
            sub, _ = self.greedy_order([frozenset(self.legs[i]) for i in members])
            ids = list(members)
            for a, b in sub:
                merges.append((ids[a], ids[b]))
                ids.append(n_t + len(merges) - 1)
            node_id[grp] = ids[-1]
        for j, (x, y) in enumerate(step_nodes):
            if x not in node_id or y not in node_id or x == y:
                raise ValueError(f"step {j} merges an unknown node")
            merges.append((node_id.pop(x), node_id.pop(y)))
            node_id[n_groups + j] = n_t + len(merges) - 1
        used = [i for m in merges for i in m]
        if len(merges) != n_t - 1 or len(set(used)) != len(used) or len(node_id) != 1:
            raise ValueError("the tree does not contract every tensor exactly once")
        return merges

    def plan_along_tree(self, fixed_legs: Iterable[Label], leaf_of_gate: Sequence[int],
                        step_nodes: Sequence[Tuple[int, int]],
                        max_log2: int = 27) -> Tuple[List[Tuple[int, int]], List[Label]]:
        """tree_order() plus the extra wires the oracle slices itself so that no
        tensor of that order (with `fixed_legs` removed) exceeds 2^max_log2."""
        merges = self.tree_order(leaf_of_gate, step_nodes)
        fixed = set(fixed_legs)
        sets = [frozenset(l for l in legs if l not in fixed) for legs in self.legs]
        for a, b in merges:
            sets.append(sets[a] ^ sets[b])
        return merges, self._extra_slices(sets, max_log2)

    def _extra_slices(self, sets: Sequence[frozenset], max_log2: int) -> List[Label]:
        """Wires the oracle slices so that no set exceeds max_log2 legs: the
        wire shared by most oversized sets first (never an open wire)."""
        extra: List[Label] = []
        open_set = set(self.open_legs)
        while True:
            gone = frozenset(extra)
            big = [s - gone for s in sets if len(s - gone) > max_log2]
            if not big:
                return extra
            counts: Dict[Label, int] = {}
            for s in big:
                for leg in s:
                    if leg not in open_set:
                        counts[leg] = counts.get(leg, 0) + 1
            if not counts:
                raise ValueError("open legs alone exceed the oracle's size limit")
            extra.append(max(sorted(counts), key=lambda l: counts[l]))

    @staticmethod
    def flops_of(merges: Sequence[Tuple[int, int]], sets: Sequence[frozenset]) -> int:
        """Complex multiply-adds of an order: 2^|legs(A) u legs(B)| per merge."""
        return sum(1 << len(sets[a] | sets[b]) for a, b in merges)

    # -- execution ---------------------------------------------------------------
    def _fixed_arrays(self, values: Dict[Label, int]):
        arrays, legs = [], []
        for lg, arr in zip(self.legs, self.data):
            keep = []
            idx = []
            for leg in lg:
                if leg in values:
                    idx.append(values[leg])
                else:
                    idx.append(slice(None))
                    keep.append(leg)
            arrays.append(arr[tuple(idx)])
            legs.append(tuple(keep))
        return arrays, legs

    def _run(self, merges, values: Dict[Label, int]) -> np.ndarray:
        arrays, legs = self._fixed_arrays(values)
        arrays = list(arrays)
        legs = list(legs)
        for a, b in merges:
            la, lb = legs[a], legs[b]
            shared = [l for l in la if l in lb]
            ax_a = [la.index(l) for l in shared]
            ax_b = [lb.index(l) for l in shared]
            out = np.tensordot(arrays[a], arrays[b], axes=(ax_a, ax_b))
            arrays.append(out)
            legs.append(tuple(l for l in la if l not in shared) + tuple(l for l in lb if l not in shared))
            arrays[a] = arrays[b] = None
        final, final_legs = arrays[-1], legs[-1]
        # amplitude index = sum_j b(open_j) 2^j: C order wants open_{k-1} first
        want = tuple(reversed(self.open_legs))
        if len(merges) == 0:
            final, final_legs = arrays[0], legs[0]
        perm = [final_legs.index(l) for l in want]
        return np.transpose(final, perm).reshape(-1)

    def contract_in_order(self, merges: Sequence[Tuple[int, int]], sliced: Sequence[Label],
                          slice_ids: Iterable[int], extra: Sequence[Label] = ()) -> np.ndarray:
        """Sum over slice ids of the network with `sliced` fixed (slice id s sets
        sliced[j] to bit j of s), contracted along a given order of this network
        (e.g. the order plan() returned together with these wires); each slice
        is itself the sum over every value of the `extra` wires."""
        total = np.zeros(1 << len(self.open_legs), dtype=np.complex128)
        for s in slice_ids:
            s = int(s)
            base = {leg: (s >> j) & 1 for j, leg in enumerate(sliced)}
            for sub in range(1 << len(extra)):
                values = dict(base)
                values.update({leg: (sub >> j) & 1 for j, leg in enumerate(extra)})
                total += self._run(merges, values)
        return total

    def contract(self, sliced: Sequence[Label] = (), slice_ids: Optional[Iterable[int]] = None,
                 max_log2: int = 27, method: str = "greedy", trials: int = 8, seed: int = 0) -> np.ndarray:
        """Sum over the given slice ids (all 2^S when None) of the network with the
        sliced wires fixed: slice id s sets sliced[j] to bit j of s.  Returns the
        2^k complex128 batch amplitudes (partial sums when not all slices)."""
        sliced = list(sliced)
        for leg in sliced:
            if leg in self.open_legs:
                raise ValueError("an open output wire cannot be sliced")
        merges, extra = self.plan(sliced, max_log2, method, trials, seed)
        if slice_ids is None:
            slice_ids = range(1 << len(sliced))
        total = np.zeros(1 << len(self.open_legs), dtype=np.complex128)
        for s in slice_ids:
            s = int(s)
            base = {leg: (s >> j) & 1 for j, leg in enumerate(sliced)}
            for sub in range(1 << len(extra)):
                values = dict(base)
                values.update({leg: (sub >> j) & 1 for j, leg in enumerate(extra)})
                total += self._run(merges, values)
        return total


def batch_amplitudes(circuit, closed_bits: int, open_mask: int, sliced: Sequence[Label] = (),
                     slice_ids: Optional[Iterable[int]] = None, max_log2: int = 27,
                     method: str = "greedy", trials: int = 8, seed: int = 0) -> np.ndarray:
    """Convenience wrapper: amplitudes (or a slice subset's partial sum) of one batch."""
    return CircuitNetwork(circuit, closed_bits, open_mask).contract(sliced, slice_ids, max_log2,
                                                                    method, trials, seed)
