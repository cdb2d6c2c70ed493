"""The oracle's own contraction orders for larger networks.

The order only decides how fast and in how much memory the oracle reaches the
result; the result itself is the plain sum of the network, whatever the order.
SI, TN section: good orders come from partitioning the network's graph into
subtrees; this module does that with recursive balanced bisection (starts from
the graph Laplacian's Fiedler vector, numpy.linalg.eigh, and from random
splits, refined by passes of single-node moves that lower the number of cut
wires), after first folding every rank <= 2 tensor into a neighbour and merging
neighbours whose union is not larger than the larger of the two.  Small parts
are ordered greedily.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import math
from typing import Dict, List, Sequence, Tuple

import numpy as np


def _greedy(ids: List[int], sets: List[frozenset], merges: List[Tuple[int, int]]) -> int:
    """Greedy pairwise order inside a small part; returns the part's final id."""
    alive = list(ids)
    while len(alive) > 1:
        best = None
        for i in range(len(alive)):
            for j in range(i + 1, len(alive)):
                a, b = alive[i], alive[j]
                if not (sets[a] & sets[b]) and best is not None and best[0] < 0:
                    continue
                c = sets[a] ^ sets[b]
                score = (1 << len(c)) - (1 << len(sets[a])) - (1 << len(sets[b]))
                if not (sets[a] & sets[b]):
                    score = 1 << 62 if best is None else max(score, 0) + (1 << 61)
                if best is None or score < best[0]:
                    best = (score, i, j)
        _, i, j = best
        a, b = alive[i], alive[j]
        sets.append(sets[a] ^ sets[b])
        merges.append((a, b))
        nid = len(sets) - 1
        alive = [x for k, x in enumerate(alive) if k not in (i, j)] + [nid]
    return alive[0]


def _cut(side: Dict[int, int], edges: List[Tuple[int, int]]) -> int:
    return sum(1 for a, b in edges if side[a] != side[b])


def _fm(nodes: List[int], nbr: Dict[int, List[int]], side: Dict[int, int], rng, imbalance: float,
        passes: int = 6) -> int:
    """Passes of single-node moves with locking; each pass keeps its best prefix."""
    n = len(nodes)
    lo = max(1, int(math.floor(n * (0.5 - imbalance))))

    def cut() -> int:
        return sum(1 for v in nodes for u in nbr[v] if side[u] != side[v]) // 2

    best_cut = cut()
    for _ in range(passes):
        locked = set()
        cnt = [sum(1 for v in nodes if side[v] == 0), 0]
        cnt[1] = n - cnt[0]
        cur = best_cut
        trace = []
        for _ in range(n):
            best = None
            for v in nodes:
                if v in locked or cnt[side[v]] - 1 < lo:
                    continue
                g = sum(1 if side[u] != side[v] else -1 for u in nbr[v]) + 1e-3 * rng.random()
                if best is None or g > best[0]:
                    best = (g, v)
            if best is None:
                break
            g, v = best
            cnt[side[v]] -= 1
            side[v] ^= 1
            cnt[side[v]] += 1
            locked.add(v)
            cur -= round(g)
            trace.append((cur, v))
        if not trace:
            break
        k = min(range(len(trace)), key=lambda i: trace[i][0])
        if trace[k][0] >= best_cut:
            for _, v in trace:
                side[v] ^= 1
            break
        for _, v in trace[k + 1:]:
            side[v] ^= 1
        best_cut = trace[k][0]
    return best_cut


def _split(nodes: List[int], sets: List[frozenset], rng: np.random.Generator, imbalance: float
           ) -> Tuple[List[int], List[int]]:
    """Balanced bisection: spectral start (Fiedler vector) and random starts, each
    refined by _fm; the split with the fewest cut wires wins."""
    idx = {v: k for k, v in enumerate(nodes)}
    owner: Dict = {}
    for v in nodes:
        for leg in sets[v]:
            owner.setdefault(leg, []).append(v)
    edges = [(o[0], o[1]) for o in owner.values() if len(o) == 2]
    nbr: Dict[int, List[int]] = {v: [] for v in nodes}
    for a, b in edges:
        nbr[a].append(b)
        nbr[b].append(a)
    n = len(nodes)
    lap = np.zeros((n, n))
    for a, b in edges:
        i, j = idx[a], idx[b]
        lap[i, j] -= 1
        lap[j, i] -= 1
        lap[i, i] += 1
        lap[j, j] += 1
    _, vec = np.linalg.eigh(lap)
    best = None
    for start in range(3):
        if start < 2:
            fied = vec[:, 1] + 1e-9 * rng.standard_normal(n)
            order = np.argsort(fied)
        else:
            order = rng.permutation(n)
        side = {nodes[k]: (0 if r < n // 2 else 1) for r, k in enumerate(order)}
        c = _fm(nodes, nbr, side, rng, imbalance)
        if best is None or c < best[0]:
            best = (c, dict(side))
    side = best[1]
    return [v for v in nodes if side[v] == 0], [v for v in nodes if side[v] == 1]


def bisection_order(leg_sets: Sequence[frozenset], seed: int = 0, leaf: int = 8,
                    imbalance: float = 0.2) -> Tuple[List[Tuple[int, int]], List[frozenset]]:
    """Order (merge list, leg set per id) in the same format as
    CircuitNetwork.greedy_order."""
    rng = np.random.default_rng(seed)
    sets: List[frozenset] = list(leg_sets)
    merges: List[Tuple[int, int]] = []
    alive = set(range(len(sets)))
    # fold rank <= 2 tensors into a neighbour
    changed = True
    while changed:
        changed = False
        owner: Dict = {}
        for v in alive:
            for leg in sets[v]:
                owner.setdefault(leg, []).append(v)
        for v in sorted(alive):
            if v not in alive or len(sets[v]) > 2:
                continue
            nb = [u for leg in sets[v] for u in owner.get(leg, []) if u != v and u in alive]
            if not nb:
                continue
            u = max(nb, key=lambda x: (len(sets[x]), -x))
            sets.append(sets[u] ^ sets[v])
            merges.append((u, v))
            nid = len(sets) - 1
            alive -= {u, v}
            alive.add(nid)
            changed = True
            break
    # pre-contract neighbours whose merge is not larger than the larger of the two
    changed = True
    while changed:
        changed = False
        owner = {}
        for v in alive:
            for leg in sets[v]:
                owner.setdefault(leg, []).append(v)
        for leg, vs in sorted(owner.items()):
            if len(vs) != 2 or vs[0] not in alive or vs[1] not in alive:
                continue
            u, v = vs
            if len(sets[u] ^ sets[v]) <= max(len(sets[u]), len(sets[v])):
                sets.append(sets[u] ^ sets[v])
                merges.append((u, v))
                alive -= {u, v}
                alive.add(len(sets) - 1)
                changed = True
                break

    def rec(nodes: List[int]) -> int:
        if len(nodes) <= leaf:
            return _greedy(nodes, sets, merges)
        a, b = _split(nodes, sets, rng, imbalance)
        if not a or not b:
            return _greedy(nodes, sets, merges)
        ia, ib = rec(a), rec(b)
        sets.append(sets[ia] ^ sets[ib])
        merges.append((ia, ib))
        return len(sets) - 1

    rec(sorted(alive))
    return merges, sets


def order_flops(merges, sets, removed: frozenset = frozenset()) -> float:
    return sum(2.0 ** len((sets[a] | sets[b]) - removed) for a, b in merges)


def best_bisection_order(leg_sets: Sequence[frozenset], trials: int = 8, seed: int = 0):
    """Best of several randomised bisection orders by complex multiply-adds; the
    t-th trial uses seed + t and cycles through leaf sizes and imbalances."""
    best = None
    for t in range(trials):
        m, s = bisection_order(leg_sets, seed=seed + t, leaf=(6, 8, 10, 12)[t % 4],
                               imbalance=(0.05, 0.1, 0.2, 0.3)[(t // 4) % 4])
        f = order_flops(m, s)
        if best is None or f < best[0]:
            best = (f, m, s)
    return best[1], best[2]
