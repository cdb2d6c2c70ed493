"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test targets a plausible mistake: a transposed gate, a swapped qubit order
in a two-qubit matrix, a wrong bit order in the amplitude index, a dropped
slice, a wrong XEB formula.  None of them compares the oracle with itself.
"""
import itertools
import math

import numpy as np
import pytest

import rqcgen
from oracle import statevector as sv
from oracle import tensornet as tn
from oracle import xeb

S2 = 1.0 / math.sqrt(2.0)


# ----------------------------------------------------------------- gate set (SI)

def test_gate_closed_forms():
    """SI gate definitions: actions on basis states, and squares that are Pauli
    matrices up to the phase -i (sqrt(X)^2 = -iX etc.)."""
    x = np.array([[0, 1], [1, 0]], dtype=complex)
    y = np.array([[0, -1j], [1j, 0]])
    w = (x + y) / math.sqrt(2.0)
    for f, p in ((rqcgen.sqrt_x, x), (rqcgen.sqrt_y, y), (rqcgen.sqrt_w, w)):
        u = f()
        np.testing.assert_allclose(u @ u.conj().T, np.eye(2), atol=1e-15)
        np.testing.assert_allclose(u @ u, -1j * p, atol=1e-15)
    np.testing.assert_allclose(rqcgen.sqrt_x() @ [1, 0], [S2, -1j * S2], atol=1e-16)
    # sqrt(Y) is not symmetric: its first column is (1, 1)/sqrt2, second (-1, 1)/sqrt2
    np.testing.assert_allclose(rqcgen.sqrt_y() @ [1, 0], [S2, S2], atol=1e-16)
    np.testing.assert_allclose(rqcgen.sqrt_y() @ [0, 1], [-S2, S2], atol=1e-16)


def test_fsim_closed_form():
    """fSim(pi/2, phi): |00> fixed, |01> -> -i|10>, |10> -> -i|01>, |11> -> e^{-i phi}|11>."""
    phi = math.pi / 6
    u = rqcgen.fsim(math.pi / 2, phi)
    e = np.eye(4)
    np.testing.assert_allclose(u @ e[0], e[0], atol=1e-15)
    np.testing.assert_allclose(u @ e[1], -1j * e[2], atol=1e-15)
    np.testing.assert_allclose(u @ e[2], -1j * e[1], atol=1e-15)
    np.testing.assert_allclose(u @ e[3], np.exp(-1j * phi) * e[3], atol=1e-15)
    # the five-parameter form with the (2,2) entry read as exp(i(D+ - D-)) cos(theta) is unitary
    v = rqcgen.fsim(0.7, 0.3, 0.2, 0.5, 0.9)
    np.testing.assert_allclose(v @ v.conj().T, np.eye(4), atol=1e-14)


# ----------------------------------------------------------------- generator (SI)

def test_pattern_invariants():
    """Every nearest-neighbour pair gets exactly one gate per block of A, B, C, D."""
    for rows, cols in ((3, 4), (5, 6), (6, 7), (6, 9)):
        allpairs = set()
        for r in range(rows):
            for c in range(cols):
                if c + 1 < cols:
                    allpairs.add(((r, c), (r, c + 1)))
                if r + 1 < rows:
                    allpairs.add(((r, c), (r + 1, c)))
        seen = []
        for letter in "ABCD":
            pairs = rqcgen.pattern_pairs(rows, cols, letter)
            qs = [q for p in pairs for q in p]
            assert len(qs) == len(set(qs)), "a pattern must be a matching"
            seen.extend(pairs)
        assert sorted(seen) == sorted(allpairs)
    assert rqcgen.cycle_patterns(8) == "ABCDCDAB"
    assert rqcgen.cycle_patterns(12) == "ABCDCDABABCD"


def test_generator_counts_and_determinism():
    c1, _, _ = rqcgen.config_circuit("c1")
    assert c1.n_qubits == 12 and c1.n_two_qubit() == 34
    assert c1.n_gates - c1.n_two_qubit() == 9 * 12
    c1b, _, _ = rqcgen.config_circuit("c1")
    assert c1.to_json() == c1b.to_json()
    c5, om5, _ = rqcgen.config_circuit("c5")
    assert c5.n_qubits == 53 and bin(om5).count("1") == 6
    # single-qubit gates never repeat on a qubit in consecutive layers
    for circ in (c1, c5):
        last = {}
        for g in range(circ.n_gates):
            q0, q1 = circ.gate_qubits[g]
            if q1 < 0:
                name = circ.gate_names[g]
                assert last.get(int(q0)) != name
                last[int(q0)] = name


def test_circuit_json_roundtrip():
    c, _, _ = rqcgen.config_circuit("c1")
    d = rqcgen.Circuit.from_json(c.to_json())
    assert d.n_gates == c.n_gates
    for g in range(c.n_gates):
        np.testing.assert_array_equal(d.gate_matrices[g], c.gate_matrices[g])


# ----------------------------------------------------------------- state vector

def _random_unitary(rng, dim):
    z = rng.normal(size=(dim, dim)) + 1j * rng.normal(size=(dim, dim))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def _random_circuit(n, n_gates, seed):
    """Random gates (Haar-ish 2x2 and 4x4, not symmetric) on random qubits."""
    rng = np.random.default_rng(seed)
    qs, mats = [], []
    for _ in range(n_gates):
        if n > 1 and rng.random() < 0.5:
            a, b = rng.choice(n, size=2, replace=False)
            qs.append((int(a), int(b)))
            mats.append(_random_unitary(rng, 4))
        else:
            qs.append((int(rng.integers(n)), -1))
            mats.append(_random_unitary(rng, 2))
    return rqcgen.Circuit(n, np.array(qs, dtype=np.int32), mats,
                          np.arange(len(qs), dtype=np.int32))


def _dense_gate(n, qubits, u):
    """Full 2^n x 2^n matrix of a gate, from the definition: entry (x', x) is
    u[row(x'), col(x)] when all other bits agree, with row/col = 2 b(q0) + b(q1)."""
    dim = 1 << n
    m = np.zeros((dim, dim), dtype=complex)
    for x in range(dim):
        for xp in range(dim):
            others_equal = all(((x >> q) & 1) == ((xp >> q) & 1)
                               for q in range(n) if q not in qubits)
            if not others_equal:
                continue
            if len(qubits) == 1:
                r, c = (xp >> qubits[0]) & 1, (x >> qubits[0]) & 1
            else:
                q0, q1 = qubits
                r = 2 * ((xp >> q0) & 1) + ((xp >> q1) & 1)
                c = 2 * ((x >> q0) & 1) + ((x >> q1) & 1)
            m[xp, x] = u[r, c]
    return m


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_statevector_against_dense_definition(seed):
    n = 4
    circ = _random_circuit(n, 10, seed)
    psi = np.zeros(1 << n, dtype=complex)
    psi[0] = 1.0
    for g in range(circ.n_gates):
        q0, q1 = map(int, circ.gate_qubits[g])
        qs = (q0,) if q1 < 0 else (q0, q1)
        psi = _dense_gate(n, qs, circ.gate_matrices[g]) @ psi
    np.testing.assert_allclose(sv.simulate(circ), psi, atol=1e-13)


def test_statevector_closed_forms_and_norm():
    n = 5
    # sqrt(Y) on every qubit of |0..0>: every amplitude is +2^{-n/2}
    c = rqcgen.Circuit(n, np.array([(q, -1) for q in range(n)], dtype=np.int32),
                       [rqcgen.sqrt_y()] * n, np.zeros(n, dtype=np.int32))
    np.testing.assert_allclose(sv.simulate(c), np.full(1 << n, 2 ** (-n / 2)), atol=1e-15)
    # sqrt(X) on every qubit: amplitude of x is (-i)^{popcount(x)} 2^{-n/2}
    c = rqcgen.Circuit(n, np.array([(q, -1) for q in range(n)], dtype=np.int32),
                       [rqcgen.sqrt_x()] * n, np.zeros(n, dtype=np.int32))
    want = np.array([(-1j) ** bin(x).count("1") for x in range(1 << n)]) * 2 ** (-n / 2)
    np.testing.assert_allclose(sv.simulate(c), want, atol=1e-15)
    # sqrt(X) on q0, then fSim(pi/2) on (q0, q1): (|00> - |01>... in bit order) / sqrt2
    c = rqcgen.Circuit(2, np.array([(0, -1), (0, 1)], dtype=np.int32),
                       [rqcgen.sqrt_x(), rqcgen.fsim(math.pi / 2, math.pi / 6)],
                       np.zeros(2, dtype=np.int32))
    psi = sv.simulate(c)
    # sqrt(X)|0> on q0 = (|x=0> - i|x=1>)/sqrt2 (x = b0 + 2 b1); fSim maps b0=1,b1=0 (row 2) to -i * (b0=0,b1=1)
    np.testing.assert_allclose(psi, [S2, 0, -S2, 0], atol=1e-15)
    circ, _, _ = rqcgen.config_circuit("c1")
    assert abs(np.linalg.norm(sv.simulate(circ)) - 1.0) < 1e-12


# ----------------------------------------------------------------- tensor network

def _feynman_amplitude(circ, x):
    """<x|U|0> as an explicit sum over every value of every internal wire (the
    definition of contracting the network), pure Python loops, tiny circuits."""
    n = circ.n_qubits
    t = [0] * n
    gates = []
    for g in range(circ.n_gates):
        q0, q1 = map(int, circ.gate_qubits[g])
        if q1 < 0:
            gates.append(((q0,), [(q0, t[q0] + 1)], [(q0, t[q0])], circ.gate_matrices[g]))
            t[q0] += 1
        else:
            gates.append(((q0, q1), [(q0, t[q0] + 1), (q1, t[q1] + 1)],
                          [(q0, t[q0]), (q1, t[q1])], circ.gate_matrices[g]))
            t[q0] += 1
            t[q1] += 1
    internal = [(q, k) for q in range(n) for k in range(1, t[q])]
    total = 0j
    for vals in itertools.product((0, 1), repeat=len(internal)):
        val = dict(zip(internal, vals))
        for q in range(n):
            val[(q, 0)] = 0
            val[(q, t[q])] = (x >> q) & 1
        term = 1 + 0j
        for _, outs, ins, u in gates:
            if len(outs) == 1:
                term *= u[val[outs[0]], val[ins[0]]]
            else:
                term *= u[2 * val[outs[0]] + val[outs[1]], 2 * val[ins[0]] + val[ins[1]]]
            if term == 0:
                break
        total += term
    return total


@pytest.mark.parametrize("seed", [3, 4])
def test_tensornet_against_path_sum(seed):
    circ = _random_circuit(3, 6, seed)
    for open_mask in (0b000, 0b101, 0b111):
        closed = 0b010
        got = tn.batch_amplitudes(circ, closed, open_mask)
        idx = sv.batch_indices(3, closed, open_mask)
        want = np.array([_feynman_amplitude(circ, int(x)) for x in idx])
        np.testing.assert_allclose(got, want, atol=1e-13)


@pytest.mark.parametrize("seed", [5, 6, 7])
def test_tensornet_against_statevector(seed):
    n = 9
    circ = _random_circuit(n, 40, seed)
    psi = sv.simulate(circ)
    rng = np.random.default_rng(seed)
    open_mask = int(rng.integers(1 << n))
    closed = int(rng.integers(1 << n))
    got = tn.batch_amplitudes(circ, closed, open_mask)
    want = sv.batch_amplitudes(psi, n, closed, open_mask)
    assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)


def test_tensornet_c1_against_statevector():
    circ, om, cb = rqcgen.config_circuit("c1")
    psi = sv.simulate(circ)
    got = tn.batch_amplitudes(circ, cb, om)
    want = sv.batch_amplitudes(psi, circ.n_qubits, cb, om)
    assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)


def test_slicing_identity_and_additivity():
    """Main text, section II: the sliced network is the sum of the smaller networks."""
    circ, om, cb = rqcgen.config_circuit("c1")
    net = tn.CircuitNetwork(circ, cb, om & 0xF0F)
    full = net.contract()
    rng = np.random.default_rng(0)
    internal = [(q, t) for q in range(circ.n_qubits) for t in range(1, net.wire_count[q])]
    for s_count in (1, 3, 6):
        pick = [internal[i] for i in rng.choice(len(internal), size=s_count, replace=False)]
        tot = net.contract(pick)
        assert np.linalg.norm(tot - full) <= 1e-12 * np.linalg.norm(full)
        ids = np.arange(1 << s_count)
        part_a = net.contract(pick, ids[: len(ids) // 3])
        part_b = net.contract(pick, ids[len(ids) // 3:])
        assert np.linalg.norm(part_a + part_b - full) <= 1e-12 * np.linalg.norm(full)
        one = net.contract(pick, [1])
        assert np.linalg.norm(one - full) > 1e-6 * np.linalg.norm(full)  # a slice is not the sum


def test_bisection_order_matches_greedy():
    """The oracle's two contraction orders give the same amplitudes (the order
    only changes rounding), on a 30-qubit batch."""
    circ, om, cb = rqcgen.config_circuit("c2")
    net = tn.CircuitNetwork(circ, cb, om)
    a = net.contract(method="greedy")
    b = net.contract(method="bisect", trials=4, max_log2=20)
    assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(a)


def test_contract_in_order_sums_slices_of_its_own_order():
    """Slicing the wires plan() picks and summing every slice along plan()'s
    order reproduces the unsliced amplitudes."""
    circ, _, cb = rqcgen.config_circuit("c1")
    net = tn.CircuitNetwork(circ, cb, 0b1111)
    merges, wires = net.plan([], max_log2=6, method="bisect", trials=2)
    assert len(wires) > 0
    a = net.contract_in_order(merges, wires, range(1 << len(wires)))
    b = net.contract()
    assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)


def _random_tree(rng, n_gates, n_groups):
    """A random grouping of gates (every group non-empty) and a random binary
    merge order over the groups (ids: groups first, merge j creates n_groups + j)."""
    leaf = np.concatenate([np.arange(n_groups), rng.integers(0, n_groups, size=n_gates - n_groups)])
    rng.shuffle(leaf)
    alive = list(range(n_groups))
    pairs = []
    while len(alive) > 1:
        i, j = sorted(rng.choice(len(alive), size=2, replace=False))
        pairs.append((alive[i], alive[j]))
        alive = [x for k, x in enumerate(alive) if k not in (i, j)] + [n_groups + len(pairs) - 1]
    return [int(x) for x in leaf], pairs


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_tree_order_against_statevector(seed):
    """An order given by its tree shape (random groups of gates, random merges
    of the groups, some groups not even connected) contracts the same network:
    sliced or not, the amplitudes are the state vector's."""
    n = 7
    circ = _random_circuit(n, 22, seed)
    rng = np.random.default_rng(seed)
    open_mask = int(rng.integers(1 << n)) | 1
    closed = int(rng.integers(1 << n))
    want = sv.batch_amplitudes(sv.simulate(circ), n, closed, open_mask)
    net = tn.CircuitNetwork(circ, closed, open_mask)
    leaf, pairs = _random_tree(rng, circ.n_gates, 6)
    internal = [(q, t) for q in range(n) for t in range(1, net.wire_count[q])]
    pick = [internal[i] for i in rng.choice(len(internal), size=3, replace=False)]
    for sliced, max_log2 in (([], 27), (pick, 27), (pick, 8)):
        merges, extra = net.plan_along_tree(sliced, leaf, pairs, max_log2=max_log2)
        got = net.contract_in_order(merges, sliced, range(1 << len(sliced)), extra)
        assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)
    # a partial sum over a slice range is the sum of its parts
    merges, extra = net.plan_along_tree(pick, leaf, pairs)
    a = net.contract_in_order(merges, pick, [0, 1, 2], extra)
    b = net.contract_in_order(merges, pick, [3, 4, 5, 6, 7], extra)
    assert np.linalg.norm(a + b - want) <= 1e-12 * np.linalg.norm(want)


def test_tree_order_rejects_incomplete_trees():
    """A tree that merges a node twice, leaves a group out, or names an unknown
    node is not a contraction of the network."""
    circ = _random_circuit(6, 20, 3)
    net = tn.CircuitNetwork(circ, 0, 0b111)
    rng = np.random.default_rng(3)
    leaf, pairs = _random_tree(rng, circ.n_gates, 5)
    net.tree_order(leaf, pairs)
    with pytest.raises(ValueError):
        net.tree_order(leaf, pairs[:-1])                       # two nodes left
    with pytest.raises(ValueError):
        net.tree_order(leaf, pairs[:-1] + [(pairs[-1][0], pairs[-1][0])])
    with pytest.raises(ValueError):
        net.tree_order(leaf, pairs + [(0, 1)])                 # merged twice
    bad = list(leaf)
    bad[bad.index(4)] = 9                                      # a gap in the group ids
    with pytest.raises(ValueError):
        net.tree_order(bad, pairs)


def test_oracle_subslicing_changes_nothing():
    circ, om, cb = rqcgen.config_circuit("c1")
    net = tn.CircuitNetwork(circ, cb, om)
    a = net.contract(max_log2=27)
    b = net.contract(max_log2=12)
    assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(a)


def test_batches_cover_unit_norm():
    """Sum over all batches of |a|^2 is 1 (the state is normalised)."""
    circ, _, _ = rqcgen.config_circuit("c1")
    open_mask = 0b000011110000
    total = 0.0
    for closed_hi in range(1 << 8):
        closed = (closed_hi & 0xF) | ((closed_hi >> 4) << 8)
        a = tn.batch_amplitudes(circ, closed, open_mask)
        total += float(np.sum(np.abs(a) ** 2))
    assert abs(total - 1.0) < 1e-12


# ----------------------------------------------------------------- XEB, Eq. (1)

def test_fxeb_density_is_normalised_with_mean_one_plus_f():
    x = np.linspace(0, 60, 600001)
    for f in (0.0, 0.3, 1.0):
        p = xeb.fxeb_density(x, f)
        assert abs(np.trapezoid(p, x) - 1.0) < 1e-8
        assert abs(np.trapezoid(x * p, x) - (1.0 + f)) < 1e-8
        assert abs(np.trapezoid(x * x * p, x) - xeb.fxeb_moment(2, f)) < 1e-7


def test_linear_xeb_special_cases():
    n = 10
    uniform = np.full(1 << n, 2 ** (-n / 2), dtype=complex)
    assert abs(xeb.linear_xeb(uniform, n)) < 1e-13
    # a point mass: F = 2^n - 1
    delta = np.zeros(1 << n, dtype=complex)
    delta[3] = 1.0
    assert abs(xeb.linear_xeb(delta[3:4], n) - (2 ** n - 1)) < 1e-9


def test_porter_thomas_and_ideal_xeb():
    """A deep random circuit's output is Porter-Thomas: x = N p over all
    bitstrings follows Eq. (1) with F = 0, so E[x] = 1, E[x^2] = 2, E[x^3] = 6.
    Ideal sampling then gives XEB = N sum p^2 - 1 = E[x^2] - 1 ~ 1, and
    bitstrings drawn from p give a sampled linear XEB near that value."""
    circ = rqcgen.sycamore_style(4, 4, 20, seed=11)
    n = circ.n_qubits
    psi = sv.simulate(circ)
    x = (1 << n) * np.abs(psi) ** 2
    assert abs(x.mean() - 1.0) < 1e-12
    sd2 = math.sqrt((xeb.fxeb_moment(4, 0.0) - 4.0) / x.size)   # sd of the mean of x^2
    assert abs((x * x).mean() - xeb.fxeb_moment(2, 0.0)) < 4 * sd2
    assert abs((x ** 3).mean() - xeb.fxeb_moment(3, 0.0)) < 0.25
    ideal = float((1 << n) * np.sum(np.abs(psi) ** 4) - 1.0)
    assert abs(ideal - 1.0) < 4 * sd2
    m = 20000
    picks = xeb.sample_bitstrings(np.abs(psi) ** 2, m, seed=0)
    f = xeb.linear_xeb(psi[picks], n)
    assert abs(f - ideal) < 4 * math.sqrt(6.0 / m)
    # uniformly chosen bitstrings (F = 0 sampler) give XEB ~ 0
    rng = np.random.default_rng(1)
    f0 = xeb.linear_xeb(psi[rng.integers(0, 1 << n, size=m)], n)
    assert abs(f0) < 4 * math.sqrt(1.0 / m)


# ----------------------------------------------------------------- frugal sampling (main text, section III)
def test_frugal_sampling_special_cases():
    from oracle import sampling
    n = 6
    a = np.zeros(64, dtype=np.complex128)
    a[37] = 1.0                                   # all weight on one member: N p = 64 > M
    cand = np.array([3, 37, 37, 5])
    u = np.array([0.0, 0.999999, 0.1, 0.0])
    assert sampling.frugal_sample(a, n, 10.0, cand, u) == 1     # zero-probability proposals never pass
    assert sampling.frugal_sample(a, n, 10.0, np.array([3, 5]), np.array([0.0, 0.0])) == -1
    # N p exactly M: accepted for every u < 1
    b = np.zeros(4, dtype=np.complex128)
    b[2] = 0.75 + 0.25j                           # n = 4: N p = 16 * (0.5625 + 0.0625) = 10 exactly
    assert sampling.accept_mask(b, 4, 10.0, np.array([2, 2]), np.array([0.0, np.nextafter(1.0, 0)])).all()
    assert not sampling.accept_mask(b, 4, 10.0, np.array([2]), np.array([1.0]))[0]


def test_frugal_sampling_law_and_sampled_xeb():
    """Accepted members follow min(1, N p / M) (here = p / M, no member has
    N p > M), the acceptance rate per draw is the mean of that law, and the
    linear XEB of the samples from Porter-Thomas amplitudes is 1 (ideal)."""
    from oracle import sampling
    rng = np.random.default_rng(2024)
    n, m_bound = 8, 40.0
    a = (rng.normal(size=256) + 1j * rng.normal(size=256))
    a /= np.linalg.norm(a)
    assert np.max(np.ldexp(np.abs(a) ** 2, n)) < m_bound
    law = sampling.acceptance_law(a, n, m_bound)
    rate = law.sum()
    trials, draws = 20000, 1000
    counts = np.zeros(256)
    used = 0
    samples = []
    for _ in range(trials):
        cand = rng.integers(0, 256, size=draws)
        u = rng.random(draws)
        t = sampling.frugal_sample(a, n, m_bound, cand, u)
        assert t >= 0                              # 1000 draws at rate ~1/40 fail with prob. e^-25
        used += t + 1
        counts[cand[t]] += 1
        samples.append(cand[t])
    # draws until acceptance: geometric with mean 1 / rate
    mean_draws = used / trials
    sd = math.sqrt((1 - rate) / rate ** 2 / trials)
    assert abs(mean_draws - 1 / rate) < 5 * sd
    # member frequencies against p (chi-square, 255 degrees of freedom)
    expect = trials * law / rate
    chi2 = np.sum((counts - expect) ** 2 / expect)
    assert chi2 < 255 + 6 * math.sqrt(2 * 255)
    # sampled linear XEB of an ideal sampler of Porter-Thomas amplitudes is ~1
    f = xeb.linear_xeb(a[np.array(samples)], n)
    assert abs(f - (256 * np.sum(np.abs(a) ** 4) - 1)) < 0.1


@pytest.mark.parametrize("name", ["c2", "c3"])
def test_stored_xeb_is_the_oracle_xeb_of_the_stored_amplitudes(name):
    """The stored XEB beside a workload's stored amplitudes is the oracle's
    linear XEB of exactly those amplitudes (it is what the benchmark compares
    the library's XEB with), and it obeys Eq. (1)'s range: F = N<p> - 1 > -1."""
    from tests.golden import make_golden
    circ, _, _ = rqcgen.config_circuit(name)
    amps = make_golden.read(name)
    stored = make_golden.read_xeb(name)
    assert stored == pytest.approx(xeb.linear_xeb(amps, circ.n_qubits), rel=1e-15, abs=1e-17)
    assert stored > -1.0


# ---------------------------------------------------------------- pairwise contraction / permutation
# SI Eq. (2) and the storage convention of figure S7's caption: a tensor over
# wires w_0..w_{r-1} is a flat array whose element sum_i b(w_i) 2^i holds the
# entry with wire w_i set to b(w_i).  The brute force below walks every wire
# assignment with plain integer loops (no einsum, no reshape).

def _bruteforce_pair(a, a_wires, b, b_wires, c_wires):
    wires = sorted(set(a_wires) | set(b_wires))
    out = np.zeros(2 ** len(c_wires), dtype=np.complex128)
    for assign in range(2 ** len(wires)):
        val = {w: (assign >> i) & 1 for i, w in enumerate(wires)}
        ia = sum(val[w] << i for i, w in enumerate(a_wires))
        ib = sum(val[w] << i for i, w in enumerate(b_wires))
        ic = sum(val[w] << i for i, w in enumerate(c_wires))
        out[ic] += a[ia] * b[ib]
    return out


@pytest.mark.parametrize("seed", range(6))
def test_pairwise_contraction_against_bruteforce(seed):
    from oracle import pairwise
    rng = np.random.default_rng(700 + seed)
    m, k, n = (int(x) for x in rng.integers(0, 4, size=3))
    free_a, shared, free_b = list(range(m)), list(range(10, 10 + k)), list(range(20, 20 + n))
    a_w = [int(w) for w in rng.permutation(free_a + shared)]
    b_w = [int(w) for w in rng.permutation(shared + free_b)]
    c_w = [int(w) for w in rng.permutation(free_a + free_b)]
    a = rng.normal(size=2 ** len(a_w)) + 1j * rng.normal(size=2 ** len(a_w))
    b = rng.normal(size=2 ** len(b_w)) + 1j * rng.normal(size=2 ** len(b_w))
    got = pairwise.contract_pair(a, a_w, b, b_w, c_w)
    np.testing.assert_allclose(got, _bruteforce_pair(a, a_w, b, b_w, c_w), rtol=1e-13, atol=1e-13)


def test_pairwise_contraction_is_a_column_major_matrix_product():
    """Special case: A over wires (m, k) and B over (k, n), both 2^2 x 2^2
    with the first listed wires fastest, give C = A B of the column-major
    matrices (numpy's matmul on reshape(order='F'))."""
    from oracle import pairwise
    rng = np.random.default_rng(5)
    a = rng.normal(size=16) + 1j * rng.normal(size=16)
    b = rng.normal(size=16) + 1j * rng.normal(size=16)
    got = pairwise.contract_pair(a, [0, 1, 2, 3], b, [2, 3, 4, 5], [0, 1, 4, 5])
    want = (a.reshape(4, 4, order="F") @ b.reshape(4, 4, order="F")).reshape(-1, order="F")
    np.testing.assert_allclose(got, want, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("rank", [1, 3, 5])
def test_permute_against_bruteforce(rank):
    from oracle import pairwise
    rng = np.random.default_rng(rank)
    perm = [int(p) for p in rng.permutation(rank)]
    t = rng.normal(size=2 ** rank) + 1j * rng.normal(size=2 ** rank)
    want = np.zeros_like(t)
    for i in range(2 ** rank):
        # output bit p is input bit perm[p]
        o = sum(((i >> perm[p]) & 1) << p for p in range(rank))
        want[o] = t[i]
    np.testing.assert_array_equal(pairwise.permute(t, rank, perm), want)
