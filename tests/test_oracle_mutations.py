"""Planted mistakes in the oracle (on the CPU): each must make a pin fail.

This shows the pins in test_oracle_pins.py are sensitive to the mistakes they
are meant to catch, rather than passing for any implementation.
"""
import numpy as np
import pytest

import rqcgen
from oracle import statevector as sv
from oracle import tensornet as tn

from tests.test_oracle_pins import _feynman_amplitude, _random_circuit


def _mutated_network(monkeypatch, mutate):
    orig_init = tn.CircuitNetwork.__init__

    def init(self, circuit, closed_bits, open_mask):
        orig_init(self, circuit, closed_bits, open_mask)
        mutate(self)

    monkeypatch.setattr(tn.CircuitNetwork, "__init__", init)


def _tn_vs_pathsum(circ, open_mask, closed):
    got = tn.batch_amplitudes(circ, closed, open_mask)
    idx = sv.batch_indices(circ.n_qubits, closed, open_mask)
    want = np.array([_feynman_amplitude(circ, int(x)) for x in idx])
    return float(np.max(np.abs(got - want)))


def test_planted_transposed_single_qubit_gates_are_caught(monkeypatch):
    circ = _random_circuit(3, 6, 3)

    def mutate(net):
        net.data = [d.T.copy() if d.ndim == 2 else d for d in net.data]

    assert _tn_vs_pathsum(circ, 0b111, 0) < 1e-12
    _mutated_network(monkeypatch, mutate)
    assert _tn_vs_pathsum(circ, 0b111, 0) > 1e-3


def test_planted_swapped_two_qubit_order_is_caught(monkeypatch):
    circ = _random_circuit(3, 6, 4)

    def mutate(net):
        net.data = [d.transpose(1, 0, 3, 2).copy() if d.ndim == 4 else d for d in net.data]

    _mutated_network(monkeypatch, mutate)
    assert _tn_vs_pathsum(circ, 0b111, 0) > 1e-3


def test_planted_reversed_amplitude_bit_order_is_caught(monkeypatch):
    circ, om, cb = rqcgen.config_circuit("c1")
    psi = sv.simulate(circ)
    want = sv.batch_amplitudes(psi, circ.n_qubits, cb, om)

    def mutate(net):
        net.open_legs = list(reversed(net.open_legs))

    _mutated_network(monkeypatch, mutate)
    got = tn.batch_amplitudes(circ, cb, om)
    assert np.linalg.norm(got - want) > 1e-3 * np.linalg.norm(want)


def test_planted_dropped_slice_is_caught():
    circ, om, cb = rqcgen.config_circuit("c1")
    net = tn.CircuitNetwork(circ, cb, om)
    full = net.contract()
    sliced = [(0, 3), (5, 4), (9, 2)]
    partial = net.contract(sliced, range(1, 8))        # slice 0 left out
    assert np.linalg.norm(partial - full) > 1e-6 * np.linalg.norm(full)


@pytest.mark.parametrize("mistake", ["drop_N", "greater_equal_u_side", "ignore_imaginary"])
def test_planted_frugal_sampling_mistakes_are_caught(monkeypatch, mistake):
    """Accepting with p instead of N p, comparing the wrong way round, or
    dropping Im a from p each breaks the frugal-sampling law pin."""
    from oracle import sampling
    from tests.test_oracle_pins import test_frugal_sampling_law_and_sampled_xeb as pin
    orig = sampling.accept_mask

    def mutated(amplitudes, n_qubits, m_bound, candidates, uniforms):
        a = np.asarray(amplitudes, dtype=np.complex128).reshape(-1)
        c, u = np.asarray(candidates), np.asarray(uniforms, dtype=np.float64)
        if mistake == "drop_N":
            return orig(a, 0, m_bound / 2 ** 6, c, u)   # N = 64 instead of 2^n
        if mistake == "greater_equal_u_side":
            return u * m_bound > np.ldexp(np.abs(a[c]) ** 2, n_qubits)
        return u * m_bound < np.ldexp(a.real[c] ** 2, n_qubits)

    pin()
    monkeypatch.setattr(sampling, "accept_mask", mutated)
    with pytest.raises(AssertionError):
        pin()


def test_planted_pairwise_mistakes_are_caught(monkeypatch):
    """A conjugated operand and a reversed storage order (wire 0 slowest) in the
    pairwise oracle each fail its brute-force pin."""
    from oracle import pairwise
    from tests.test_oracle_pins import _bruteforce_pair
    rng = np.random.default_rng(11)
    a_w, b_w, c_w = [0, 10, 1], [10, 20], [1, 20, 0]
    a = rng.normal(size=8) + 1j * rng.normal(size=8)
    b = rng.normal(size=4) + 1j * rng.normal(size=4)
    want = _bruteforce_pair(a, a_w, b, b_w, c_w)
    assert np.max(np.abs(pairwise.contract_pair(a, a_w, b, b_w, c_w) - want)) < 1e-13
    orig = pairwise.contract_pair

    monkeypatch.setattr(pairwise, "contract_pair",
                        lambda a_, aw, b_, bw, cw: orig(np.conj(a_), aw, b_, bw, cw))
    assert np.max(np.abs(pairwise.contract_pair(a, a_w, b, b_w, c_w) - want)) > 1e-3
    monkeypatch.setattr(pairwise, "to_axes",
                        lambda flat, rank: np.asarray(flat).reshape((2,) * rank) if rank else np.asarray(flat).reshape(()))
    monkeypatch.setattr(pairwise, "contract_pair", orig)
    assert np.max(np.abs(pairwise.contract_pair(a, a_w, b, b_w, c_w) - want)) > 1e-3
