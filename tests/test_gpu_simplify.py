"""GPU parity of network simplification (rosnet_simplify: rank-1 and rank-2
tensors absorbed into neighbours by device tensordots before path search)
against the complex128 state-vector oracle.

Cases: full amplitude networks of random grid circuits (every |0>, one-qubit
gate and projector absorbed), the same with the output projectors kept and
rebound per bitstring (the serving pattern), the GHZ closed form, open
output wires (never summed), rank-1-only absorption, and 2-D-grid circuits
whose simplified networks are contracted along searched paths.
"""
import numpy as np
import pytest

import oracle
import paper_2201_06620_b300 as R
import workloads as W

pytestmark = pytest.mark.gpu


def _leaves(net):
    return [R.btensor(np.asarray(t, dtype=np.complex64)) for t in net.tensors]


def _rel(got, ref, n):
    return abs(got - ref) / max(abs(ref), 2.0 ** (-n / 2))


@pytest.mark.parametrize("n,depth,seed", [(8, 6, 1), (12, 8, 2), (16, 10, 3)])
def test_full_simplification_matches_state_vector(n, depth, seed):
    circ = W.random_circuit(n, depth, seed)
    net = W.circuit_network(circ)
    ts = _leaves(net)
    st, sl, origin = R.simplify(ts, net.labels, net.out_labels)
    n2q = sum(1 for _, qs, _ in circ.gates if len(qs) == 2)
    assert len(st) <= max(n2q, 1) + n      # about one tensor per two-qubit gate
    assert len(st) < len(ts) // 2
    assert all(len(l) <= 4 for l in sl)
    assert origin == sorted(origin)
    path = R.path_greedy(st, sl, [])
    got = complex(R.contract(st, sl, [], path).download())
    assert _rel(got, oracle.amplitude_sv(circ), n) <= 1e-5


def test_kept_projectors_rebound_per_bitstring():
    """Projectors kept: the circuit part is simplified once and every
    bitstring only swaps the projector tensors of the simplified network."""
    circ = W.random_circuit(12, 8, 7)
    net = W.circuit_network(circ)
    ts = _leaves(net)
    n = circ.n
    first_proj = len(ts) - n
    st, sl, origin = R.simplify(ts, net.labels, net.out_labels, keep=range(first_proj, len(ts)))
    slot = {o: i for i, o in enumerate(origin)}
    assert all(first_proj + q in slot for q in range(n))          # projectors survive in place
    assert all(st[slot[first_proj + q]] is ts[first_proj + q] for q in range(n))
    proj = [R.btensor(np.eye(2, dtype=np.complex64)[b]) for b in (0, 1)]
    nw = R.Network(st, sl, [])
    path = nw.greedy_path()
    psi = oracle.statevector(circ)
    rng = np.random.default_rng(0)
    for _ in range(4):
        bits = rng.integers(0, 2, n)
        for q in range(n):
            nw.set_tensor(slot[first_proj + q], proj[int(bits[q])])
        got = complex(R.contract(nw, path=path).download())
        assert _rel(got, psi[oracle.bitstring_index(bits)], n) <= 1e-5


def test_ghz_closed_form():
    n = 10
    circ = W.ghz_circuit(n)
    for bits, want in (([0] * n, 2 ** -0.5), ([1] * n, 2 ** -0.5), ([0] * (n - 1) + [1], 0.0)):
        net = W.circuit_network(circ, bitstring=bits)
        st, sl, _ = R.simplify(_leaves(net), net.labels, net.out_labels)
        got = complex(R.contract(st, sl, [], R.path_greedy(st, sl, [])).download())
        assert abs(got - want) <= 1e-6


def test_open_outputs_are_never_summed():
    circ = W.random_circuit(8, 6, 5)
    net = W.circuit_network(circ, open_output=True)
    st, sl, _ = R.simplify(_leaves(net), net.labels, net.out_labels)
    assert sorted(x for l in sl for x in l if x in set(net.out_labels)) == sorted(net.out_labels)
    got = R.contract(st, sl, net.out_labels, R.path_greedy(st, sl, net.out_labels)).download()
    ref = oracle.statevector(circ).reshape((2,) * circ.n)
    assert oracle.rel_frobenius(got, ref) <= 1e-5


def test_rank1_only():
    circ = W.random_circuit(10, 6, 9)
    net = W.circuit_network(circ)
    ts = _leaves(net)
    st, sl, _ = R.simplify(ts, net.labels, net.out_labels, max_rank=1)
    assert len(st) < len(ts)
    got = complex(R.contract(st, sl, [], R.path_greedy(st, sl, [])).download())
    assert _rel(got, oracle.amplitude_sv(circ), circ.n) <= 1e-5


def test_searched_paths_on_simplified_grid_circuits():
    for seed in (11, 12):
        circ = W.random_circuit(16, 12, seed)
        net = W.circuit_network(circ)
        st, sl, _ = R.simplify(_leaves(net), net.labels, net.out_labels)
        path, _ = R.path_search(sl, [t.shape for t in st], [], ntrials=16, seed=seed)
        got = complex(R.contract(st, sl, [], path).download())
        assert _rel(got, oracle.amplitude_sv(circ), circ.n) <= 1e-5


def test_cheaper_network_never_costs_more_than_the_raw_one():
    for seed in (21, 22, 23):
        circ = W.random_circuit(14, 10, seed)
        net = W.circuit_network(circ)
        ts = _leaves(net)
        _, raw_flops = R.path_search(net.labels, [t.shape for t in ts], [], ntrials=8, seed=seed)
        st, sl, path, flops = R.cheaper_network(ts, net.labels, [], ntrials=8, seed=seed)
        assert flops <= raw_flops
        got = complex(R.contract(st, sl, [], path).download())
        assert _rel(got, oracle.amplitude_sv(circ), circ.n) <= 1e-5
