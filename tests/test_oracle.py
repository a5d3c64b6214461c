"""Pins of the CPU oracle to things other than itself.

Each pin is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign in the complex product, a transposed operand, a wrong axis order, a
mis-paired block) fails at least one of them:

* numpy's tensordot / matmul on random tiny complex tensors (library special
  cases of the pairwise contraction of Sec. II-A);
* a brute-force pure-Python sum over every index;
* permutation invariance of the result;
* blocked == unblocked for every block grid, including one pair (B_k = 1) and
  all pairs (Sec. II-C);
* network contraction == state-vector simulation (Sec. II-A) on small random
  grid circuits, and the closed forms GHZ = (|0..0> + |1..1>)/sqrt 2,
  H^n|0> = 2^(-n/2) everywhere, |<x|sqrt-layer|0>|^2 = 2^-n, U U^dag = I,
  fSim|00> = |00>, and sum_x |<x|C|0>|^2 = 1;
* the memory equations (Eq. 1, Eq. 2) against values in tests/golden/.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W

RNG = np.random.default_rng(1234)


def crand(shape, rng=RNG):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# ---------------------------------------------------------------------------
# pairwise tensordot
# ---------------------------------------------------------------------------
CASES = [
    # shapes a, b, axes_a, axes_b
    ((3, 4), (4, 5), [1], [0]),                 # matrix product
    ((2, 3, 4), (4, 3, 5), [1, 2], [1, 0]),     # pairs out of order
    ((2, 3), (4, 5), [], []),                    # outer product
    ((2, 3, 4), (2, 3, 4), [0, 1, 2], [0, 1, 2]),  # full contraction -> scalar
    ((5,), (5,), [0], [0]),                      # dot
    ((2, 2, 2, 2, 2), (2, 2, 2, 2), [4, 0, 2], [1, 3, 0]),
    ((1, 3, 1), (3, 1, 2), [1, 2], [0, 1]),      # extent-1 axes
    ((), (3,), [], []),                          # rank-0 operand (scalar times tensor)
    ((2, 5), (), [], []),
    ((), (), [], []),
]


@pytest.mark.parametrize("sa,sb,ax_a,ax_b", CASES)
def test_tensordot_matches_numpy(sa, sb, ax_a, ax_b):
    a, b = crand(sa), crand(sb)
    got = oracle.tensordot(a, b, ax_a, ax_b)
    ref = np.tensordot(a, b, axes=(ax_a, ax_b))
    assert got.shape == ref.shape
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-13)


def test_matrix_product_not_transposed():
    a, b = crand((3, 7)), crand((7, 2))
    np.testing.assert_allclose(oracle.tensordot(a, b, [1], [0]), a @ b, rtol=1e-13, atol=1e-13)
    # the complex product: (i)(i) = -1 must come out with the right sign
    one_i = np.array([[1j]])
    assert oracle.tensordot(one_i, one_i, [1], [0])[0, 0] == -1.0
    assert oracle.tensordot(np.array([[2 + 3j]]), np.array([[5 - 7j]]), [1], [0])[0, 0] == (2 + 3j) * (5 - 7j)


def test_brute_force_sum():
    sa, sb = (2, 3, 2, 2), (2, 2, 3)
    ax_a, ax_b = [3, 1], [0, 2]
    a, b = crand(sa), crand(sb)
    got = oracle.tensordot(a, b, ax_a, ax_b)
    ref = np.zeros((2, 2, 2), dtype=complex)
    for i0, i2, j1 in itertools.product(range(2), range(2), range(2)):
        s = 0j
        for k0 in range(2):      # A axis 3 <-> B axis 0
            for k1 in range(3):  # A axis 1 <-> B axis 2
                s += a[i0, k1, i2, k0] * b[k0, j1, k1]
        ref[i0, i2, j1] = s
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-13)


def test_permutation_invariance():
    sa, sb = (2, 3, 4, 5), (5, 3, 6)
    a, b = crand(sa), crand(sb)
    ref = oracle.tensordot(a, b, [1, 3], [1, 0])        # -> (2, 4, 6)
    perm = [2, 1, 3, 0]  # storage order (a2, a1, a3, a0): free axes come out as (4, 2)
    ap = np.ascontiguousarray(np.transpose(a, perm))
    inv = {p: i for i, p in enumerate(perm)}
    got = oracle.tensordot(ap, b, [inv[1], inv[3]], [1, 0])  # free order now (4, 2)
    np.testing.assert_allclose(np.transpose(got, [1, 0, 2]), ref, rtol=1e-13, atol=1e-13)


def test_invalid_args_raise():
    a, b = crand((2, 3)), crand((4, 5))
    with pytest.raises(ValueError):
        oracle.tensordot(a, b, [1], [0])       # extent mismatch
    with pytest.raises(ValueError):
        oracle.tensordot(a, crand((3, 3)), [1, 1], [0, 1])  # repeated axis


def test_single_thread_equals_multithread():
    a, b = crand((8, 16, 4)), crand((16, 4, 8))
    c1 = oracle.tensordot(a, b, [1, 2], [0, 1], nthreads=1)
    c8 = oracle.tensordot(a, b, [1, 2], [0, 1], nthreads=8)
    assert np.array_equal(c1, c8)  # same summation order per entry


# ---------------------------------------------------------------------------
# blocked == unblocked (Sec. II-C)
# ---------------------------------------------------------------------------
def _all_blockings(shape):
    choices = [[d for d in range(1, s + 1) if s % d == 0] for s in shape]
    return list(itertools.product(*choices))


def test_blocked_equals_unblocked_exhaustive_small():
    sa, sb = (2, 4, 2), (4, 2, 3)
    ax_a, ax_b = [1, 2], [0, 1]
    a, b = crand(sa), crand(sb)
    ref = oracle.tensordot(a, b, ax_a, ax_b)
    n = 0
    for ba in _all_blockings(sa):
        for bb in _all_blockings(sb):
            if ba[1] != bb[0] or ba[2] != bb[1]:
                continue
            got = oracle.block_tensordot(a, ba, b, bb, ax_a, ax_b)
            np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-13)
            n += 1
    assert n > 20


def test_blocked_single_config_all_pair_counts():
    for gc in (0, 2, 6):   # B_k = 1, 4, 64
        prob = W.tensordot_single_config(grid_free=2, grid_contracted=gc)
        ref = oracle.tensordot(prob["a"], prob["b"], prob["axes_a"], prob["axes_b"])
        got = oracle.block_tensordot(prob["a"], prob["block_a"], prob["b"], prob["block_b"],
                                     prob["axes_a"], prob["axes_b"])
        assert ref.shape == (2,) * 16
        assert oracle.rel_frobenius(got, ref) < 1e-14


def test_blocked_rejects_mismatched_blocks():
    a, b = crand((4, 4)), crand((4, 4))
    with pytest.raises(ValueError):
        oracle.block_tensordot(a, (2, 2), b, (4, 2), [1], [0])
    with pytest.raises(ValueError):
        oracle.block_tensordot(a, (3, 4), b, (4, 4), [1], [0])  # 3 does not divide 4


# ---------------------------------------------------------------------------
# circuits: network contraction vs state vector vs closed forms (Sec. II-A)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,depth,seed", [(4, 4, 0), (6, 8, 1), (9, 12, 2), (12, 6, 3)])
def test_network_equals_statevector(n, depth, seed):
    circ = W.random_circuit(n, depth, seed)
    net = W.circuit_network(circ)
    amp_net = oracle.contract(net, oracle.greedy_path(net))
    amp_sv = oracle.amplitude_sv(circ)
    assert np.ndim(amp_net) == 0
    assert abs(complex(amp_net) - amp_sv) <= 1e-12 * max(abs(amp_sv), 2.0 ** (-n / 2))


def test_sliced_sum_equals_unsliced():
    """Sec. II-B: projecting bonds onto each basis state and summing over all
    projections gives the unsliced result (FP64, to 1e-12), for any choice of
    bonds, including a bond next to an output projector."""
    circ = W.random_circuit(10, 8, 12)
    net = W.circuit_network(circ)
    path = oracle.greedy_path(net)
    ref = oracle.amplitude_sv(circ)
    counts = {}
    for l in net.labels:
        for x in l:
            counts[x] = counts.get(x, 0) + 1
    bonds = sorted(x for x, c in counts.items() if c == 2)
    for cut in (bonds[:1], bonds[100:104], bonds[-3:]):
        got = complex(oracle.sliced_contract(net, path, cut))
        assert abs(got - ref) <= 1e-12 * max(abs(ref), 2.0 ** -5)
    # one projection alone is not the amplitude (the slices really are partial sums)
    one = W.Network(tensors=list(net.tensors), labels=list(net.labels), out_labels=[])
    part = complex(oracle.sliced_contract(one, path, []))
    assert abs(part - ref) <= 1e-12


def test_two_paths_agree():
    circ = W.random_circuit(8, 8, 5)
    net = W.circuit_network(circ)
    a1 = complex(oracle.contract(net, oracle.greedy_path(net)))
    a2 = complex(oracle.contract(net, oracle.circuit_order_path(net)))
    assert abs(a1 - a2) <= 1e-13


def test_ghz_closed_form():
    n = 7
    circ = W.ghz_circuit(n)
    psi = oracle.statevector(circ)
    ref = np.zeros(1 << n, dtype=complex)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    np.testing.assert_allclose(psi, ref, atol=1e-15)
    for bits, want in (([0] * n, 1 / math.sqrt(2)), ([1] * n, 1 / math.sqrt(2)),
                       ([1] + [0] * (n - 1), 0.0)):
        net = W.circuit_network(circ, bitstring=bits)
        amp = complex(oracle.contract(net, oracle.greedy_path(net)))
        assert abs(amp - want) < 1e-15


def test_hadamard_closed_form():
    n = 6
    circ = W.hadamard_circuit(n)
    net = W.circuit_network(circ, open_output=True)
    psi = oracle.contract(net, oracle.greedy_path(net))
    np.testing.assert_allclose(psi.ravel(), np.full(1 << n, 2.0 ** (-n / 2)), atol=1e-15)


def test_sqrt_gate_layer_uniform():
    n = 5
    circ = W.random_circuit(n, 1, 9, rows=1, cols=5)
    circ.gates = [g for g in circ.gates if len(g[1]) == 1]  # the 1q layer only
    psi = oracle.statevector(circ)
    np.testing.assert_allclose(np.abs(psi) ** 2, np.full(1 << n, 2.0 ** -n), atol=1e-15)


def test_gate_matrices():
    for g in (W.SQRT_X, W.SQRT_Y, W.SQRT_W, W.FSIM):
        np.testing.assert_allclose(g @ g.conj().T, np.eye(len(g)), atol=1e-15)
    # Pauli matrices written out here, independently of the generator: each
    # gate is a square root of its rotation axis up to the phase -i
    X = np.array([[0, 1], [1, 0]])
    Y = np.array([[0, -1j], [1j, 0]])
    Wm = np.array([[0, (1 - 1j) / np.sqrt(2)], [(1 + 1j) / np.sqrt(2), 0]])   # (X + Y) / sqrt 2
    np.testing.assert_allclose(Wm @ Wm, np.eye(2), atol=1e-15)
    np.testing.assert_allclose(W.SQRT_X @ W.SQRT_X, -1j * X, atol=1e-15)
    np.testing.assert_allclose(W.SQRT_Y @ W.SQRT_Y, -1j * Y, atol=1e-15)
    np.testing.assert_allclose(W.SQRT_W @ W.SQRT_W, -1j * Wm, atol=1e-15)
    # fSim(pi/2, pi/6): |01> <-> -i|10>, phase e^(-i pi/6) on |11>
    ref = np.zeros((4, 4), dtype=complex)
    ref[0, 0] = 1
    ref[1, 2] = ref[2, 1] = -1j
    ref[3, 3] = np.exp(-1j * np.pi / 6)
    np.testing.assert_allclose(W.FSIM, ref, atol=1e-15)


def test_u_udagger_identity():
    circ = W.random_circuit(6, 6, 11)
    inv = W.Circuit(n=6)
    inv.gates = list(circ.gates)
    for name, qs, mat in reversed(circ.gates):
        m = np.asarray(mat).reshape(2 ** len(qs), 2 ** len(qs)).conj().T
        inv.gates.append((name + "_dag", qs, m.reshape((2,) * (2 * len(qs)))))
    net = W.circuit_network(inv, bitstring=[0] * 6)
    amp = complex(oracle.contract(net, oracle.greedy_path(net)))
    assert abs(amp - 1.0) < 1e-13


def test_fsim_on_00():
    circ = W.Circuit(n=2, gates=[("fsim", (0, 1), W.FSIM.reshape(2, 2, 2, 2))])
    psi = oracle.statevector(circ)
    np.testing.assert_allclose(psi, [1, 0, 0, 0], atol=1e-15)


def test_open_network_norm_and_statevector():
    circ = W.random_circuit(10, 8, 21)
    net = W.circuit_network(circ, open_output=True)
    psi = oracle.contract(net, oracle.greedy_path(net)).ravel()
    assert abs(np.sum(np.abs(psi) ** 2) - 1.0) < 1e-12
    np.testing.assert_allclose(psi, oracle.statevector(circ), atol=1e-13)


def test_circuit_structure():
    circ = W.rqc20_config()
    assert circ.n == 20 and circ.rows == 4 and circ.cols == 5
    n1 = sum(1 for g in circ.gates if len(g[1]) == 1)
    n2 = sum(1 for g in circ.gates if len(g[1]) == 2)
    assert n1 == 20 * 12
    # couplers per layer on a 4x5 grid: A 8, B 8, C 10, D 5; "ABCDCDAB" over 12 cycles
    assert n2 == 8 + 8 + 10 + 5 + 10 + 5 + 8 + 8 + 8 + 8 + 10 + 5
    prev = {}
    for name, qs, _ in circ.gates:
        if len(qs) == 1:
            assert prev.get(qs[0]) != name
            prev[qs[0]] = name


# ---------------------------------------------------------------------------
# memory equations (Sec. IV-A)
# ---------------------------------------------------------------------------
def test_memory_equations_golden():
    path = os.path.join(os.path.dirname(__file__), "golden", "memory_equations.txt")
    rows = [list(map(int, l.split())) for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 5
    for bk, mb, nb, kb, e1, e2, b1, b2 in rows:
        assert oracle.mem_sequential(bk, mb, nb, kb) == e1
        assert oracle.mem_pair(mb, nb, kb) == e2
        assert e1 * 8 == b1 and e2 * 8 == b2
    # Eq. 1 with one pair is Eq. 2
    assert oracle.mem_sequential(1, 7, 5, 3) == oracle.mem_pair(7, 5, 3)
