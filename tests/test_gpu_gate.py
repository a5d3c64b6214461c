"""GPU parity of the low-arithmetic-intensity kernel (gett_gate_kernel):
one- and two-qubit gates and projections applied along axes of a large
complex64 tensor, against the complex128 CPU oracle (relative Frobenius
error <= 1e-5).

Cases run as plain tensordots and as the second step of a planned network
(the large operand an intermediate of the plan), where the heavy launch's
kernel family is recorded.  The gate's output axis goes
last (tensordot(T, G)) or first (tensordot(G, T)), so both vector store
paths of C are taken; a gate on the innermost axis leaves no unit-stride run
and takes the thread-per-output kernel.
"""
import numpy as np
import pytest

import oracle
import paper_2201_06620_b300 as R
import workloads as W

pytestmark = pytest.mark.gpu


def gate_kind(k, n):
    lg = {1: 0, 2: 1, 4: 2}
    return 16 + 3 * lg[k] + lg[n]


def _c64(shape, seed):
    return W.complex_normal(shape, seed).astype(np.complex64)


@pytest.mark.parametrize("rank,axes,gate_first", [(16, (5,), False), (16, (5,), True), (16, (0,), False),
                                                  (18, (3, 11), False), (18, (7, 8), True), (16, (15,), False)])
def test_gate_tensordot(rank, axes, gate_first):
    t = _c64((2,) * rank, 81)
    q = len(axes)
    g = _c64((2,) * (2 * q), 82)                 # G[out..., in...]
    g_in = list(range(q, 2 * q))
    T, G = R.btensor(t), R.btensor(g)
    if gate_first:
        got = R.tensordot(G, T, g_in, list(axes)).download()
        ref = oracle.tensordot(g, t, g_in, list(axes))
    else:
        got = R.tensordot(T, G, list(axes), g_in).download()
        ref = oracle.tensordot(t, g, list(axes), g_in)
    assert oracle.rel_frobenius(got, ref) <= 1e-5


@pytest.mark.parametrize("rank,axes,gate_first,vector", [(16, (5,), False, True), (16, (5,), True, True),
                                                         (18, (3, 11), False, True), (18, (7, 8), True, True),
                                                         (16, (16,), False, False)])
def test_gate_on_intermediate(rank, axes, gate_first, vector):
    """Network (T, v, G): the outer product of T with a 2-vector v (the
    intermediate, twice T's size, v's axis last), then G on `axes` of that
    intermediate: the second step has twice the flops, so it is the timed
    heavy launch.  It takes the gate kernel when the intermediate's innermost
    run stays unit-stride (a gate on its last axis breaks it)."""
    t = _c64((2,) * rank, 91)
    v = _c64((2,), 92)
    q = len(axes)
    g = _c64((2,) * (2 * q), 93)
    inter = list(range(rank)) + [300]                 # labels of the intermediate, in order
    gl = [inter[a] for a in axes]
    gate_out = [200 + i for i in range(q)]
    rest = [x for x in inter if x not in gl]
    out = gate_out + rest if gate_first else rest + gate_out
    labels = [list(range(rank)), [300], gate_out + gl]
    T, V, G = R.btensor(t), R.btensor(v), R.btensor(g)
    R.timing_drain()
    got = R.contract([T, V, G], labels, out, [(0, 1), (2, 3)] if gate_first else [(0, 1), (3, 2)],
                     flags=R.OPT_GRAPH | R.OPT_TIMING).download()
    recs = R.timing_drain()
    if vector:
        assert recs and recs[-1][3] == gate_kind(2 ** q, 2 ** q), recs[-1:]
    tv = oracle.tensordot(t, v, [], [])
    ref = (oracle.tensordot(g, tv, list(range(q, 2 * q)), list(axes)) if gate_first
           else oracle.tensordot(tv, g, list(axes), list(range(q, 2 * q))))
    assert oracle.rel_frobenius(got, ref) <= 1e-5


def test_projection_and_other_extents():
    """A rank-1 projection (K = 2, N = 1) on an inner axis, and a 2 x 2 gate
    on a tensor with extents 3, 2, 1000, 8 (runs of 8000, not powers of two
    in the middle; 1000 * 8 / 8 rows per thread leave a ragged last CTA)."""
    t = _c64((24, 3, 2, 1000), 95)
    v = _c64((2,), 96)
    got = R.tensordot(R.btensor(t), R.btensor(v), [2], [0]).download()
    assert oracle.rel_frobenius(got, oracle.tensordot(t, v, [2], [0])) <= 1e-5
    t2 = _c64((3, 2, 1000, 8), 97)
    g = _c64((2, 2), 98)
    got = R.tensordot(R.btensor(g), R.btensor(t2), [1], [1]).download()
    assert oracle.rel_frobenius(got, oracle.tensordot(g, t2, [1], [1])) <= 1e-5
    got = R.tensordot(R.btensor(t2), R.btensor(g), [1], [1]).download()
    assert oracle.rel_frobenius(got, oracle.tensordot(t2, g, [1], [1])) <= 1e-5
