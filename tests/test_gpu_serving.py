"""The continuous-batching amplitude server: every query's amplitudes match
the oracle's state vector, and each query gives the same result alone and in
a mix of concurrent queries (within the FP32 tolerance, 1e-5)."""
import numpy as np
import pytest

import oracle
import paper_2201_06620_b300 as R
import workloads as W
from paper_2201_06620_b300.serving import AmplitudeServer, Query

pytestmark = pytest.mark.gpu


def _queries(circs, rng, count):
    qs = []
    for _ in range(count):
        ci = int(rng.integers(len(circs)))
        n = circs[ci].n
        k = int(rng.integers(0, 5))
        prefix = tuple(int(b) for b in rng.integers(0, 2, n - k))
        m = int(rng.integers(1, 2 ** k + 1))
        suffixes = sorted(int(x) for x in rng.choice(2 ** k, size=m, replace=False))
        qs.append(Query(circuit=ci, prefix=prefix, k=k, suffixes=suffixes))
    return qs


def _copy(q):
    return Query(circuit=q.circuit, prefix=q.prefix, k=q.k, suffixes=list(q.suffixes))


def test_server_alone_vs_mix_and_oracle():
    rng = np.random.default_rng(11)
    circs = [W.random_circuit(int(rng.integers(9, 14)), int(rng.integers(4, 9)), 700 + i) for i in range(5)]
    psi = [oracle.statevector(c) for c in circs]
    queries = _queries(circs, rng, 24)
    # alone: one query in the server at a time
    alone_srv = AmplitudeServer(circs, slots=1)
    alone = []
    for q in queries:
        qq = _copy(q)
        alone_srv.submit(qq)
        alone_srv.drain()
        alone.append(qq.result)
    # mix: everything submitted at once over 4 slots
    mix_srv = AmplitudeServer(circs, slots=4)
    mixed = [_copy(q) for q in queries]
    for q in mixed:
        mix_srv.submit(q)
    mix_srv.drain()
    assert len(mix_srv.finished) == len(queries)
    for q, a, m in zip(queries, alone, mixed):
        n = circs[q.circuit].n
        base = 0
        for b in q.prefix:
            base = (base << 1) | b
        ref = np.array([psi[q.circuit][(base << q.k) | s] for s in q.suffixes])
        scale = max(np.abs(ref).max(), 2.0 ** (-n / 2))
        assert np.abs(a - ref).max() / scale <= 1e-5
        assert np.abs(m.result - a).max() / scale <= 1e-5


def test_admission_by_footprint():
    """With a budget below one query's footprint the server still makes
    progress one query at a time; with a generous budget several run at once."""
    rng = np.random.default_rng(3)
    circs = [W.random_circuit(12, 6, 900 + i) for i in range(3)]
    qs = _queries(circs, rng, 8)
    tight = AmplitudeServer(circs, slots=4, memory_budget=1.0)
    for q in qs:
        tight.submit(_copy(q))
    tight.step()
    assert len(tight.running) == 1
    tight.drain()
    assert len(tight.finished) == 8
    loose = AmplitudeServer(circs, slots=4, memory_budget=1e12)
    for q in qs:
        loose.submit(_copy(q))
    loose.step()
    assert len(loose.running) == 4
    loose.drain()


def _tc_steps(circ, k, cid):
    """Steps of the served (circuit, k) path (the server's path search, seeded
    with the circuit's index) that are large enough for the
    tensor-core kernels (max(M, N) >= 128, min(M, N) >= 64, K >= 32)."""
    import math
    labels = [(q,) for q in range(circ.n)]
    ext = [(2,)] * circ.n
    wire, nl = list(range(circ.n)), circ.n
    for _, qs, mat in circ.gates:
        outs = list(range(nl, nl + len(qs)))
        nl += len(qs)
        labels.append(tuple(outs + [wire[q] for q in qs]))
        ext.append(np.asarray(mat).shape)
        for q, o in zip(qs, outs):
            wire[q] = o
    closed = circ.n - k
    labels += [(wire[q],) for q in range(closed)]
    ext += [(2,)] * closed
    out = [wire[q] for q in range(closed, circ.n)]
    path, _ = R.path_search(labels, ext, out, ntrials=16, seed=cid)
    e = {x: v for l, s in zip(labels, ext) for x, v in zip(l, s)}
    live = {i: list(l) for i, l in enumerate(labels)}
    nid, count = len(labels), 0
    for a, b in path:
        la, lb = live.pop(a), live.pop(b)
        sh = set(la) & set(lb)
        M = math.prod(e[x] for x in la if x not in sh)
        N = math.prod(e[x] for x in lb if x not in sh)
        K = math.prod(e[x] for x in sh)
        count += max(M, N) >= 128 and min(M, N) >= 64 and K >= 32
        live[nid] = [x for x in la if x not in sh] + [x for x in lb if x not in sh]
        nid += 1
    return count


def test_server_tf32x3_vs_oracle():
    """The served 3xTF32 form (the benchmark's serving default) against the
    state vector at the FP32 bar, on circuits whose k = 10 queries contain
    tensor-core-sized steps; alone and in a mix of concurrent queries."""
    circs = [W.random_circuit(18, 10, 700), W.random_circuit(20, 8, 700), W.random_circuit(16, 8, 701)]
    psi = [oracle.statevector(c) for c in circs]
    assert _tc_steps(circs[0], 10, 0) + _tc_steps(circs[1], 10, 1) > 0
    rng = np.random.default_rng(5)
    queries = []
    for i in range(12):
        ci = i % len(circs)
        n = circs[ci].n
        k = 10 if i < 6 else int(rng.integers(0, 11))
        prefix = tuple(int(b) for b in rng.integers(0, 2, n - k))
        m = int(rng.integers(1, 2 ** k + 1))
        suffixes = sorted(int(x) for x in rng.choice(2 ** k, size=m, replace=False))
        queries.append(Query(circuit=ci, prefix=prefix, k=k, suffixes=suffixes))
    alone_srv = AmplitudeServer(circs, slots=1, precision=R.PREC_TF32X3)
    alone = []
    for q in queries:
        qq = _copy(q)
        alone_srv.submit(qq)
        alone_srv.drain()
        alone.append(qq.result)
    mix_srv = AmplitudeServer(circs, slots=3, precision=R.PREC_TF32X3)
    mixed = [_copy(q) for q in queries]
    for q in mixed:
        mix_srv.submit(q)
    mix_srv.drain()
    for q, a, m in zip(queries, alone, mixed):
        n = circs[q.circuit].n
        base = 0
        for b in q.prefix:
            base = (base << 1) | b
        ref = np.array([psi[q.circuit][(base << q.k) | s] for s in q.suffixes])
        scale = max(np.abs(ref).max(), 2.0 ** (-n / 2))
        assert np.abs(a - ref).max() / scale <= 1e-5
        assert np.abs(m.result - ref).max() / scale <= 1e-5


@pytest.mark.parametrize("spill", [True, False])
def test_budget_holds_resident_plans_across_many_circuits(spill):
    """Each slot keeps a plan per (circuit, k); with a budget that holds only
    a few of them, idle plans are spilled to pinned host memory (or freed,
    with spilling off), least recently used first, so that
    resident plans plus running outputs stay within the budget whenever more
    than one query runs; results still match the state vector, and plans
    freed and built again give the same amplitudes."""
    rng = np.random.default_rng(17)
    circs = [W.random_circuit(int(rng.integers(10, 13)), 6, 1100 + i) for i in range(6)]
    psi = [oracle.statevector(c) for c in circs]
    probe = AmplitudeServer(circs, slots=1)
    sizes = []
    for ci in range(len(circs)):
        q = Query(circuit=ci, prefix=(0,) * (circs[ci].n - 2), k=2, suffixes=[0, 3])
        probe.submit(q)
        probe.drain()
        sizes.append(probe.resident[probe._key(0, q)])
    budget = 2.5 * max(sizes)
    srv = AmplitudeServer(circs, slots=2, memory_budget=budget, spill=spill)
    queries = _queries(circs, rng, 40)
    for q in queries:
        srv.submit(q)
    while srv.waiting or srv.running:
        srv.step()
        busy = {(r[1], r[0].circuit, r[0].k) for r in srv.running}
        idle = [k for k in srv.resident if k not in busy]
        assert srv.device_bytes <= budget or len(srv.running) <= 1 or not idle, (srv.device_bytes, budget)
        if srv.running:
            srv.running[0][2].synchronize()
    srv.drain()
    assert len(srv.finished) == len(queries)
    assert srv.evictions > 0
    if spill:   # idle plans went to pinned host memory and came back for later queries
        assert srv.restores > 0 and srv.spilled_bytes >= 0
    for q in srv.finished:
        n = circs[q.circuit].n
        base = 0
        for b in q.prefix:
            base = (base << 1) | b
        ref = np.array([psi[q.circuit][(base << q.k) | s] for s in q.suffixes])
        scale = max(np.abs(ref).max(), 2.0 ** (-n / 2))
        assert np.abs(q.result - ref).max() / scale <= 1e-5
