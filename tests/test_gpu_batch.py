"""Batched and sliced contraction on the GPU (grouped launches over several
networks, steps shared between slices, FP64 sum over slices) against the
oracle's state vector and its own sliced contraction (Sec. II-B)."""
import numpy as np
import pytest

import oracle
import paper_2201_06620_b300 as R
import workloads as W

pytestmark = pytest.mark.gpu

NPT = {R.C64: np.complex64, R.C128: np.complex128}


def _device_network(net, dtype):
    ts = [R.btensor(np.asarray(t, dtype=NPT[dtype]), None, dtype) for t in net.tensors]
    return ts


@pytest.mark.parametrize("dtype,tol", [(R.C128, 1e-12), (R.C64, 1e-5)])
def test_sliced_20_qubit_amplitude(dtype, tol):
    """The 20-qubit 4x5 depth-12 circuit sliced over 8 bonds (256 subnetworks,
    one batch, steps shared between slices), slice results summed in FP64."""
    circ = W.rqc20_config()
    net = W.circuit_network(circ)
    ext = [t.shape for t in net.tensors]
    path, _ = R.path_search(net.labels, ext, net.out_labels, ntrials=32, seed=1)
    cut, _, _ = R.slice_search(net.labels, ext, net.out_labels, path, 8)
    ts = _device_network(net, dtype)
    subs = R.sliced_networks(ts, net.labels, net.out_labels, cut)
    assert len(subs) == 256
    nets = [n for _, n in subs]
    outs = R.contract_batch(nets, [path] * len(nets), flags=R.OPT_GRAPH)
    total = complex(R.sum_fp64(outs).download())
    ref = oracle.amplitude_sv(circ)
    assert abs(total - ref) / max(abs(ref), 2.0 ** -10) <= tol
    req, planned, launches, _ = R.plan_stats(nets, [path] * len(nets), flags=R.OPT_GRAPH)
    assert req == 256 * (len(net.tensors) - 1)
    assert planned < req / 4          # slices share every step no cut bond reaches
    assert launches < 80              # grouped by dependency wave, not per step
    # replay through the cached plan and graph gives the same sum
    outs2 = R.contract_batch(nets, [path] * len(nets), flags=R.OPT_GRAPH)
    assert complex(R.sum_fp64(outs2).download()) == total


def test_sliced_simplified_20_qubit_amplitude():
    """The batch workload's recipe: the network simplified on the device
    first, then sliced over 8 bonds of the simplified network (256
    subnetworks in one batch), slice results summed in FP64."""
    circ = W.rqc20_config()
    net = W.circuit_network(circ)
    raw = _device_network(net, R.C128)
    ts, labels, _ = R.simplify(raw, net.labels, net.out_labels)
    assert len(ts) < len(raw) // 3
    ext = [t.shape for t in ts]
    path, _ = R.path_search(labels, ext, net.out_labels, ntrials=32, seed=1)
    cut, _, _ = R.slice_search(labels, ext, net.out_labels, path, 8)
    nets = [n for _, n in R.sliced_networks(ts, labels, net.out_labels, cut)]
    assert len(nets) == 256
    total = complex(R.sum_fp64(R.contract_batch(nets, [path] * len(nets), flags=R.OPT_GRAPH)).download())
    ref = oracle.amplitude_sv(circ)
    assert abs(total - ref) / max(abs(ref), 2.0 ** -10) <= 1e-12


def test_sliced_matches_oracle_sliced_per_slice():
    """Each slice's result equals the oracle's projection of the same network."""
    circ = W.random_circuit(12, 8, 31)
    net = W.circuit_network(circ)
    ext = [t.shape for t in net.tensors]
    path, _ = R.path_search(net.labels, ext, net.out_labels, ntrials=8, seed=2)
    cut, _, _ = R.slice_search(net.labels, ext, net.out_labels, path, 3)
    ts = _device_network(net, R.C128)
    subs = R.sliced_networks(ts, net.labels, net.out_labels, cut)
    outs = R.contract_batch([n for _, n in subs], [path] * len(subs))
    for (vals, _), o in zip(subs, outs):
        proj = oracle.sliced_contract(
            W.Network(tensors=[np.asarray(t) for t in net.tensors], labels=net.labels,
                      out_labels=net.out_labels), path, [])
        # oracle of this one projection
        val = dict(zip(cut, vals))
        pts, pls = [], []
        for t, l in zip(net.tensors, net.labels):
            idx = tuple(val[x] if x in val else slice(None) for x in l)
            pts.append(np.asarray(t)[idx])
            pls.append(tuple(x for x in l if x not in val))
        ref = oracle.contract(W.Network(tensors=pts, labels=pls, out_labels=net.out_labels), path)
        assert abs(complex(o.download()) - complex(ref)) <= 1e-12
    assert proj is not None


def test_batch_of_different_circuits():
    """Circuits of 8-14 qubits and depths 4-10 in one batch: each result equals
    its own state-vector amplitude."""
    rng = np.random.default_rng(5)
    circs = [W.random_circuit(int(rng.integers(8, 15)), int(rng.integers(4, 11)), 100 + i)
             for i in range(12)]
    nets, paths = [], []
    for c in circs:
        net = W.circuit_network(c)
        ts = _device_network(net, R.C64)
        n = R.Network(ts, net.labels, net.out_labels)
        nets.append(n)
        paths.append(n.greedy_path())
    outs = R.contract_batch(nets, paths, flags=R.OPT_GRAPH)
    for c, o in zip(circs, outs):
        ref = oracle.amplitude_sv(c)
        assert abs(complex(o.download()) - ref) / max(abs(ref), 2.0 ** (-c.n / 2)) <= 1e-5


def test_sum_fp64_and_fix_views():
    a = W.complex_normal((3, 4), 1).astype(np.complex64)
    b = W.complex_normal((3, 4), 2).astype(np.complex64)
    s = R.sum_fp64([R.btensor(a), R.btensor(b), R.btensor(a)]).download()
    np.testing.assert_allclose(s, a.astype(complex) * 2 + b, rtol=1e-7)
    t = R.btensor(W.complex_normal((2, 3, 4), 3), (1, 3, 2), R.C128)
    x = t.download()
    np.testing.assert_array_equal(t.fix([1], [2]).download(), x[:, 2, :])
    np.testing.assert_array_equal(t.fix([2, 0], [3, 1]).download(), x[1, :, 3])
    with pytest.raises(R.RosnetError):
        R.sum_fp64([R.btensor(a), R.btensor(a[:2])])
