"""C-ABI checks that need no GPU: the library loads, exports every function
that include/rosnet.h declares, validates arguments before touching the
device, and its host-side path planner behaves as specified."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2201_06620_b300 as R
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    txt = open(os.path.join(ROOT, "include", "rosnet.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rosnet_[a-z_0-9]+)\s*\(", txt)))


def test_library_builds_and_loads():
    from paper_2201_06620_b300 import build
    build.build()
    assert R.lib() is not None


def test_exports_every_declared_function():
    names = header_functions()
    assert len(names) >= 15
    L = R.lib()
    for n in names:
        assert hasattr(L, n), n
    assert sorted(R.EXPORTS) == names


def test_status_strings():
    L = R.lib()
    for code, name in R.STATUS.items():
        s = L.rosnet_status_string(code).decode()
        assert s and s != "unknown status"
    assert L.rosnet_status_string(12345).decode() == "unknown status"


def _create(rank, shape, block, dtype=R.C64):
    L = R.lib()
    h = ctypes.c_void_p()
    sh = (ctypes.c_int64 * max(1, len(shape)))(*shape)
    bl = (ctypes.c_int64 * max(1, len(block)))(*block) if block is not None else None
    rc = L.rosnet_btensor_create(rank, sh, bl, dtype, None, ctypes.byref(h))
    return rc, h


def test_create_validates_before_allocating():
    L = R.lib()
    assert _create(65, [2] * 65, [2] * 65)[0] == -6          # RANK_LIMIT
    assert _create(2, [4, 6], [3, 6])[0] == -3               # 3 does not divide 4
    assert _create(1, [4], [0])[0] == -3                     # block extent < 1
    assert _create(1, [-1], [1])[0] == -1                    # negative extent
    assert _create(1, [4], [4], dtype=7)[0] == -4            # unknown dtype
    sh = (ctypes.c_int64 * 1)(4)
    assert L.rosnet_btensor_create(1, sh, None, 1, None, None) == -1  # NULL out


def test_null_arguments_rejected():
    L = R.lib()
    out = ctypes.c_void_p()
    assert L.rosnet_tensordot(None, None, 0, None, None, None, None, ctypes.byref(out)) == -1
    assert out.value is None
    assert L.rosnet_btensor_destroy(None) == 0
    assert L.rosnet_contract(None, None, None, None, ctypes.byref(out)) == -1
    rk = ctypes.c_int()
    assert L.rosnet_btensor_info(None, ctypes.byref(rk), None, None, None) == -1


def test_set_allocator_pairs():
    L = R.lib()
    alloc = R._ALLOC_T(lambda n, s, c: None)
    assert L.rosnet_set_allocator(alloc, R._FREE_T(), None) == -1   # alloc without free
    assert L.rosnet_set_allocator(R._ALLOC_T(), R._FREE_T(), None) == 0  # built-in


# ---------------------------------------------------------------------------
# greedy path (host logic)
# ---------------------------------------------------------------------------
def _simulate(labels, extents, out, path):
    """Check an SSA path and return, per step, the chosen size and the
    minimum size over all connected live pairs."""
    ext = {}
    for l, e in zip(labels, extents):
        for x, y in zip(l, e):
            ext[x] = y
    live = {i: list(l) for i, l in enumerate(labels)}
    nxt = len(labels)
    rows = []
    size = lambda ls: int(np.prod([ext[x] for x in ls], dtype=np.int64)) if ls else 1
    res = lambda a, b: [x for x in live[a] if x not in live[b]] + [x for x in live[b] if x not in live[a]]
    for a, b in path:
        assert a in live and b in live and a != b
        cands = [size(res(i, j)) for i in live for j in live
                 if i < j and set(live[i]) & set(live[j])]
        rows.append((size(res(a, b)), min(cands) if cands else None,
                     bool(set(live[a]) & set(live[b]))))
        lc = res(a, b)
        del live[a], live[b]
        live[nxt] = lc
        nxt += 1
    assert len(live) == 1
    (last,) = live.values()
    assert sorted(last) == sorted(out)
    return rows


@pytest.mark.parametrize("n,depth,seed", [(6, 4, 0), (9, 6, 1), (12, 8, 2)])
def test_greedy_path_is_greedy(n, depth, seed):
    circ = W.random_circuit(n, depth, seed)
    for open_out in (False, True):
        net = W.circuit_network(circ, open_output=open_out)
        ext = [t.shape for t in net.tensors]
        path = R.path_greedy_extents(net.labels, ext, net.out_labels)
        assert len(path) == len(net.tensors) - 1
        for chosen, best, connected in _simulate(net.labels, ext, net.out_labels, path):
            if best is not None:
                assert connected and chosen == best


def test_greedy_path_disconnected_and_errors():
    # two components: the outer product comes last
    labels = [(0, 1), (1, 2), (10, 11), (11, 12)]
    ext = [(2, 3), (3, 2), (2, 2), (2, 2)]
    path = R.path_greedy_extents(labels, ext, [0, 2, 10, 12])
    rows = _simulate(labels, ext, [0, 2, 10, 12], path)
    assert [r[2] for r in rows] == [True, True, False]
    with pytest.raises(R.RosnetError) as e:
        R.path_greedy_extents([(0,), (0,)], [(2,), (3,)], [])
    assert e.value.name == "SHAPE"
    with pytest.raises(R.RosnetError) as e:
        R.path_greedy_extents([(0,), (0,), (0,)], [(2,), (2,), (2,)], [])
    assert e.value.name == "UNSUPPORTED"


def test_greedy_path_rqc20_structure():
    circ = W.rqc20_config()
    net = W.circuit_network(circ)
    ext = [t.shape for t in net.tensors]
    path = R.path_greedy_extents(net.labels, ext, net.out_labels)
    assert len(path) == 372
    rows = _simulate(net.labels, ext, net.out_labels, path)
    assert max(r[0] for r in rows) <= 2 ** 20
