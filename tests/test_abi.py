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
    # 2^60 complex128 entries would need 2^65 bytes: refused before any
    # allocation (the byte count must not wrap around)
    assert _create(2, [1 << 30, 1 << 30], [1, 1 << 30], dtype=R.C128)[0] == -2   # SHAPE
    assert _create(3, [1 << 20, 1 << 20, 1 << 19], None)[0] == -2
    rc, h = _create(2, [0, 1 << 62], None)                  # empty: nothing to size
    assert rc != -2
    if rc == 0:
        L.rosnet_btensor_destroy(h)
    sh = (ctypes.c_int64 * 1)(4)
    assert L.rosnet_btensor_create(1, sh, None, 1, None, None) == -1  # NULL out


def test_null_arguments_rejected():
    L = R.lib()
    out = ctypes.c_void_p()
    assert L.rosnet_tensordot(None, None, 0, None, None, None, None, ctypes.byref(out)) == -1
    assert out.value is None
    assert L.rosnet_btensor_destroy(None) == 0
    assert L.rosnet_btensor_upload_raw(None, None, None) == -1
    assert L.rosnet_btensor_download_raw(None, None, None) == -1
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


def test_predict_footprint_matches_eq2_for_one_pair():
    """For one pair of blocks the serving footprint predictor gives the
    paper's per-task memory of Eq. 2, k_b (m_b + n_b) + m_b n_b elements."""
    import oracle
    from paper_2201_06620_b300.serving import predict_footprint
    for mb, nb, kb in ((8, 4, 16), (1, 1, 1), (64, 32, 128)):
        got = predict_footprint([(0, 1), (1, 2)], [(mb, kb), (kb, nb)], [0, 2], [(0, 1)], elem_bytes=1)
        assert got == oracle.mem_pair(mb, nb, kb)


def _path_flops(labels, extents, path, cut=()):
    ext = {}
    for l, e in zip(labels, extents):
        for x, y in zip(l, e):
            ext[x] = 1 if x in cut else y
    live = {i: list(l) for i, l in enumerate(labels)}
    nxt, tot, mx = len(labels), 0.0, 0.0
    for a, b in path:
        la, lb = live.pop(a), live.pop(b)
        union = set(la) | set(lb)
        tot += 8.0 * float(np.prod([ext[x] for x in union]))
        lc = [x for x in la if x not in lb] + [x for x in lb if x not in la]
        mx = max(mx, float(np.prod([ext[x] for x in lc])) if lc else 1.0)
        live[nxt] = lc
        nxt += 1
    return tot, mx


def test_path_search_never_worse_than_greedy_and_reports_flops():
    circ = W.random_circuit(16, 8, 4)
    net = W.circuit_network(circ)
    ext = [t.shape for t in net.tensors]
    greedy = R.path_greedy_extents(net.labels, ext, net.out_labels)
    path, flops = R.path_search(net.labels, ext, net.out_labels, ntrials=8, seed=3)
    _simulate(net.labels, ext, net.out_labels, path)       # a valid SSA path
    assert abs(_path_flops(net.labels, ext, path)[0] - flops) <= 1e-9 * flops
    assert flops <= _path_flops(net.labels, ext, greedy)[0]
    assert R.path_search(net.labels, ext, net.out_labels, ntrials=8, seed=3) == (path, flops)


def test_slice_search_shrinks_the_largest_intermediate():
    circ = W.random_circuit(14, 8, 6)
    net = W.circuit_network(circ)
    ext = [t.shape for t in net.tensors]
    path, _ = R.path_search(net.labels, ext, net.out_labels, ntrials=4, seed=1)
    cut, mx, flops = R.slice_search(net.labels, ext, net.out_labels, path, 4)
    assert len(set(cut)) == 4
    counts = {}
    for l in net.labels:
        for x in l:
            counts[x] = counts.get(x, 0) + 1
    assert all(counts[c] == 2 for c in cut)                # bonds, not open legs
    t0, m0 = _path_flops(net.labels, ext, path)
    t1, m1 = _path_flops(net.labels, ext, path, cut)
    assert mx == m1 < m0
    assert abs(flops - 16 * t1) <= 1e-9 * flops             # 2^4 slices



def test_slice_search_rejects_malformed_paths():
    circ = W.random_circuit(6, 4, 2)
    net = W.circuit_network(circ)
    ext = [t.shape for t in net.tensors]
    path = R.path_greedy_extents(net.labels, ext, net.out_labels)
    nt = len(net.labels)
    R.slice_search(net.labels, ext, net.out_labels, path, 1)          # the valid path is accepted
    bad = [
        path[:-1],                                                      # a step short
        [(0, nt + 5)] + path[1:],                                       # an id not yet created
        [(0, 0)] + path[1:],                                            # an id paired with itself
        [path[0], (path[0][0], path[1][1])] + path[2:],                 # an id used twice
        [(-1, path[0][1])] + path[1:],                                  # negative id
    ]
    for p in bad:
        with pytest.raises(R.RosnetError) as e:
            R.slice_search(net.labels, ext, net.out_labels, p, 1)
        assert e.value.name == "INVALID_ARG", p

def test_tune_table_roundtrip_and_validation():
    """Autotuner decisions move between processes as text; every imported
    entry is checked against its shape (no device needed)."""
    good = ("1 9 4096 256 256 10 1 1\n1 11 2048 512 32 3 1 0\n2 0 300 200 5000 2 16 0\n"
            "1 1 300 13 4000 11 8 0\n1 1 200 30 300 12 1 0\n1 3 2048 512 32 13 1 0\n2 3 300 40 20 13 1 0\n"
            "1 9 256 16 4096 14 128 0\n1 9 300 200 100 13 4 0\n1 9 1000 700 200 10 1 0\n")
    R.tune_import(good)
    lines = set(R.tune_export().splitlines())
    assert set(good.splitlines()) <= lines
    R.tune_import("1 9 4096 256 256 2 4\n")          # replaces the first entry; no schedule field = 0
    assert "1 9 4096 256 256 2 4 0" in R.tune_export().splitlines()
    bad = ["1 9 4096 256 256 10 2",      # packed kind cannot split
           "1 9 100 40 256 3 1",         # 128x64 tiles need M >= 128, N >= 48
           "2 0 64 64 64 10 1",          # packed FP32 is complex64 only
           "1 0 64 64 64 2 5",           # 4 k-tiles cannot make 5 ranges
           "1 0 64 64 64 7 1",           # not a CUDA-core GEMM kind
           "3 0 64 64 64 2 1",           # unknown dtype
           "1 0 64 64",                  # short line
           "1 0 64 64 64 2 1 9",         # schedule is 0 or 1
           "1 0 64 64 64 2 1 1",         # stream-K is a schedule of the packed kind only
           "1 0 64 64 64 10 1 0 0",      # extra field
           "2 0 300 13 200 11 1",        # 256x16 tiles are complex64 only
           "1 0 100 13 200 11 1",        # 256x16 tiles need M >= 128
           "1 0 300 300 33 13 1",        # direct tiles hold 32 contracted indices per CTA
           "1 0 300 300 32 13 2",        # so K = 32 is one range
           "1 0 300 13 4096 14 64",      # and K = 4096 is 128, not 64
           "2 0 300 13 4096 14 128"]     # 256x16 direct tiles are complex64 only
    before = R.tune_export()
    for b in bad:
        with pytest.raises(R.RosnetError) as e:
            R.tune_import("1 0 128 128 128 2 1\n" + b + "\n")
        assert e.value.name == "INVALID_ARG", b
    assert R.tune_export() == before      # nothing merged from a rejected text


def test_allocator_switch_needs_no_live_blocks_and_stats():
    """A block is freed by the allocator that made it: with no library memory
    alive the allocator can be swapped back and forth (no device needed)."""
    req, live = R.alloc_stats()
    assert req >= 0 and live >= 0
    if live == 0:
        alloc = R._ALLOC_T(lambda n, s, c: None)
        free = R._FREE_T(lambda p, s, c: None)
        assert R.lib().rosnet_set_allocator(alloc, free, None) == 0
        assert R.lib().rosnet_set_allocator(R._ALLOC_T(), R._FREE_T(), None) == 0


def test_plan_cache_limit_is_host_side():
    """Setting and querying the plan-cache bound needs no device (nothing is
    cached once the plans are released, whatever ran earlier in the process)."""
    R.release_plans()
    assert R.plan_cache_limit() == 0
    assert R.plan_cache_limit(3) == 0
    assert R.plan_cache_limit(-1) == 0
    assert R.plan_cache_limit(0) == 0


def test_network_labels_reach_the_c_side_unchanged():
    """The binding packs all label rows into one flat array with row pointers;
    every label, rank and output label reads back through the structure the C
    side receives (empty rows and 64-bit labels included)."""
    rng = np.random.default_rng(5)

    class Handle:   # Network only records a tensor's handle
        handle = ctypes.c_void_p(0)

    for _ in range(50):
        n = int(rng.integers(1, 30))
        labels = [tuple(int(x) for x in rng.integers(-10**12, 10**12, int(rng.integers(0, 7))))
                  for _ in range(n)]
        out = [int(x) for x in rng.integers(0, 100, int(rng.integers(0, 5)))]
        net = R.Network([Handle() for _ in range(n)], labels, out)
        assert net.net.ntensors == n and net.net.nout == len(out)
        for t, l in enumerate(labels):
            assert net.net.ranks[t] == len(l)
            assert [net.net.labels[t][i] for i in range(len(l))] == list(l)
        assert [net.net.out_labels[i] for i in range(len(out))] == out

