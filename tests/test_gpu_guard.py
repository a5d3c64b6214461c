"""Out-of-bounds guard for the kernels' stores (the stand-in for a memory
checker): every device block the library allocates comes from a test
allocator that surrounds it with 4 KiB canary bands, and the bands are
checked when the block is freed and after every case.  A kernel writing past
an output tile, a split-K partial, an offset table or a packed workspace
changes a band and fails the test, where a parity check alone could miss it.

Cases cover ragged tiles of every CUDA-core family, split-K partials and
their sum, the packed FP32 GEMM (pack pass, in-place operands, stream-K
pieces), the tensor-core GEMM with ragged edges, the gate kernel, and a
network plan replayed as a graph; each result is also checked against the
oracle.
"""
import gc

import numpy as np
import pytest

import oracle
import paper_2201_06620_b300 as R
import workloads as W

pytestmark = pytest.mark.gpu

GUARD = 4096
CANARY = 0xA5


class GuardedAllocator:
    def __init__(self, torch):
        self.torch = torch
        self.blocks = {}     # user pointer -> (backing tensor, bytes)
        self.broken = []

    def _check(self, ptr):
        buf, n = self.blocks[ptr]
        head = buf[:GUARD]
        tail = buf[GUARD + n:]
        if not (bool((head == CANARY).all()) and bool((tail == CANARY).all())):
            self.broken.append(n)

    def alloc(self, nbytes, stream, ctx):
        torch = self.torch
        torch.cuda.synchronize()
        buf = torch.full((int(nbytes) + 2 * GUARD,), CANARY, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        ptr = buf.data_ptr() + GUARD
        self.blocks[ptr] = (buf, int(nbytes))
        return ptr

    def free(self, ptr, stream, ctx):
        self.torch.cuda.synchronize()
        self._check(ptr)
        del self.blocks[ptr]

    def check_all(self):
        self.torch.cuda.synchronize()
        for p in list(self.blocks):
            self._check(p)
        return not self.broken


@pytest.fixture()
def guarded():
    import torch
    gc.collect()
    R.release_plans()
    R.sync()
    assert R.alloc_stats()[1] == 0, "library blocks still alive before switching allocators"
    ga = GuardedAllocator(torch)
    cbs = (R._ALLOC_T(ga.alloc), R._FREE_T(ga.free))
    R._check(R.lib().rosnet_set_allocator(cbs[0], cbs[1], None), "rosnet_set_allocator")
    try:
        yield ga
    finally:
        gc.collect()
        R.release_plans()
        R.sync()
        R._check(R.lib().rosnet_set_allocator(R._ALLOC_T(), R._FREE_T(), None), "rosnet_set_allocator")
        del cbs


def _c(shape, seed, dt=np.complex64):
    return W.complex_normal(shape, seed).astype(dt)


def _case_tensordot(a, b, ax_a, ax_b, tol, **kw):
    A, B = R.btensor(a), R.btensor(b)
    C = R.tensordot(A, B, ax_a, ax_b, **kw)
    got = C.download()
    assert oracle.rel_frobenius(got, oracle.tensordot(a, b, ax_a, ax_b)) <= tol
    del A, B, C


def test_kernel_stores_stay_inside_their_blocks(guarded):
    cases = [
        # ragged 64x64 / 128x64 / 128x32 / 256x16 tiles and direct tiles
        ((257, 130), (130, 515), [1], [0], np.complex64, {}),
        ((300, 24), (24, 13), [1], [0], np.complex64, {}),
        ((257, 130), (130, 31), [1], [0], np.complex64, {}),
        ((257, 130), (130, 515), [1], [0], np.complex128, {}),
        # split-K: stored partials (tree) and order-free adds (commutative)
        ((65, 4100), (4100, 63), [1], [0], np.complex64, {"flags": R.REDUCE_TREE}),
        ((65, 4100), (4100, 63), [1], [0], np.complex64, {"flags": R.REDUCE_COMMUTATIVE}),
        # packed FP32: pack pass (M x K storage), in place (K x M), stream-K pieces
        ((1000, 200), (200, 700), [1], [0], np.complex64, {}),
        ((200, 1000), (200, 700), [0], [0], np.complex64, {}),
        ((1100, 1000), (1100, 900), [0], [0], np.complex64, {}),
        # tensor cores with ragged edges
        ((257, 130), (130, 515), [1], [0], np.complex64, {"precision": R.PREC_TF32X3}),
        ((257, 130), (130, 515), [1], [0], np.complex64, {"precision": R.PREC_BF16X3}),
        # gate kernel (both store paths) and a projection
        ((2,) * 16, (2, 2), [5], [1], np.complex64, {}),
        ((2, 2), (2,) * 16, [1], [5], np.complex64, {}),
        ((2,) * 16, (2,), [3], [0], np.complex64, {}),
    ]
    for i, (sa, sb, ax_a, ax_b, dt, kw) in enumerate(cases):
        tol = 1e-12 if dt == np.complex128 else (1e-4 if kw.get("precision") == R.PREC_BF16X3 else 1e-5)
        _case_tensordot(_c(sa, 2 * i + 1, dt), _c(sb, 2 * i + 2, dt), ax_a, ax_b, tol, **kw)
        assert guarded.check_all(), (i, sa, sb, kw, guarded.broken)
    # a network plan (arena, shared tables, grouped launches) replayed as a graph
    circ = W.random_circuit(14, 10, 5)
    net = W.circuit_network(circ)
    ts = [R.btensor(np.asarray(t, dtype=np.complex64)) for t in net.tensors]
    path = R.path_greedy(ts, net.labels, net.out_labels)
    ref = oracle.amplitude_sv(circ)
    for _ in range(3):
        got = complex(R.contract(ts, net.labels, net.out_labels, path, flags=R.OPT_GRAPH,
                                 max_block_entries=256).download())
        assert abs(got - ref) / max(abs(ref), 2.0 ** -7) <= 1e-5
    assert guarded.check_all(), guarded.broken
    del ts
    gc.collect()
    R.release_plans()
    R.sync()
    assert guarded.check_all() and not guarded.blocks, (guarded.broken, len(guarded.blocks))
