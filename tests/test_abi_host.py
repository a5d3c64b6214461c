"""Host-side logic of the C ABI exercised without a GPU: block tensors are
created with an injected allocator that hands out host memory, so layouts,
views and the argument checks of tensordot, out-of-core tensordot, sums and
network contraction can be tested on the CPU.  Every call here either does no
device work at all (views, info, paths) or must be refused before any device
work is enqueued (invalid arguments); none runs a kernel.  On a machine with a
GPU the module is skipped, so host pointers can never reach a kernel there."""
import ctypes

import pytest

import paper_2201_06620_b300 as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.skipif(torch.cuda.is_available(),
                                reason="host-memory tensors are only made where no GPU exists")

vp = ctypes.c_void_p
STATUS = R.STATUS   # code -> name


@pytest.fixture(scope="module")
def L():
    lib = R.lib()
    held = {}

    def alloc(nbytes, stream, ctx):
        buf = ctypes.create_string_buffer(max(int(nbytes), 1))
        held[ctypes.addressof(buf)] = buf
        return ctypes.addressof(buf)

    def free(ptr, stream, ctx):
        held.pop(ptr)

    cbs = (R._ALLOC_T(alloc), R._FREE_T(free))
    if lib.rosnet_set_allocator(cbs[0], cbs[1], None) != 0:
        pytest.skip("the library holds device blocks; its allocator cannot be swapped")
    lib.rosnet_btensor_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int)]
    lib.rosnet_btensor_planes.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp)]
    lib.rosnet_tensordot.argtypes = [vp, vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(R._Opts), vp,
                                     ctypes.POINTER(vp)]
    lib.rosnet_tensordot_ooc.argtypes = [vp, vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int64,
                                         ctypes.c_int64, ctypes.POINTER(R._Opts), vp, ctypes.c_size_t, vp]
    lib.rosnet_tensordot_ooc_host.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                              ctypes.POINTER(ctypes.c_int64), vp, vp, ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                              ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                              ctypes.POINTER(R._Opts), vp, ctypes.c_size_t, vp]
    lib.rosnet_path_greedy.argtypes = [ctypes.POINTER(R._Network), ctypes.POINTER(ctypes.c_int32),
                                       ctypes.POINTER(ctypes.c_int32)]
    lib._held = held
    yield lib
    assert not held, "tensors left alive"
    assert lib.rosnet_set_allocator(R._ALLOC_T(), R._FREE_T(), None) == 0


class T:
    """A host-memory block tensor (destroyed explicitly)."""

    def __init__(self, L, shape, block=None, dtype=R.C64):
        self.L = L
        self.handle = vp()
        sh = (ctypes.c_int64 * max(1, len(shape)))(*shape)
        bl = (ctypes.c_int64 * max(1, len(shape)))(*block) if block is not None else None
        rc = L.rosnet_btensor_create(len(shape), sh, bl, dtype, None, ctypes.byref(self.handle))
        assert rc == 0, STATUS.get(rc, rc)

    @classmethod
    def wrap(cls, L, h):
        t = cls.__new__(cls)
        t.L, t.handle = L, h
        return t

    def info(self):
        rk = ctypes.c_int()
        sh = (ctypes.c_int64 * 64)()
        bl = (ctypes.c_int64 * 64)()
        dt = ctypes.c_int()
        assert self.L.rosnet_btensor_info(self.handle, ctypes.byref(rk), sh, bl, ctypes.byref(dt)) == 0
        return tuple(sh[:rk.value]), tuple(bl[:rk.value]), dt.value

    def planes(self):
        re, im = vp(), vp()
        assert self.L.rosnet_btensor_planes(self.handle, ctypes.byref(re), ctypes.byref(im)) == 0
        return re.value, im.value

    def destroy(self):
        assert self.L.rosnet_btensor_destroy(self.handle) == 0


def _i64(seq):
    seq = list(seq)
    return (ctypes.c_int64 * max(1, len(seq)))(*seq)


def _i32(seq):
    seq = list(seq)
    return (ctypes.c_int * max(1, len(seq)))(*seq)


def test_block_major_layout_and_views(L):
    """Sec. II-C storage: blocks in row-major order of their grid coordinates,
    each block row-major inside; views share the storage at those offsets."""
    A = T(L, (4, 6, 8), (2, 3, 4))            # grid (2, 2, 2), blocks of 24 entries
    try:
        assert A.info() == ((4, 6, 8), (2, 3, 4), R.C64)
        re, im = A.planes()
        assert im - re == 4 * 6 * 8 * 4       # imaginary plane after the real one
        for g in [(0, 0, 0), (0, 1, 1), (1, 0, 1), (1, 1, 1)]:
            v = vp()
            assert L.rosnet_btensor_block(A.handle, _i64(g), ctypes.byref(v)) == 0
            V = T.wrap(L, v)
            assert V.info() == ((2, 3, 4), (2, 3, 4), R.C64)
            # block g starts after (row-major index of g) whole blocks
            assert V.planes()[0] - re == ((g[0] * 2 + g[1]) * 2 + g[2]) * 24 * 4
            V.destroy()
        # element (x0, x1, x2): block (x // b) then row-major inside it
        x = (3, 4, 6)
        v = vp()
        assert L.rosnet_btensor_fix(A.handle, 3, _i32([0, 1, 2]), _i64(x), ctypes.byref(v)) == 0
        V = T.wrap(L, v)
        assert V.info() == ((), (), R.C64)
        blk = ((x[0] // 2) * 2 + x[1] // 3) * 2 + x[2] // 4
        inner = ((x[0] % 2) * 3 + x[1] % 3) * 4 + x[2] % 4
        assert V.planes()[0] - re == (blk * 24 + inner) * 4
        V.destroy()
        # fixing one axis keeps the others with their blocks
        assert L.rosnet_btensor_fix(A.handle, 1, _i32([1]), _i64([4]), ctypes.byref(v)) == 0
        V = T.wrap(L, v)
        assert V.info() == ((4, 8), (2, 4), R.C64)
        V.destroy()
        for axes, vals in (([1, 1], [0, 0]), ([3], [0]), ([0], [4]), ([0], [-1])):
            rc = L.rosnet_btensor_fix(A.handle, len(axes), _i32(axes), _i64(vals), ctypes.byref(v))
            assert STATUS[rc] == "INVALID_ARG" and v.value is None, (axes, vals)
        assert STATUS[L.rosnet_btensor_block(A.handle, _i64([2, 0, 0]), ctypes.byref(v))] == "INVALID_ARG"
        # slicing wants grid axes (block extent 1)
        assert STATUS[L.rosnet_btensor_slice(A.handle, 1, _i64([0]), ctypes.byref(v))] == "BLOCK_MISMATCH"
    finally:
        A.destroy()
    S = T(L, (3, 6), (1, 3), R.C128)
    try:
        assert L.rosnet_btensor_slice(S.handle, 1, _i64([2]), ctypes.byref(v)) == 0
        V = T.wrap(L, v)
        assert V.info() == ((6,), (3,), R.C128)
        assert V.planes()[0] - S.planes()[0] == 2 * 6 * 8
        # raw copies need an owning tensor, not a view
        assert STATUS[L.rosnet_btensor_upload_raw(V.handle, S.planes()[0], None)] == "UNSUPPORTED"
        V.destroy()
        assert STATUS[L.rosnet_btensor_slice(S.handle, 1, _i64([3]), ctypes.byref(v))] == "INVALID_ARG"
        # upload ranges are checked against the tensor
        buf = ctypes.create_string_buffer(16 * 18)
        for start, count in ((0, 19), (18, 1), (-1, 1), (5, -1)):
            rc = L.rosnet_btensor_upload_range(S.handle, buf, start, count, None)
            assert STATUS[rc] == "INVALID_ARG", (start, count)
    finally:
        S.destroy()


def _opts(precision=0, flags=0, reserved0=0):
    o = R._Opts()
    o.precision, o.flags = precision, flags
    o.reserved[0] = reserved0
    return o


def _tdot(L, A, B, ax_a, ax_b, opts=None):
    out = vp(1234)
    rc = L.rosnet_tensordot(A.handle, B.handle, len(ax_a), _i32(ax_a), _i32(ax_b),
                            ctypes.byref(opts) if opts is not None else None, None, ctypes.byref(out))
    assert out.value is None       # nothing returned on error
    return STATUS[rc]


def test_tensordot_argument_checks(L):
    """numpy tensordot rules and the block rules of Sec. II-C, refused before
    any device work."""
    A = T(L, (2, 3, 4), (1, 3, 2))
    B = T(L, (4, 3), (2, 3))
    Bc = T(L, (4, 3), (2, 3), R.C128)
    Bb = T(L, (4, 3), (4, 3))
    W1 = T(L, (1,) * 40)
    W2 = T(L, (1,) * 40)
    try:
        assert _tdot(L, A, B, [1], [0]) == "SHAPE"              # extents 3 and 4
        assert _tdot(L, A, B, [3], [0]) == "INVALID_ARG"        # no axis 3
        assert _tdot(L, A, B, [-4], [0]) == "INVALID_ARG"
        assert _tdot(L, A, B, [2, 2], [0, 1]) == "INVALID_ARG"  # axis twice
        assert _tdot(L, A, B, [2, 1, 0], [0, 1, 1]) == "INVALID_ARG"   # more axes than B has
        assert _tdot(L, A, Bc, [2], [0]) == "DTYPE"
        assert _tdot(L, A, Bb, [2], [0]) == "BLOCK_MISMATCH"     # block extents 2 and 4
        assert _tdot(L, W1, W2, [], []) == "RANK_LIMIT"          # rank-80 result
        assert _tdot(L, A, B, [2], [0], _opts(precision=99)) == "INVALID_ARG"
        assert _tdot(L, A, B, [2], [0], _opts(precision=R.PREC_FP64)) == "UNSUPPORTED"
        assert _tdot(L, A, B, [2], [0], _opts(reserved0=1)) == "INVALID_ARG"
        assert _tdot(L, A, B, [2], [0], _opts(flags=R.REDUCE_TREE | R.REDUCE_SEQUENTIAL)) == "INVALID_ARG"
        Ac = T(L, (2, 3, 4), (1, 3, 2), R.C128)
        try:
            assert _tdot(L, Ac, Bc, [2], [0], _opts(precision=R.PREC_TF32)) == "UNSUPPORTED"
        finally:
            Ac.destroy()
        # out-of-core: split axes must be free grid axes and the chunk range in bounds
        host = ctypes.create_string_buffer(1 << 12)

        def ooc(nsplit, first, n, ax_a=(2,), ax_b=(0,)):
            return STATUS[L.rosnet_tensordot_ooc(A.handle, B.handle, len(ax_a), _i32(ax_a), _i32(ax_b),
                                                 nsplit, first, n, None, host, len(host), None)]
        assert ooc(1, 0, 3) == "INVALID_ARG"                    # only 2 chunks along axis 0
        assert ooc(1, -1, 1) == "INVALID_ARG"
        assert ooc(4, 0, 1) == "INVALID_ARG"                    # more split axes than A has
        assert ooc(2, 0, 1) == "BLOCK_MISMATCH"                 # axis 1 has block extent 3
        assert ooc(1, 0, 1, (0,), (1,)) == "SHAPE"                # extents 2 and 3
        assert ooc(1, 0, 0) == "OK"                             # empty range: nothing to do
        # the same checks with A in host memory (described by shape and blocks)
        a_host = ctypes.create_string_buffer(2 * 24 * 8)

        def ooch(nsplit, first, n, shape=(2, 3, 4), block=(1, 3, 2), ax_a=(2,), ax_b=(0,), src=a_host):
            sh = (ctypes.c_int64 * len(shape))(*shape)
            bl = (ctypes.c_int64 * len(block))(*block)
            return STATUS[L.rosnet_tensordot_ooc_host(len(shape), sh, bl, src, B.handle, len(ax_a), _i32(ax_a),
                                                      _i32(ax_b), nsplit, first, n, None, host, len(host), None)]
        assert ooch(1, 0, 3) == "INVALID_ARG"                   # only 2 chunks along axis 0
        assert ooch(2, 0, 1) == "BLOCK_MISMATCH"                # axis 1 has block extent 3
        assert ooch(1, 0, 1, block=(1, 3, 3)) == "BLOCK_MISMATCH"   # 3 does not divide 4
        assert ooch(1, 0, 1, ax_a=(0,), ax_b=(1,)) == "SHAPE"
        assert ooch(1, 0, 1, src=None) == "INVALID_ARG"          # no host array
        assert ooch(1, 0, 1, block=(1, 3, 4)) == "BLOCK_MISMATCH"   # contracted blocks 4 and 2
        assert ooch(1, 0, 0) == "OK"
    finally:
        for t in (A, B, Bc, Bb, W1, W2):
            t.destroy()


def test_sum_argument_checks(L):
    A = T(L, (2, 4), (1, 2))
    B = T(L, (2, 4), (2, 2))
    C = T(L, (2, 4), (1, 2), R.C128)
    try:
        out = vp(1)

        def s(*ts):
            arr = (vp * max(1, len(ts)))(*[t.handle.value for t in ts])
            return STATUS[L.rosnet_sum(len(ts), arr, None, ctypes.byref(out))]
        assert s() == "INVALID_ARG"
        assert s(A, B) == "SHAPE"           # different blocks
        assert s(A, C) == "DTYPE"
        assert out.value is None
    finally:
        for t in (A, B, C):
            t.destroy()


def _network(L, tensors, labels, out_labels):
    return R.Network(tensors, labels, out_labels)


def _contract(L, net, path):
    p = net._cpath(path)
    out = vp(1)
    rc = L.rosnet_contract(ctypes.byref(net.net), ctypes.byref(p), None, None, ctypes.byref(out))
    assert out.value is None
    return STATUS[rc]


def test_network_checks_and_greedy_path(L):
    """Sec. II-A networks: a label shared by two tensors is contracted, open
    labels must be listed as outputs; malformed networks and paths are refused
    while planning, before anything is allocated on the device."""
    a = T(L, (2, 3))
    b = T(L, (3, 4))
    c = T(L, (4, 2))
    d = T(L, (4,))
    z = T(L, (3, 4), None, R.C128)
    try:
        ring = _network(L, [a, b, c], [(0, 1), (1, 2), (2, 0)], [])
        pairs = (ctypes.c_int32 * 4)()
        ns = ctypes.c_int32()
        assert L.rosnet_path_greedy(ctypes.byref(ring.net), pairs, ctypes.byref(ns)) == 0
        path = [(pairs[0], pairs[1]), (pairs[2], pairs[3])]
        assert ns.value == 2 and sorted(path[0]) in ([0, 1], [0, 2], [1, 2]) and 3 in path[1]
        # the smallest first result: a-b gives 2x4 = 8 entries, b-c 3x2 = 6, a-c 3x4 = 12
        assert sorted(path[0]) == [1, 2]
        cases = [
            (_network(L, [a, b], [(0, 0), (0, 1)], [1]), [(0, 1)], "UNSUPPORTED"),        # trace
            (_network(L, [a, b], [(0, 1), (1, 2)], [0]), [(0, 1)], "INVALID_ARG"),         # 2 not listed
            (_network(L, [a, b], [(0, 1), (1, 2)], [0, 2, 0]), [(0, 1)], "INVALID_ARG"),   # repeated output
            (_network(L, [a, c], [(0, 1), (1, 0)], []), [(0, 1)], "SHAPE"),                # 3 vs 4, 2 vs 2
            (_network(L, [a, z], [(0, 1), (1, 2)], [0, 2]), [(0, 1)], "DTYPE"),
            (_network(L, [a, b, c], [(0, 1), (1, 2), (2, 0)], []), [(0, 1)], "INVALID_ARG"),          # a step short
            (_network(L, [a, b, c], [(0, 1), (1, 2), (2, 0)], []), [(0, 1), (0, 2)], "INVALID_ARG"),  # 0 reused
            (_network(L, [a, b, c], [(0, 1), (1, 2), (2, 0)], []), [(0, 1), (2, 4)], "INVALID_ARG"),  # id 4 unborn
        ]
        for net, p, want in cases:
            assert _contract(L, net, p) == want, (net.labels, p)
        three = _network(L, [a, b, d], [(0, 1), (1, 2), (2, 5)], [0, 5])
        assert _contract(L, three, [(0, 1)]) == "INVALID_ARG"
        bad_rank = _network(L, [a, b], [(0, 1), (1, 2)], [0, 2])
        bad_rank.ranks[0] = 3
        assert _contract(L, bad_rank, [(0, 1)]) == "INVALID_ARG"
        # spilling a plan that was never built is refused before any device work
        ring_path = (ctypes.c_int32 * 4)(pairs[0], pairs[1], pairs[2], pairs[3])
        rp = R._Path(2, ctypes.cast(ring_path, ctypes.POINTER(ctypes.c_int32)))
        L.rosnet_plan_spill.argtypes = [ctypes.c_int32, ctypes.POINTER(R._Network), ctypes.POINTER(R._Path),
                                        ctypes.POINTER(R._Opts), vp, ctypes.POINTER(ctypes.c_int64)]
        hb = ctypes.c_int64(-1)
        assert STATUS[L.rosnet_plan_spill(1, ctypes.byref(ring.net), ctypes.byref(rp), None, None,
                                          ctypes.byref(hb))] == "INVALID_ARG"
        assert hb.value == -1
        # a label on three tensors is not a pairwise bond
        tri = _network(L, [a, T.wrap(L, a.handle), T.wrap(L, a.handle)],
                       [(0, 1), (0, 2), (0, 3)], [1, 2, 3])
        assert _contract(L, tri, [(0, 1), (2, 3)]) == "UNSUPPORTED"
    finally:
        for t in (a, b, c, d, z):
            t.destroy()


def test_simplify_without_merges_does_no_device_work(L):
    """rosnet_simplify on networks where nothing may be absorbed (every small
    tensor kept, or only rank-3 tensors) returns the caller's handles, labels
    and positions unchanged without touching the device; bad arguments are
    refused."""
    L.rosnet_simplify.argtypes = [ctypes.POINTER(R._Network), ctypes.POINTER(ctypes.c_uint8), ctypes.c_int32,
                                  ctypes.POINTER(R._Opts), vp, ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int32),
                                  ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32),
                                  ctypes.POINTER(ctypes.c_int32)]
    a = T(L, (2, 3))
    b = T(L, (3, 4))
    c = T(L, (4, 2, 2))
    d = T(L, (2, 2, 5))
    try:
        def run(tensors, labels, out, keep, max_rank=2):
            net = _network(L, tensors, labels, out)
            n = len(tensors)
            kp = (ctypes.c_uint8 * n)(*keep) if keep is not None else None
            tout = (vp * n)()
            rout = (ctypes.c_int32 * n)()
            lout = (ctypes.c_int64 * sum(len(x) for x in labels))()
            oout = (ctypes.c_int32 * n)()
            nn = ctypes.c_int32()
            rc = L.rosnet_simplify(ctypes.byref(net.net), kp, max_rank, None, None, tout, rout, lout, oout,
                                   ctypes.byref(nn))
            return STATUS[rc], [tout[i] for i in range(nn.value)], [rout[i] for i in range(nn.value)], \
                list(lout[:sum(rout[i] for i in range(nn.value))]), [oout[i] for i in range(nn.value)]
        labels = [(0, 1), (1, 2), (2, 3, 4)]
        st, ts, rk, lb, og = run([a, b, c], labels, [0, 3, 4], [1, 1, 0])
        assert st == "OK" and ts == [a.handle.value, b.handle.value, c.handle.value]
        assert rk == [2, 2, 3] and lb == [0, 1, 1, 2, 2, 3, 4] and og == [0, 1, 2]
        st, ts, rk, lb, og = run([c, d], [(0, 1, 2), (1, 2, 3)], [0, 3], None)   # rank 3 only
        assert st == "OK" and og == [0, 1] and lb == [0, 1, 2, 1, 2, 3]
        st, ts, rk, lb, og = run([a, b], [(0, 1), (1, 2)], [0, 2], [0, 0], max_rank=3)
        assert st == "INVALID_ARG" and ts == []
        st, *_ = run([a, b], [(0, 1), (1, 2)], [0, 2], [0, 0], max_rank=-1)
        assert st == "INVALID_ARG"
        st, *_ = run([a, b], [(0, 1), (1, 2)], [0, 2], [0, 0], max_rank=0)       # rank-0 tensors only
        assert st == "OK"
    finally:
        for t in (a, b, c, d):
            t.destroy()
