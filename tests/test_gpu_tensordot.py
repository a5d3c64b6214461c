"""GPU parity of rosnet_tensordot against the complex128 CPU oracle.

Tolerances (relative Frobenius error ||C - C_ref|| / ||C_ref||): 1e-12 for the
complex128 / FP64 path and 1e-5 for the complex64 / FP32 path.  Inputs are
seeded; for complex64 the oracle runs on the same (rounded) complex64 values.
"""
import numpy as np
import pytest

import oracle
import paper_2201_06620_b300 as R
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {R.C64: 1e-5, R.C128: 1e-12}
NPT = {R.C64: np.complex64, R.C128: np.complex128}


def run(a, ba, b, bb, ax_a, ax_b, dtype, precision=R.PREC_DEFAULT):
    A = R.btensor(a.astype(NPT[dtype]), ba, dtype)
    B = R.btensor(b.astype(NPT[dtype]), bb, dtype)
    C = R.tensordot(A, B, ax_a, ax_b, precision=precision)
    return C, C.download()


def ref_of(a, b, ax_a, ax_b, dtype):
    return oracle.tensordot(a.astype(NPT[dtype]), b.astype(NPT[dtype]), ax_a, ax_b)


@pytest.mark.parametrize("gc", [0, 2, 6])
def test_single_blocked_tensordot_fp64(gc):
    """[2]^14 x [2]^14 complex128 in blocks of 2^10, 6 contracted axes, B_k = 2^gc."""
    prob = W.tensordot_single_config(grid_contracted=gc)
    C, got = run(prob["a"], prob["block_a"], prob["b"], prob["block_b"], prob["axes_a"],
                 prob["axes_b"], R.C128)
    ref = oracle.tensordot(prob["a"], prob["b"], prob["axes_a"], prob["axes_b"])
    assert got.shape == (2,) * 16 and C.block_shape == tuple(
        [prob["block_a"][i] for i in range(14) if i not in prob["axes_a"]] +
        [prob["block_b"][i] for i in range(14) if i not in prob["axes_b"]])
    assert oracle.rel_frobenius(got, ref) <= 1e-12


def test_single_blocked_tensordot_c64():
    prob = W.tensordot_single_config()
    _, got = run(prob["a"], prob["block_a"], prob["b"], prob["block_b"], prob["axes_a"],
                 prob["axes_b"], R.C64)
    ref = ref_of(prob["a"], prob["b"], prob["axes_a"], prob["axes_b"], R.C64)
    assert oracle.rel_frobenius(got, ref) <= 1e-5


def _random_problem(rng, max_rank=5, max_ext=6, min_k=0):
    while True:
        nk = int(rng.integers(min_k, 3))
        nfa = int(rng.integers(0, 3))
        nfb = int(rng.integers(0, 3))
        kext = [int(rng.integers(1, max_ext + 1)) for _ in range(nk)]
        fa = [int(rng.integers(1, max_ext + 1)) for _ in range(nfa)]
        fb = [int(rng.integers(1, max_ext + 1)) for _ in range(nfb)]
        if nfa + nk <= max_rank and nfb + nk <= max_rank:
            break
    pa = rng.permutation(nfa + nk)
    pb = rng.permutation(nfb + nk)
    la = [("f", i) for i in range(nfa)] + [("k", i) for i in range(nk)]
    lb = [("k", i) for i in range(nk)] + [("g", i) for i in range(nfb)]
    la = [la[i] for i in pa]
    lb = [lb[i] for i in pb]
    ext = lambda t: fa[t[1]] if t[0] == "f" else (fb[t[1]] if t[0] == "g" else kext[t[1]])
    sa = tuple(ext(t) for t in la)
    sb = tuple(ext(t) for t in lb)
    ax_a = [la.index(("k", i)) for i in range(nk)]
    ax_b = [lb.index(("k", i)) for i in range(nk)]

    def divisor(s):
        ds = [d for d in range(1, s + 1) if s % d == 0]
        return int(rng.choice(ds))
    ba = [divisor(s) for s in sa]
    bb = [divisor(s) for s in sb]
    for i, j in zip(ax_a, ax_b):
        bb[j] = ba[i]
    return sa, sb, ax_a, ax_b, tuple(ba), tuple(bb)


@pytest.mark.parametrize("dtype", [R.C64, R.C128])
def test_random_permutations_and_blockings(dtype):
    rng = np.random.default_rng(77)
    for trial in range(60):
        sa, sb, ax_a, ax_b, ba, bb = _random_problem(rng)
        a = W.complex_normal(sa, 1000 + trial)
        b = W.complex_normal(sb, 2000 + trial)
        _, got = run(a, ba, b, bb, ax_a, ax_b, dtype)
        ref = ref_of(a, b, ax_a, ax_b, dtype)
        assert got.shape == ref.shape
        err = oracle.rel_frobenius(got, ref) if ref.size and np.any(ref) else np.abs(got).max(initial=0)
        assert err <= TOL[dtype], (trial, sa, sb, ax_a, ax_b, ba, bb, err)


@pytest.mark.parametrize("dtype", [R.C64, R.C128])
@pytest.mark.parametrize("mnk", [(130, 70, 37), (64, 64, 16), (65, 33, 17), (200, 3, 300),
                                 (1, 1, 5000), (7, 300, 200), (31, 500, 129), (129, 257, 1),
                                 (64, 64, 4096), (20, 300, 3001), (300, 20, 2999), (257, 130, 515),
                                 (7, 30, 3000), (16, 16, 2048)])
def test_tiles_and_ragged_tails(dtype, mnk):
    """Matrix-shaped problems that span several tiles with ragged edges and
    exercise each kernel family (tiled 128x64 / 64x64, split-K with its
    reduction, CTA-per-output, warp-per-output, thread-per-output)."""
    M, N, K = mnk
    a = W.complex_normal((M, K), 11)
    b = W.complex_normal((K, N), 12)
    _, got = run(a, None, b, None, [1], [0], dtype)
    ref = ref_of(a, b, [1], [0], dtype)
    assert oracle.rel_frobenius(got, ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [R.C64, R.C128])
@pytest.mark.parametrize("mnk", [(2048, 512, 32), (1000, 70, 8), (130, 200, 17), (64, 64, 31), (3000, 20, 9)])
def test_short_contractions_direct(dtype, mnk):
    """K of 8..32: whole tiles gathered in one pass (direct kernel), ragged."""
    M, N, K = mnk
    a = W.complex_normal((M, K), 15)
    b = W.complex_normal((K, N), 16)
    _, got = run(a, None, b, None, [1], [0], dtype)
    assert oracle.rel_frobenius(got, ref_of(a, b, [1], [0], dtype)) <= TOL[dtype]


@pytest.mark.parametrize("mnk", [(300, 13, 200), (513, 16, 4000), (16, 700, 333), (200, 30, 300),
                                 (130, 29, 2000), (1000, 17, 64)])
def test_narrow_tiles(mnk):
    """Few-column problems take the 256x16 / 128x32 tiles (with and without a
    contracted-range split); ragged in every dimension."""
    M, N, K = mnk
    a = W.complex_normal((M, K), 13)
    b = W.complex_normal((K, N), 14)
    A, B = R.btensor(a.astype(np.complex64)), R.btensor(b.astype(np.complex64))
    ref = ref_of(a, b, [1], [0], R.C64)
    for flags in (0, R.REDUCE_TREE, R.REDUCE_COMMUTATIVE):
        got = R.tensordot(A, B, [1], [0], flags=flags).download()
        assert oracle.rel_frobenius(got, ref) <= 1e-5, flags


@pytest.mark.parametrize("dtype", [R.C64, R.C128])
def test_qubit_tensors_permuted_blocked(dtype):
    """[2]^r tensors with seeded axis permutations and mixed grid/intra axes."""
    rng = np.random.default_rng(5)
    for trial in range(12):
        nk, nfa, nfb = int(rng.integers(1, 7)), int(rng.integers(0, 8)), int(rng.integers(0, 8))
        prob = W._block_tensordot_problem(10 + trial, 20 + trial, nfa, nk, nfb,
                                          int(rng.integers(0, nfa + 1)), int(rng.integers(0, nk + 1)),
                                          int(rng.integers(0, nfb + 1)), perm_seed=100 + trial)
        _, got = run(prob["a"], prob["block_a"], prob["b"], prob["block_b"], prob["axes_a"],
                     prob["axes_b"], dtype)
        ref = ref_of(prob["a"], prob["b"], prob["axes_a"], prob["axes_b"], dtype)
        assert oracle.rel_frobenius(got, ref) <= TOL[dtype], trial


def test_high_rank_and_large_output():
    """Rank-22 operand, rank-24 output (more than 16 index digits per class)."""
    a = W.complex_normal((2,) * 22, 31).astype(np.complex64)
    b = W.complex_normal((2,) * 4, 32).astype(np.complex64)
    ba = (1,) * 10 + (2,) * 12
    _, got = run(a, ba, b, (2, 1, 2, 1), [21, 3], [2, 1], R.C64)
    ref = ref_of(a, b, [21, 3], [2, 1], R.C64)
    assert got.shape == (2,) * 22
    assert oracle.rel_frobenius(got, ref) <= 1e-5


def test_outer_product_scalar_and_degenerate():
    a = W.complex_normal((3, 4), 1)
    b = W.complex_normal((5,), 2)
    _, got = run(a, None, b, None, [], [], R.C128)
    np.testing.assert_allclose(got, np.multiply.outer(a, b), rtol=1e-13, atol=1e-13)
    # full contraction: rank-0 result
    c = W.complex_normal((3, 4), 3)
    C, got = run(a, (1, 2), c, (1, 2), [0, 1], [0, 1], R.C128)
    assert C.shape == () and got.shape == ()
    assert abs(got - np.sum(a * c)) <= 1e-12 * abs(np.sum(a * c))
    # rank-0 operands
    s = np.array(2.0 - 1.0j)
    _, got = run(s, (), a, None, [], [], R.C128)
    np.testing.assert_allclose(got, s * a, rtol=1e-14)
    # extent-0 free axis: empty result; extent-0 contracted axis: zeros
    z = np.zeros((0, 3), dtype=np.complex128)
    _, got = run(z, None, W.complex_normal((3, 2), 4), None, [1], [0], R.C128)
    assert got.shape == (0, 2)
    _, got = run(np.zeros((4, 0)), None, np.zeros((0, 5)), None, [1], [0], R.C128)
    assert got.shape == (4, 5) and not np.any(got)


def test_negative_axes_like_numpy():
    a = W.complex_normal((3, 4, 5), 6)
    b = W.complex_normal((5, 4), 7)
    _, got = run(a, None, b, None, [-1, -2], [0, 1], R.C128)
    np.testing.assert_allclose(got, np.tensordot(a, b, axes=([2, 1], [0, 1])), rtol=1e-12, atol=1e-12)


def test_upload_download_roundtrip_blocked():
    rng = np.random.default_rng(3)
    for dtype in (R.C64, R.C128):
        for shape, block in [((4, 6, 2), (2, 3, 1)), ((2,) * 10, (1, 2) * 5), ((7,), (7,)), ((), ())]:
            x = W.complex_normal(shape, int(rng.integers(1 << 30))).astype(NPT[dtype])
            t = R.btensor(x, block, dtype)
            assert np.array_equal(t.download(), x)


def test_raw_storage_copies():
    """upload_raw / download_raw move the planar storage (real plane, then
    imaginary plane, block-major order) with one copy; they agree with the
    regular (interleaved, any layout) copies and refuse views."""
    import torch
    for dtype in (R.C64, R.C128):
        real = np.float32 if dtype == R.C64 else np.float64
        x = W.complex_normal((6, 4), 81).astype(NPT[dtype])
        t = R.btensor(x, None, dtype)                   # one block: row-major storage
        raw = np.zeros(2 * x.size, dtype=real)
        t.download_raw(raw)
        R.sync()
        assert np.array_equal(raw[:x.size], x.real.ravel()) and np.array_equal(raw[x.size:], x.imag.ravel())
        y = W.complex_normal((6, 4), 82).astype(NPT[dtype])
        host = torch.from_numpy(np.concatenate([y.real.ravel(), y.imag.ravel()]).astype(real)).pin_memory()
        t.upload_raw(host)
        assert np.array_equal(t.download(), y)
        # the result of a tensordot, read raw, equals its regular download
        c = R.tensordot(t, R.btensor(x.T.copy(), None, dtype), [1], [0])
        out = np.zeros(2 * c.numel, dtype=real)
        c.download_raw(out)
        R.sync()
        ref = c.download()
        assert np.array_equal(out[:c.numel] + 1j * out[c.numel:].astype(np.complex128), ref.ravel())
        with pytest.raises(R.RosnetError) as e:
            t.fix([0], [1]).download_raw(np.zeros(8, dtype=real))
        assert e.value.name == "UNSUPPORTED"
        with pytest.raises(ValueError):
            t.upload_raw(np.zeros(3, dtype=real))


def test_error_codes():
    a = R.btensor(W.complex_normal((4, 4), 1), (2, 2), R.C128)
    b = R.btensor(W.complex_normal((4, 4), 2), (4, 2), R.C128)
    c = R.btensor(W.complex_normal((3, 4), 3), None, R.C128)
    d = R.btensor(W.complex_normal((4, 4), 4).astype(np.complex64), None, R.C64)
    cases = [
        (lambda: R.tensordot(a, b, [1], [0]), "BLOCK_MISMATCH"),
        (lambda: R.tensordot(a, c, [1], [0]), "SHAPE"),
        (lambda: R.tensordot(a, d, [1], [0]), "DTYPE"),
        (lambda: R.tensordot(a, a, [2], [0]), "INVALID_ARG"),
        (lambda: R.tensordot(a, a, [0, 0], [0, 1]), "INVALID_ARG"),
        (lambda: R.tensordot(d, d, [1], [0], precision=R.PREC_FP64), "UNSUPPORTED"),
        (lambda: R.tensordot(a, a, [1], [0], precision=R.PREC_FP32), "UNSUPPORTED"),
        (lambda: R.empty((4,), (3,)), "BLOCK_MISMATCH"),
    ]
    for fn, name in cases:
        with pytest.raises(R.RosnetError) as e:
            fn()
        assert e.value.name == name


def test_fp32_mode_equals_default_c64():
    prob = W.tensordot_single_config()
    A = R.btensor(prob["a"].astype(np.complex64), prob["block_a"])
    B = R.btensor(prob["b"].astype(np.complex64), prob["block_b"])
    c0 = R.tensordot(A, B, prob["axes_a"], prob["axes_b"]).download()
    c1 = R.tensordot(A, B, prob["axes_a"], prob["axes_b"], precision=R.PREC_FP32).download()
    assert np.array_equal(c0, c1)


@pytest.mark.parametrize("dtype", [R.C64, R.C128])
@pytest.mark.parametrize("mode", [R.REDUCE_SEQUENTIAL, R.REDUCE_TREE, R.REDUCE_COMMUTATIVE])
def test_reduction_modes(dtype, mode):
    """Sec. IV-A's three ways of summing the B_k block-pair partials: one CTA
    over all pairs, split with a stored-partials tree, split with order-free
    adds.  All agree with the oracle; sequential and tree are bitwise
    reproducible."""
    prob = W._block_tensordot_problem(90, 91, 7, 9, 7, 3, 5, 2, perm_seed=92)   # B_k = 32
    A = R.btensor(prob["a"].astype(NPT[dtype]), prob["block_a"], dtype)
    B = R.btensor(prob["b"].astype(NPT[dtype]), prob["block_b"], dtype)
    ref = ref_of(prob["a"], prob["b"], prob["axes_a"], prob["axes_b"], dtype)
    c1 = R.tensordot(A, B, prob["axes_a"], prob["axes_b"], flags=mode).download()
    c2 = R.tensordot(A, B, prob["axes_a"], prob["axes_b"], flags=mode).download()
    assert oracle.rel_frobenius(c1, ref) <= TOL[dtype]
    assert oracle.rel_frobenius(c2, ref) <= TOL[dtype]
    if mode != R.REDUCE_COMMUTATIVE:
        assert np.array_equal(c1, c2)


def test_reduction_modes_matrix_ragged():
    a = W.complex_normal((70, 3001), 5)
    b = W.complex_normal((3001, 90), 6)
    ref = ref_of(a, b, [1], [0], R.C64)
    A, B = R.btensor(a.astype(np.complex64)), R.btensor(b.astype(np.complex64))
    for mode in (R.REDUCE_SEQUENTIAL, R.REDUCE_TREE, R.REDUCE_COMMUTATIVE):
        got = R.tensordot(A, B, [1], [0], flags=mode).download()
        assert oracle.rel_frobenius(got, ref) <= 1e-5, mode
    with pytest.raises(R.RosnetError):
        R.tensordot(A, B, [1], [0], flags=R.REDUCE_TREE | R.REDUCE_COMMUTATIVE)


def test_bounded_wait_reports_timeout_and_context_survives():
    """A kernel waiting on a barrier that nothing completes gives up after its
    budget (~1 ms here) and rosnet_sync reports ROSNET_ERR_TIMEOUT; the status
    is cleared and later work runs normally."""
    R._init()
    assert R.lib().rosnet_selftest_timeout(2_000_000, R._default_stream()) == 0
    with pytest.raises(R.RosnetError) as e:
        R.sync()
    assert e.value.name == "TIMEOUT"
    R.sync()   # cleared
    a = W.complex_normal((3, 4), 1)
    _, got = run(a, None, a.T.copy(), None, [1], [0], R.C128)
    np.testing.assert_allclose(got, a @ a.T, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dtype", [R.C64, R.C128])
@pytest.mark.parametrize("mnk", [(1, 1, 1024), (1, 1, 4096), (16, 16, 2000), (2, 3, 4097), (1, 1, 70001)])
def test_long_contractions_into_few_entries(dtype, mnk):
    """Outputs of at most 256 entries over K >= 1024 (a network's final
    scalar): a cluster of CTAs per entry, products and sums in FP64, the
    result rounded once to C's type, the same bits on every call."""
    M, N, K = mnk
    npt = np.complex64 if dtype == R.C64 else np.complex128
    a = W.complex_normal((M, K), 61).astype(npt)
    b = W.complex_normal((K, N), 62).astype(npt)
    A, B = R.btensor(a, None, dtype), R.btensor(b, None, dtype)
    got = R.tensordot(A, B, [1], [0]).download()
    ref = oracle.tensordot(a, b, [1], [0])
    # FP64 accumulation: the error is the operands' own rounding (none) and
    # the final rounding to C's type, far below the FP32 bar
    tol = 1e-7 if dtype == R.C64 else 1e-12
    assert oracle.rel_frobenius(got, ref) <= tol
    assert np.array_equal(got, R.tensordot(A, B, [1], [0]).download())
