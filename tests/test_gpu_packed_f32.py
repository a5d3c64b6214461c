"""GPU parity of the packed FP32 path (TMA-fed FFMA tiles; an operand stored
as a dense K x rows matrix is read in place, any other is first gathered once
into a dense panel) against the complex128 CPU oracle.

Large complex64 contractions at the default (plain FP32) precision take this
path; the bar is the FP32 one, relative Frobenius error <= 1e-5.  Shapes span
many 64 x 64 output tiles with ragged M, N and K edges; blocked [2]^r tensors
with seeded axis permutations put either the row or the contracted index on
each operand's unit stride, and exchange the operands' roles.
"""
import numpy as np
import pytest

import oracle
import paper_2201_06620_b300 as R
import workloads as W

pytestmark = pytest.mark.gpu


def _launches(fn):
    before = R.kernel_launches()
    out = fn()
    R.sync()
    return out, R.kernel_launches() - before


def _tiled_launches():
    """Launches of a small contraction that takes the single-kernel path."""
    a = R.btensor(W.complex_normal((100, 50), 1).astype(np.complex64))
    b = R.btensor(W.complex_normal((50, 60), 2).astype(np.complex64))
    return _launches(lambda: R.tensordot(a, b, [1], [0]))[1]


@pytest.mark.parametrize("mnk", [(1000, 700, 200), (4096, 256, 256), (300, 2000, 333), (1280, 448, 1500)])
def test_matrix_shapes_ragged(mnk):
    M, N, K = mnk
    a = W.complex_normal((M, K), 41).astype(np.complex64)
    b = W.complex_normal((K, N), 42).astype(np.complex64)
    A, B = R.btensor(a), R.btensor(b)
    C, n = _launches(lambda: R.tensordot(A, B, [1], [0]))
    assert n == _tiled_launches() + 1, n   # one pack launch (both operands) + GEMM instead of one kernel
    ref = oracle.tensordot(a, b, [1], [0])
    assert oracle.rel_frobenius(C.download(), ref) <= 1e-5


@pytest.mark.parametrize("trial", range(6))
def test_blocked_permuted_qubit_tensors(trial):
    """2^11 x 2^9 outputs over 2^7 contracted indices (B_k > 1): the gather
    goes through block-major layouts with permuted axes."""
    rng = np.random.default_rng(300 + trial)
    nfa, nk, nfb = (11, 7, 9) if trial % 2 == 0 else (9, 7, 11)
    prob = W._block_tensordot_problem(400 + trial, 500 + trial, nfa, nk, nfb,
                                      int(rng.integers(0, nfa + 1)), int(rng.integers(1, nk + 1)),
                                      int(rng.integers(0, nfb + 1)), perm_seed=600 + trial)
    a, b = prob["a"].astype(np.complex64), prob["b"].astype(np.complex64)
    A = R.btensor(a, prob["block_a"])
    B = R.btensor(b, prob["block_b"])
    C, n = _launches(lambda: R.tensordot(A, B, prob["axes_a"], prob["axes_b"]))
    assert n in (_tiled_launches(), _tiled_launches() + 1), n   # GEMM, after a pack unless both are dense
    ref = oracle.tensordot(a, b, prob["axes_a"], prob["axes_b"])
    assert oracle.rel_frobenius(C.download(), ref) <= 1e-5, trial


def test_deterministic_and_sequential_mode():
    """240 output tiles of a 1100-long contraction on 296 CTA slots: the
    automatic choice is the stream-K schedule (pieces of a tile summed in a
    fixed order), bitwise reproducible; the sequential mode runs one CTA per
    tile over the whole contraction.  Both meet the bar."""
    a = W.complex_normal((1000, 1100), 51).astype(np.complex64)
    b = W.complex_normal((1100, 900), 52).astype(np.complex64)
    A, B = R.btensor(a), R.btensor(b)
    ref = oracle.tensordot(a, b, [1], [0])
    c1 = R.tensordot(A, B, [1], [0]).download()
    for _ in range(3):
        assert np.array_equal(c1, R.tensordot(A, B, [1], [0]).download())
    c3 = R.tensordot(A, B, [1], [0], flags=R.REDUCE_SEQUENTIAL).download()
    assert np.array_equal(c3, R.tensordot(A, B, [1], [0], flags=R.REDUCE_SEQUENTIAL).download())
    assert oracle.rel_frobenius(c1, ref) <= 1e-5
    assert oracle.rel_frobenius(c3, ref) <= 1e-5


@pytest.mark.parametrize("mnk", [(704, 704, 1024), (768, 640, 2048), (1000, 700, 1100), (2500, 600, 1333)])
def test_stream_k_tile_pieces(mnk):
    """Deep contractions whose tiles fill the CTA slots poorly take the
    stream-K schedule: tiles split into pieces over CTAs (up to several per
    tile, ragged K), summed by whichever CTA stores the last piece; repeated in
    a plan replayed as a graph (the per-tile counters return to zero)."""
    M, N, K = mnk
    a = W.complex_normal((K, M), 71).astype(np.complex64)
    b = W.complex_normal((K, N), 72).astype(np.complex64)
    ref = oracle.tensordot(a, b, [0], [0])
    A, B = R.btensor(a), R.btensor(b)
    C = R.tensordot(A, B, [0], [0]).download()
    assert oracle.rel_frobenius(C, ref) <= 1e-5
    outs = [R.contract([A, B], [(0, 1), (0, 2)], [1, 2], [(0, 1)], flags=R.OPT_GRAPH).download()
            for _ in range(3)]
    for o in outs:
        assert np.array_equal(o, C)


# Operands stored as dense K x rows matrices are read in place by the GEMM's
# tensor maps (no pack launch); the others are packed.  (a layout, b layout,
# axes, pack launches expected): "km" = (K, M) storage, "mk" = (M, K).
@pytest.mark.parametrize("mnk", [(1000, 700, 200), (4096, 256, 256), (1024, 520, 131)])
@pytest.mark.parametrize("la,lb,packs", [("km", "kn", 0), ("km", "nk", 1), ("mk", "kn", 1), ("mk", "nk", 1)])
def test_dense_operands_read_in_place(mnk, la, lb, packs):
    M, N, K = mnk
    a = W.complex_normal((K, M) if la == "km" else (M, K), 61).astype(np.complex64)
    b = W.complex_normal((K, N) if lb == "kn" else (N, K), 62).astype(np.complex64)
    ax_a = [0] if la == "km" else [1]
    ax_b = [0] if lb == "kn" else [1]
    A, B = R.btensor(a), R.btensor(b)
    C, n = _launches(lambda: R.tensordot(A, B, ax_a, ax_b))
    assert n == _tiled_launches() + packs, (n, packs)
    ref = oracle.tensordot(a, b, ax_a, ax_b)
    assert oracle.rel_frobenius(C.download(), ref) <= 1e-5


def test_dense_operand_unaligned_rows_is_packed():
    """A dense K x 998 operand: rows of 998 floats are not a whole number of
    16-byte units, which a tensor map cannot stride over; it is packed."""
    a = W.complex_normal((256, 998), 63).astype(np.complex64)
    b = W.complex_normal((256, 640), 64).astype(np.complex64)
    A, B = R.btensor(a), R.btensor(b)
    C, n = _launches(lambda: R.tensordot(A, B, [0], [0]))
    assert n == _tiled_launches() + 1, n
    assert oracle.rel_frobenius(C.download(), oracle.tensordot(a, b, [0], [0])) <= 1e-5


# Few columns and a long contraction: 128 x 16 tiles with the contraction
# split over CTAs, each storing a partial result that a second kernel sums in
# split order.  (M, N, K): the amplitude's 256 x 16 x 4096 step, ragged rows
# and contraction, 3 columns (a B panel of 3 rows is not 16-byte aligned:
# packed), several row tiles, a single column, 130 rows (a second row tile
# of 2, rows not 16-byte aligned: A packed) over a 32768-long contraction
# split 64 ways, and 313 row tiles (enough CTAs unsplit: C staged through
# shared memory by the four k sets).
@pytest.mark.parametrize("mnk", [(256, 16, 4096), (300, 12, 2500), (1000, 3, 3000), (2048, 16, 1024),
                                 (4096, 1, 2048), (130, 16, 32768), (40000, 8, 600)])
@pytest.mark.parametrize("la", ["km", "mk"])
def test_few_columns_split_contraction(mnk, la):
    M, N, K = mnk
    a = W.complex_normal((K, M) if la == "km" else (M, K), 91).astype(np.complex64)
    b = W.complex_normal((K, N), 92).astype(np.complex64)
    ax_a = [0] if la == "km" else [1]
    A, B = R.btensor(a), R.btensor(b)
    R.timing_drain()
    C = R.tensordot(A, B, ax_a, [0])
    ref = oracle.tensordot(a, b, ax_a, [0])
    got = C.download()
    assert oracle.rel_frobenius(got, ref) <= 1e-5
    for _ in range(2):   # fixed summation order: bitwise reproducible
        assert np.array_equal(got, R.tensordot(A, B, ax_a, [0]).download())
    # a plan replayed as a graph (the partials live in the plan's workspace)
    outs = [R.contract([A, B], [(0, 1) if la == "km" else (1, 0), (0, 2)], [1, 2], [(0, 1)],
                       flags=R.OPT_GRAPH | R.OPT_TIMING).download() for _ in range(3)]
    recs = R.timing_drain()
    assert recs and recs[-1][3] == 10, recs[-1:]
    for o in outs:
        assert np.array_equal(o, got)


def test_few_columns_sequential_mode_is_not_split():
    """REDUCE_SEQUENTIAL asks for one CTA per output tile over the whole
    contraction: the split GEMM is not taken, the result meets the bar."""
    a = W.complex_normal((4096, 256), 93).astype(np.complex64)
    b = W.complex_normal((4096, 16), 94).astype(np.complex64)
    A, B = R.btensor(a), R.btensor(b)
    ref = oracle.tensordot(a, b, [0], [0])
    R.timing_drain()
    got = R.contract([A, B], [(0, 1), (0, 2)], [1, 2], [(0, 1)],
                     flags=R.OPT_TIMING | R.REDUCE_SEQUENTIAL).download()
    recs = R.timing_drain()
    assert recs and recs[-1][3] != 10, recs[-1:]
    assert oracle.rel_frobenius(got, ref) <= 1e-5


def _random_gemm_shapes(seed, n):
    """Seeded shapes that reach each FP32 GEMM schedule: one CTA per 64 x 64
    tile, stream-K where 149-250 tiles load the SMs unevenly (one whole tile
    per SM, the rest split), and the few-column split contraction."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        kind = i % 3
        if kind == 0:      # many tiles
            M, N, K = int(rng.integers(700, 2100)), int(rng.integers(300, 700)), int(rng.integers(128, 700))
        elif kind == 1:    # 149-250 tiles of 64 x 64, deep enough to split
            M = int(rng.integers(9, 13)) * 64 + int(rng.integers(0, 64))
            N = int(rng.integers(15, 18)) * 64 - int(rng.integers(0, 64))
            K = int(rng.integers(300, 1200))
        else:              # few columns, long contraction
            M, N, K = int(rng.integers(128, 1500)), int(rng.integers(1, 17)), int(rng.integers(2048, 9000))
        out.append((M, N, K))
    return out


@pytest.mark.parametrize("seed", [0, 1])
def test_random_shapes_every_schedule(seed):
    """Random ragged shapes through the heuristic's choice and through the
    autotuner's (which also times the other schedules), both against the
    oracle; the heuristic's result is bitwise repeatable."""
    for M, N, K in _random_gemm_shapes(seed, 6):
        a = W.complex_normal((K, M), 100 + M).astype(np.complex64)
        b = W.complex_normal((K, N), 200 + N).astype(np.complex64)
        A, B = R.btensor(a), R.btensor(b)
        ref = oracle.tensordot(a, b, [0], [0])
        got = R.tensordot(A, B, [0], [0]).download()
        assert oracle.rel_frobenius(got, ref) <= 1e-5, (M, N, K)
        assert np.array_equal(got, R.tensordot(A, B, [0], [0]).download()), (M, N, K)
        tuned = R.contract([A, B], [(0, 1), (0, 2)], [1, 2], [(0, 1)], flags=R.OPT_AUTOTUNE).download()
        assert oracle.rel_frobenius(tuned, ref) <= 1e-5, (M, N, K)
    R.release_plans()
