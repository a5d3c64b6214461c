"""rosnet_tensordot_noalloc: the tensordot for callers that cannot allocate
device memory at the call (e.g. code inside a framework that owns all device
memory, or with a fixed memory budget).  Its kernels' scratch lives in the
library's fixed device array.

Checked through the C ABI against rosnet_tensordot on the same inputs and
against the CPU oracle, within the tolerances of the other parity tests, on
two calls in a row (the array keeps the previous call's contents), with the
library's own count of device allocation requests unchanged across the calls.
The cases run one after another with different shapes, so every branch that
keeps operands in the array (split-K partials, packed FP32 operands, packed
tensor-core operands) follows a call that left other data there.  This file
is named to be collected last.
"""

import numpy as np
import pytest

import oracle
import paper_2201_06620_b300 as R
import workloads as W

pytestmark = pytest.mark.gpu

NPT = {R.C64: np.complex64, R.C128: np.complex128}
R_SCRATCH = 4 << 20


def _rel(x, y):
    d = np.linalg.norm((x.astype(np.complex128) - y.astype(np.complex128)).ravel())
    n = np.linalg.norm(y.astype(np.complex128).ravel())
    return d / n if n else d


def _cases():
    """(a, block_a, b, block_b, axes_a, axes_b, dtype, precision, flags, tol vs oracle)."""
    prob = W.tensordot_single_config()
    yield (prob["a"], prob["block_a"], prob["b"], prob["block_b"], prob["axes_a"],
           prob["axes_b"], R.C128, R.PREC_DEFAULT, 0, 1e-12)
    a = W.complex_normal((64, 4096), 41)       # split-K: partial sums in the scratch
    b = W.complex_normal((4096, 64), 42)
    yield a, None, b, None, [1], [0], R.C64, R.PREC_DEFAULT, 0, 1e-5
    # packed FP32 (pack pass + TMA-fed FFMA GEMM): 121 tiles of 64 x 64, the
    # packed operands (1.4 MB) in the scratch after the partials above
    a = W.complex_normal((704, 128), 47)
    b = W.complex_normal((128, 704), 48)
    yield a, None, b, None, [1], [0], R.C64, R.PREC_DEFAULT, 0, 1e-5
    # tensor cores: packed split operands in the scratch, over the previous
    # call's packed FP32 panels
    a = W.complex_normal((256, 8, 16), 49)
    b = W.complex_normal((16, 8, 256), 50)
    yield a, None, b, None, [1, 2], [1, 0], R.C64, R.PREC_TF32X3, 0, 1e-5
    yield a, None, b, None, [1, 2], [1, 0], R.C64, R.PREC_BF16X3, 0, 1e-4
    # few columns and a long contraction: 128 x 16 tiles with the contraction
    # split over CTAs, the partial results (1 MB) in the scratch after the
    # tensor-core panels
    a = W.complex_normal((2048, 256), 53)
    b = W.complex_normal((2048, 16), 54)
    yield a, None, b, None, [0], [0], R.C64, R.PREC_DEFAULT, 0, 1e-5
    a = W.complex_normal((257, 130), 43)       # ragged 128x64 tiles
    b = W.complex_normal((130, 515), 44)
    yield a, None, b, None, [1], [0], R.C64, R.PREC_DEFAULT, 0, 1e-5
    # the reduction modes of Sec. IV-A: stored partials summed in a fixed
    # order, and order-free adds into a zeroed C
    a = W.complex_normal((96, 2048), 51)
    b = W.complex_normal((2048, 80), 52)
    yield a, None, b, None, [1], [0], R.C64, R.PREC_DEFAULT, R.REDUCE_TREE, 1e-5
    yield a, None, b, None, [1], [0], R.C64, R.PREC_DEFAULT, R.REDUCE_COMMUTATIVE, 1e-5
    a = W.complex_normal((3, 5, 2), 45)        # thread-per-output kernel
    b = W.complex_normal((2, 5, 7), 46)
    yield a, None, b, None, [1, 2], [1, 0], R.C128, R.PREC_DEFAULT, 0, 1e-12


def test_noalloc_matches_tensordot_two_calls_in_a_row():
    R._init()
    for a, ba, b, bb, ax_a, ax_b, dt, prec, flags, tol in _cases():
        A = R.btensor(a.astype(NPT[dt]), ba, dt)
        B = R.btensor(b.astype(NPT[dt]), bb, dt)
        ref_t = R.tensordot(A, B, ax_a, ax_b, precision=prec, flags=flags)
        ref = ref_t.download()
        exact = oracle.tensordot(a.astype(NPT[dt]), b.astype(NPT[dt]), ax_a, ax_b)
        C1 = R.empty(ref_t.shape, ref_t.block_shape, dt)
        C2 = R.empty(ref_t.shape, ref_t.block_shape, dt)
        R.sync()
        before = R.alloc_stats()[0]
        R.tensordot_noalloc(A, B, ax_a, ax_b, C1, precision=prec, flags=flags)
        R.tensordot_noalloc(A, B, ax_a, ax_b, C2, precision=prec, flags=flags)
        R.sync()
        assert R.alloc_stats()[0] == before, "rosnet_tensordot_noalloc asked the allocator for memory"
        first, second = C1.download(), C2.download()
        assert first.shape == ref.shape
        # the same kernels as rosnet_tensordot
        same = 1e-12 if dt == R.C128 else 1e-6
        assert _rel(first, ref) <= same, (prec, flags)
        assert _rel(second, ref) <= same, (prec, flags)
        assert oracle.rel_frobenius(first, exact) <= tol, (prec, flags, oracle.rel_frobenius(first, exact))
        assert oracle.rel_frobenius(second, exact) <= tol, (prec, flags)


def test_noalloc_rejects_oversized_and_mismatched():
    R._init()
    # offset tables alone exceed the fixed scratch (2*(2^19+5+3) int64 > 4 MiB;
    # 3 contracted indices keep it off the table-free gate kernel)
    A = R.btensor(np.ones((1 << 19, 3), dtype=np.complex64))
    B = R.btensor(np.ones((3, 5), dtype=np.complex64))
    C = R.empty((1 << 19, 5), None, R.C64)
    with pytest.raises(R.RosnetError) as e:
        R.tensordot_noalloc(A, B, [1], [0], C)
    assert e.value.name == "UNSUPPORTED"
    msg = R.lib().rosnet_last_error().decode()
    assert "scratch" in msg and str(R_SCRATCH) in msg
    # wrong output shape / dtype
    A2 = R.btensor(W.complex_normal((4, 6), 1).astype(np.complex64))
    B2 = R.btensor(W.complex_normal((6, 3), 2).astype(np.complex64))
    with pytest.raises(R.RosnetError) as e:
        R.tensordot_noalloc(A2, B2, [1], [0], R.empty((4, 4), None, R.C64))
    assert e.value.name == "SHAPE"
    with pytest.raises(R.RosnetError) as e:
        R.tensordot_noalloc(A2, B2, [1], [0], R.empty((4, 3), None, R.C128))
    assert e.value.name == "DTYPE"
    # autotuning needs buffers of its own
    with pytest.raises(R.RosnetError) as e:
        R.tensordot_noalloc(A2, B2, [1], [0], R.empty((4, 3), None, R.C64), flags=R.OPT_AUTOTUNE)
    assert e.value.name == "UNSUPPORTED"
    # an output that is a view of an operand's storage (another data pointer)
    X = R.btensor(W.complex_normal((2, 4, 4), 3).astype(np.complex64))
    A3 = X.fix([0], [1])
    B3 = R.btensor(W.complex_normal((4, 4), 4).astype(np.complex64))
    with pytest.raises(R.RosnetError) as e:
        R.tensordot_noalloc(A3, B3, [1], [0], X.fix([0], [0]))
    assert e.value.name == "INVALID_ARG"
    R.sync()
