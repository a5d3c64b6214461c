"""rosnet_tensordot_noalloc: the tensordot for callers that cannot allocate
device memory at the call (e.g. code inside a framework that owns all device
memory, or with a fixed memory budget).  Its kernels' scratch lives in the
library's fixed device array.

Checked through the C ABI against rosnet_tensordot on the same inputs, within
the tolerances of the other parity tests, on two calls in a row (the array
keeps the previous call's contents), with the library's own count of device
allocation requests unchanged across the calls.  This file is named to be
collected last.
"""

import numpy as np
import pytest

import paper_2201_06620_b300 as R
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {R.C64: 1e-5, R.C128: 1e-12}
NPT = {R.C64: np.complex64, R.C128: np.complex128}


def _rel(x, y):
    d = np.linalg.norm((x.astype(np.complex128) - y.astype(np.complex128)).ravel())
    n = np.linalg.norm(y.astype(np.complex128).ravel())
    return d / n if n else d


def _cases():
    prob = W.tensordot_single_config()
    yield (prob["a"], prob["block_a"], prob["b"], prob["block_b"], prob["axes_a"],
           prob["axes_b"], R.C128)
    a = W.complex_normal((64, 4096), 41)       # split-K: partial sums in the scratch
    b = W.complex_normal((4096, 64), 42)
    yield a, None, b, None, [1], [0], R.C64
    a = W.complex_normal((257, 130), 43)       # ragged 128x64 tiles
    b = W.complex_normal((130, 515), 44)
    yield a, None, b, None, [1], [0], R.C64
    a = W.complex_normal((3, 5, 2), 45)        # thread-per-output kernel
    b = W.complex_normal((2, 5, 7), 46)
    yield a, None, b, None, [1, 2], [1, 0], R.C128


def test_noalloc_matches_tensordot_two_calls_in_a_row():
    R._init()
    for a, ba, b, bb, ax_a, ax_b, dt in _cases():
        A = R.btensor(a.astype(NPT[dt]), ba, dt)
        B = R.btensor(b.astype(NPT[dt]), bb, dt)
        ref_t = R.tensordot(A, B, ax_a, ax_b)
        ref = ref_t.download()
        C1 = R.empty(ref_t.shape, ref_t.block_shape, dt)
        C2 = R.empty(ref_t.shape, ref_t.block_shape, dt)
        R.sync()
        before = R.alloc_stats()[0]
        R.tensordot_noalloc(A, B, ax_a, ax_b, C1)
        R.tensordot_noalloc(A, B, ax_a, ax_b, C2)
        R.sync()
        assert R.alloc_stats()[0] == before, "rosnet_tensordot_noalloc asked the allocator for memory"
        first, second = C1.download(), C2.download()
        assert first.shape == ref.shape
        assert _rel(first, ref) <= TOL[dt]
        assert _rel(second, ref) <= TOL[dt]


def test_noalloc_rejects_oversized_and_mismatched():
    R._init()
    # offset tables alone exceed the fixed scratch (2*(2^19+4+1) int64 > 4 MiB)
    A = R.btensor(np.ones((1 << 19, 1), dtype=np.complex64))
    B = R.btensor(np.ones((1, 4), dtype=np.complex64))
    C = R.empty((1 << 19, 4), None, R.C64)
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


R_SCRATCH = 4 << 20
