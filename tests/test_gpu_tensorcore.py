"""GPU parity of the tcgen05 tensor-core precision modes against the
complex128 oracle.

Error model for complex64 inputs of unit scale (relative Frobenius error):
  * operand rounding: TF32 keeps 11 significant bits (about 2^-11 per
    operand; 2.9e-4 measured), TF32X3 big + small keep ~22 bits, BF16X3
    hi + lo keep ~16 bits (4.4e-6 measured);
  * accumulation: the tensor core's FP32 accumulator adds with a small
    one-sided error that grows linearly with the number of terms (measured
    ~1.4e-8 * K for TF32X3 with one accumulator over all of K); the kernel
    therefore accumulates at most 256 contracted indices per TMEM chunk and
    sums the chunks in FP32 registers, which keeps the error flat in K
    (3.6e-6 for TF32X3, 4.7e-6 for BF16X3 measured for K = 32 .. 32768).
Bounds: TF32 1e-3; TF32X3 and BF16X3 1e-5, the bar of FP32-class paths.
"""
import numpy as np
import pytest

import oracle
import paper_2201_06620_b300 as R
import workloads as W

pytestmark = pytest.mark.gpu

MODES = [R.PREC_TF32, R.PREC_TF32X3, R.PREC_BF16X3]


def bound(prec, K):
    return 1e-3 if prec == R.PREC_TF32 else 1e-5


def run(a, ba, b, bb, ax_a, ax_b, prec):
    A = R.btensor(a.astype(np.complex64), ba)
    B = R.btensor(b.astype(np.complex64), bb)
    C = R.tensordot(A, B, ax_a, ax_b, precision=prec)
    got = C.download()
    R.sync()   # raises ROSNET_ERR_TIMEOUT if a bounded device wait gave up
    ref = oracle.tensordot(a.astype(np.complex64), b.astype(np.complex64), ax_a, ax_b)
    return oracle.rel_frobenius(got, ref)


@pytest.mark.parametrize("prec", MODES)
@pytest.mark.parametrize("mnk", [(128, 128, 32), (200, 130, 100), (64, 300, 47), (513, 257, 1031),
                                 (1024, 1024, 256), (300, 129, 9001)])
def test_matrix_shapes(prec, mnk):
    M, N, K = mnk
    err = run(W.complex_normal((M, K), 1), None, W.complex_normal((K, N), 2), None, [1], [0], prec)
    assert err <= bound(prec, K), err


@pytest.mark.parametrize("prec", MODES)
def test_blocked_permuted_qubit_tensors(prec):
    """[2]^r operands with permuted axes and block grids (any layout goes
    through the tensor-core path's offset-table gather)."""
    for trial in range(4):
        prob = W._block_tensordot_problem(60 + trial, 70 + trial, 8, 7, 8, 2, 3, 1, perm_seed=80 + trial)
        err = run(prob["a"], prob["block_a"], prob["b"], prob["block_b"], prob["axes_a"],
                  prob["axes_b"], prec)
        assert err <= bound(prec, 2 ** 7), (trial, err)


def test_single_config_all_modes_ordering():
    """On the [2]^14 x [2]^14 single-contraction workload (complex64) the
    error ordering follows the number of bits kept: tf32 > bf16x3 > tf32x3."""
    prob = W.tensordot_single_config()
    errs = {p: run(prob["a"], prob["block_a"], prob["b"], prob["block_b"], prob["axes_a"],
                   prob["axes_b"], p) for p in MODES}
    assert errs[R.PREC_TF32] > errs[R.PREC_BF16X3] > errs[R.PREC_TF32X3]
