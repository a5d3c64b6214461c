"""Full-size parity of the precision sweep workload on sampled output blocks.

A, B: complex64 [2]^30 (8 GiB each), entries from the counter-addressable
generator times 2^-15, blocks of 2^12 (6 free + 6 contracted axes of block
extent 2 per operand, B_k = 16); C = tensordot(A, B) over the last 10 axes of
both is [2]^40 (8 TiB), produced in 2^30-entry chunks (one per value of A's
first 10 axes) streamed to pinned host memory by rosnet_tensordot_ooc -- the
launch configuration the sweep benchmark times.  For each precision mode one
chunk is computed and sampled blocks (64 x 64 entries each) are compared with
the oracle, which rebuilds exactly the A and B rows a block needs from the
same generator.
"""
import numpy as np
import pytest

import oracle
import paper_2201_06620_b300 as R
import workloads as W

pytestmark = pytest.mark.gpu

PIECE = 1 << 26
TOL = {R.PREC_FP32: 1e-5, R.PREC_TF32: 1e-3, R.PREC_TF32X3: 1e-5, R.PREC_BF16X3: 1e-5}


def _upload(t, seed, scale):
    n = t.numel
    for start in range(0, n, PIECE):
        t.upload_range(W.complex_normal_range(seed, start, min(PIECE, n - start), scale), start)


@pytest.fixture(scope="module")
def operands():
    import torch
    prob = W.precision_sweep_config()
    A = R.empty(prob["shape_a"], prob["block_a"], R.C64)
    B = R.empty(prob["shape_b"], prob["block_b"], R.C64)
    _upload(A, prob["seed_a"], prob["scale"])
    _upload(B, prob["seed_b"], prob["scale"])
    R.sync()
    chunk = 1 << 30
    host = torch.empty(2 * chunk * 4, dtype=torch.uint8).pin_memory()   # one chunk, re + im planes
    yield prob, A, B, host
    del host, A, B


def _oracle_block(prob, chunk, blk):
    """C entries of block `blk` of output chunk `chunk`: rows of A with axes
    0..9 = chunk, 10..13 = the block's A grid digits; rows of B with axes
    0..13 = the block's B grid digits; sum over axes 20..29 of both."""
    ag, bg = blk >> 14, blk & 0x3FFF
    a = W.complex_normal_range(prob["seed_a"], ((chunk << 4) | ag) << 16, 1 << 16, prob["scale"])
    b = W.complex_normal_range(prob["seed_b"], bg << 16, 1 << 16, prob["scale"])
    return oracle.tensordot(a.reshape(64, 1024), b.reshape(64, 1024), [1], [1])


@pytest.mark.parametrize("prec,chunk", [(R.PREC_FP32, 0), (R.PREC_TF32, 333),
                                        (R.PREC_TF32X3, 777), (R.PREC_BF16X3, 1023)])
def test_sweep_chunk_sampled_blocks(operands, prec, chunk):
    prob, A, B, host = operands
    R.tensordot_ooc(A, B, prob["axes_a"], prob["axes_b"], 10, chunk, 1, host, precision=prec)
    planes = host.numpy().view(np.float32)
    n = 1 << 30
    rng = np.random.default_rng(chunk)
    got, ref = [], []
    for blk in [0, (1 << 18) - 1] + [int(x) for x in rng.integers(0, 1 << 18, 4)]:
        re = planes[blk * 4096:(blk + 1) * 4096]
        im = planes[n + blk * 4096:n + (blk + 1) * 4096]
        got.append((re + 1j * im.astype(np.complex128)).reshape(64, 64))
        ref.append(_oracle_block(prob, chunk, blk))
    err = oracle.rel_frobenius(np.stack(got), np.stack(ref))
    assert err <= TOL[prec], err


def test_sweep_ooc_overlap_matches_single_chunks(operands):
    """Two chunks through the double-buffered streaming path equal the same
    chunk computed alone (same kernels, same order of sums)."""
    prob, A, B, host = operands
    R.tensordot_ooc(A, B, prob["axes_a"], prob["axes_b"], 10, 5, 1, host, precision=R.PREC_BF16X3)
    first = host.numpy()[: 1 << 20].copy()
    R.tensordot_ooc(A, B, prob["axes_a"], prob["axes_b"], 10, 4, 2, host, precision=R.PREC_BF16X3)
    # one slot: chunk 5 overwrote chunk 4 in slot (5 - 4) % 1 == 0
    assert np.array_equal(host.numpy()[: 1 << 20], first)
