"""GPU parity of the out-of-core tensordot with A left in host memory
(rosnet_tensordot_ooc_host): each output chunk's slice of A is copied in on
a side stream while the previous chunk is computed, and output chunks stream
out to pinned host memory.

A is written raw (block-major planar) to host memory from a device tensor;
every chunk is checked against the complex128 oracle (the chunk is read back
through a device tensor of the chunk's layout), and against the same chunks
computed with A on the device (same kernels and order of sums: bitwise
equal).  Cases cover several chunks through both staging buffers, fewer host
slots than chunks, a pageable host array, complex128, and the packed FP32 and
tensor-core GEMMs.
"""
import numpy as np
import pytest

import oracle
import paper_2201_06620_b300 as R
import workloads as W

pytestmark = pytest.mark.gpu


def _host_raw(T, pinned=True):
    import torch
    buf = torch.empty(2 * T.numel * (4 if T.dtype == R.C64 else 8), dtype=torch.uint8)
    if pinned:
        buf = buf.pin_memory()
    T.download_raw(buf)
    R.sync()
    return buf


def _chunk_dense(raw, shape, block, dtype):
    C = R.empty(shape, block, dtype)
    C.upload_raw(raw)
    return C.download()


def _run(shape_a, block_a, shape_b, block_b, ax_a, ax_b, nsplit, first, nchunks, nslots, dt=np.complex64,
         precision=R.PREC_DEFAULT, pinned=True, seed=0):
    import torch
    a = W.complex_normal(shape_a, 11 + seed).astype(dt)
    b = W.complex_normal(shape_b, 12 + seed).astype(dt)
    A, B = R.btensor(a, block_a), R.btensor(b, block_b)
    a_host = _host_raw(A, pinned)
    # the output chunk: C's axes after the split ones, with their block extents
    free_a = [i for i in range(len(shape_a)) if i not in ax_a]
    free_b = [i for i in range(len(shape_b)) if i not in ax_b]
    cshape = tuple(shape_a[i] for i in free_a[nsplit:]) + tuple(shape_b[i] for i in free_b)
    cblock = tuple(block_a[i] for i in free_a[nsplit:]) + tuple(block_b[i] for i in free_b)
    esz = 4 if dt == np.complex64 else 8
    chunk_bytes = 2 * int(np.prod(cshape)) * esz
    host = torch.empty(nslots * chunk_bytes, dtype=torch.uint8).pin_memory()
    ref_host = torch.empty(nslots * chunk_bytes, dtype=torch.uint8).pin_memory()
    R.tensordot_ooc_host(a_host, shape_a, block_a, B, ax_a, ax_b, nsplit, first, nchunks, host,
                         precision=precision)
    R.tensordot_ooc(A, B, ax_a, ax_b, nsplit, first, nchunks, ref_host, precision=precision)
    R.sync()
    assert np.array_equal(host.numpy(), ref_host.numpy())
    full = oracle.tensordot(a.astype(np.complex128), b.astype(np.complex128), ax_a, ax_b)
    lead = [shape_a[i] for i in free_a[:nsplit]]
    dtc = R.C64 if dt == np.complex64 else R.C128
    errs = []
    # the chunks left in the host slots: the last nslots of the range
    for c in range(max(first, first + nchunks - nslots), first + nchunks):
        slot = (c - first) % nslots
        got = _chunk_dense(host[slot * chunk_bytes:(slot + 1) * chunk_bytes], cshape, cblock, dtc)
        idx = np.unravel_index(c, lead) if lead else ()
        errs.append(oracle.rel_frobenius(got, full[tuple(idx)]))
    return max(errs)


def test_several_chunks_both_buffers():
    # A [2]^12 (blocks of 2^5 on the trailing axes), 8 chunks along its first 3 axes
    err = _run((2,) * 12, (1,) * 7 + (2,) * 5, (2,) * 9, (2,) * 5 + (1,) * 4, [7, 8, 9, 10, 11],
               [0, 1, 2, 3, 4], 3, 0, 8, 8)
    assert err <= 1e-5, err


def test_fewer_slots_than_chunks_and_offset_range():
    err = _run((4, 3, 6, 8), (1, 1, 3, 4), (8, 6, 5), (4, 3, 5), [2, 3], [1, 0], 2, 3, 7, 3, seed=1)
    assert err <= 1e-5, err


def test_pageable_host_array():
    err = _run((4, 3, 6, 8), (1, 1, 3, 4), (8, 6, 5), (4, 3, 5), [2, 3], [1, 0], 1, 1, 3, 2, pinned=False, seed=2)
    assert err <= 1e-5, err


def test_complex128():
    err = _run((3, 16, 32), (1, 8, 16), (32, 24), (16, 8), [2], [0], 1, 0, 3, 3, dt=np.complex128, seed=3)
    assert err <= 1e-12, err


def test_packed_fp32_and_tensor_core_chunks():
    # 2048 x 512 x 256 per chunk (256 output tiles): the packed FP32 GEMM and the tcgen05 GEMM
    shp_a, blk_a = (2, 256, 2048), (1, 256, 512)
    shp_b, blk_b = (256, 512), (256, 512)
    assert _run(shp_a, blk_a, shp_b, blk_b, [1], [0], 1, 0, 2, 2, seed=4) <= 1e-5
    assert _run(shp_a, blk_a, shp_b, blk_b, [1], [0], 1, 0, 2, 2, precision=R.PREC_TF32X3, seed=5) <= 1e-5


def test_empty_range_and_errors():
    import torch
    b = W.complex_normal((8, 5), 7).astype(np.complex64)
    B = R.btensor(b)
    host = torch.empty(1 << 12, dtype=torch.uint8).pin_memory()
    a_host = torch.empty(2 * 2 * 8 * 4, dtype=torch.uint8).pin_memory()
    R.tensordot_ooc_host(a_host, (2, 8), (1, 8), B, [1], [0], 1, 0, 0, host)      # nothing to do
    with pytest.raises(R.RosnetError):
        R.tensordot_ooc_host(a_host, (2, 8), (1, 8), B, [1], [0], 1, 1, 2, host)  # beyond the output
