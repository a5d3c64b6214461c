"""Python binding of librosnet, the B300 blocked pairwise tensordot library.

Argument marshalling only: every step of a contraction runs in the CUDA
kernels of ``librosnet.so`` (built from ``csrc/`` by ``build.py``).  There is
no CPU fallback: importing works without a GPU, but any call that needs the
device raises ``RosnetError`` if the library or the GPU is missing.

PyTorch provides device memory (its caching allocator is installed as the
library's allocator) and streams (``torch.cuda.current_stream()`` by
default).

The C ABI is declared in ``include/rosnet.h``; the names here mirror it:

* ``BTensor`` -- a block tensor handle (Sec. II-C of the RosneT paper),
  created with ``btensor(array, block_shape)`` or ``empty(...)``;
* ``tensordot(A, B, axes_a, axes_b, precision=...)`` -- the blocked pairwise
  contraction (Sec. II-A, II-C);
* ``path_greedy(...)`` and ``contract(...)`` -- a network contracted along a
  pairwise path (Sec. II-A).
"""
from __future__ import annotations

import atexit
import ctypes
import os
import threading

import numpy as np

__all__ = [
    "RosnetError", "BTensor", "Network", "btensor", "empty", "tensordot", "path_greedy",
    "path_greedy_extents", "contract", "tensordot_noalloc", "tensordot_ooc", "tensordot_ooc_host", "contract_batch",
    "simplify", "cheaper_network", "plan_spill",
    "plan_stats", "path_search", "slice_search", "sliced_networks", "sum_fp64",
    "sync", "kernel_launches", "release_plans", "plan_cache_limit", "lib", "use_torch_allocator",
    "C64", "C128", "PREC_DEFAULT", "PREC_FP32", "PREC_TF32", "PREC_BF16X3", "PREC_FP64",
    "PREC_TF32X3",
    "OPT_GRAPH", "OPT_NOGROUP", "OPT_TIMING", "STATUS", "Network", "timing_drain",
    "REDUCE_SEQUENTIAL", "REDUCE_TREE", "REDUCE_COMMUTATIVE", "OPT_AUTOTUNE",
    "probe_peak", "PROBE_FFMA", "PROBE_DFMA", "PROBE_TF32", "PROBE_BF16", "plan_info", "plan_release",
    "norm2",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librosnet.so")

C64, C128 = 1, 2
PREC_DEFAULT, PREC_FP32, PREC_TF32, PREC_BF16X3, PREC_FP64, PREC_TF32X3 = 0, 1, 2, 3, 4, 5
OPT_GRAPH, OPT_NOGROUP, OPT_TIMING = 0x1, 0x2, 0x4
REDUCE_SEQUENTIAL, REDUCE_TREE, REDUCE_COMMUTATIVE = 0x10, 0x20, 0x40
OPT_AUTOTUNE = 0x80
STATUS = {
    0: "OK", -1: "INVALID_ARG", -2: "SHAPE", -3: "BLOCK_MISMATCH", -4: "DTYPE", -5: "ALLOC",
    -6: "RANK_LIMIT", -7: "CUDA", -8: "TIMEOUT", -9: "UNSUPPORTED",
}
#: every function the header declares
EXPORTS = [
    "rosnet_set_allocator", "rosnet_btensor_create", "rosnet_btensor_destroy",
    "rosnet_btensor_upload", "rosnet_btensor_download", "rosnet_btensor_info",
    "rosnet_btensor_planes", "rosnet_tensordot", "rosnet_path_greedy", "rosnet_contract",
    "rosnet_release_plans", "rosnet_sync", "rosnet_status_string", "rosnet_last_error",
    "rosnet_kernel_launches", "rosnet_path_greedy_extents", "rosnet_timing_drain",
    "rosnet_tensordot_noalloc", "rosnet_btensor_upload_range", "rosnet_btensor_slice",
    "rosnet_btensor_block", "rosnet_tensordot_ooc", "rosnet_tensordot_ooc_host", "rosnet_simplify",
    "rosnet_plan_spill",
    "rosnet_contract_batch",
    "rosnet_plan_stats",
    "rosnet_btensor_fix", "rosnet_path_search", "rosnet_slice_search", "rosnet_sum",
    "rosnet_selftest_timeout", "rosnet_tune_export", "rosnet_tune_import",
    "rosnet_btensor_download_async", "rosnet_alloc_stats", "rosnet_btensor_upload_raw",
    "rosnet_btensor_download_raw", "rosnet_plan_cache_limit", "rosnet_probe_peak",
    "rosnet_plan_release", "rosnet_norm2",
]

_lock = threading.Lock()
_lib = None
_alloc_cbs = None


class RosnetError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        self.name = STATUS.get(status, str(status))
        msg = ""
        if _lib is not None:
            msg = _lib.rosnet_last_error().decode(errors="replace")
        super().__init__(f"{where}: ROSNET_ERR_{self.name} ({status}) {msg}".strip())


class _Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("max_block_entries", ctypes.c_int64), ("reserved", ctypes.c_int64 * 6)]


class _Network(ctypes.Structure):
    _fields_ = [("ntensors", ctypes.c_int32), ("tensors", ctypes.POINTER(ctypes.c_void_p)),
                ("ranks", ctypes.POINTER(ctypes.c_int32)),
                ("labels", ctypes.POINTER(ctypes.POINTER(ctypes.c_int64))),
                ("nout", ctypes.c_int32), ("out_labels", ctypes.POINTER(ctypes.c_int64))]


class _Path(ctypes.Structure):
    _fields_ = [("nsteps", ctypes.c_int32), ("pairs", ctypes.POINTER(ctypes.c_int32))]


_ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


def lib():
    """Load librosnet.so (no GPU needed to load it)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RosnetError(-7, f"librosnet.so not built at {LIB_PATH}; run "
                                      "python -m paper_2201_06620_b300.build")
            L = ctypes.CDLL(LIB_PATH)
            vp, i64p, i32p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)
            L.rosnet_set_allocator.argtypes = [_ALLOC_T, _FREE_T, vp]
            L.rosnet_btensor_create.argtypes = [ctypes.c_int, i64p, i64p, ctypes.c_int, vp,
                                                ctypes.POINTER(vp)]
            L.rosnet_btensor_destroy.argtypes = [vp]
            L.rosnet_btensor_upload.argtypes = [vp, vp, vp]
            L.rosnet_btensor_download.argtypes = [vp, vp, vp]
            L.rosnet_btensor_upload_range.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_int64, vp]
            L.rosnet_btensor_slice.argtypes = [vp, ctypes.c_int, i64p, ctypes.POINTER(vp)]
            L.rosnet_btensor_block.argtypes = [vp, i64p, ctypes.POINTER(vp)]
            L.rosnet_btensor_fix.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), i64p,
                                             ctypes.POINTER(vp)]
            dpp = ctypes.POINTER(ctypes.c_double)
            L.rosnet_path_search.argtypes = [ctypes.c_int32, i32p, ctypes.POINTER(i64p),
                                             ctypes.POINTER(i64p), ctypes.c_int32, i64p, ctypes.c_int32,
                                             ctypes.c_uint64, ctypes.c_double, i32p, i32p, dpp]
            L.rosnet_slice_search.argtypes = [ctypes.c_int32, i32p, ctypes.POINTER(i64p),
                                              ctypes.POINTER(i64p), ctypes.c_int32, i64p, ctypes.c_int32,
                                              i32p, ctypes.c_int32, i64p, dpp, dpp]
            L.rosnet_sum.argtypes = [ctypes.c_int32, ctypes.POINTER(vp), vp, ctypes.POINTER(vp)]
            L.rosnet_selftest_timeout.argtypes = [ctypes.c_int64, vp]
            L.rosnet_probe_peak.argtypes = [ctypes.c_int32, vp, ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_double)]
            L.rosnet_contract_batch.argtypes = [ctypes.c_int32, ctypes.POINTER(_Network),
                                                ctypes.POINTER(_Path), ctypes.POINTER(_Opts), vp,
                                                ctypes.POINTER(vp)]
            L.rosnet_plan_stats.argtypes = [ctypes.c_int32, ctypes.POINTER(_Network),
                                            ctypes.POINTER(_Path), ctypes.POINTER(_Opts), vp, i64p,
                                            i64p, i64p, i64p, i64p]
            L.rosnet_plan_release.argtypes = [ctypes.c_int32, ctypes.POINTER(_Network),
                                              ctypes.POINTER(_Path), ctypes.POINTER(_Opts), vp]
            L.rosnet_plan_spill.argtypes = [ctypes.c_int32, ctypes.POINTER(_Network), ctypes.POINTER(_Path),
                                            ctypes.POINTER(_Opts), vp, i64p]
            L.rosnet_norm2.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_double)]
            L.rosnet_tensordot_ooc.argtypes = [vp, vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                               ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                               ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(_Opts),
                                               vp, ctypes.c_size_t, vp]
            L.rosnet_tensordot_ooc_host.argtypes = [ctypes.c_int, i64p, i64p, vp, vp, ctypes.c_int,
                                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                                    ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                                    ctypes.POINTER(_Opts), vp, ctypes.c_size_t, vp]
            L.rosnet_simplify.argtypes = [ctypes.POINTER(_Network), ctypes.POINTER(ctypes.c_uint8), ctypes.c_int32,
                                          ctypes.POINTER(_Opts), vp, ctypes.POINTER(vp),
                                          ctypes.POINTER(ctypes.c_int32), i64p, ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int32)]
            L.rosnet_btensor_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int), i64p, i64p,
                                              ctypes.POINTER(ctypes.c_int)]
            L.rosnet_btensor_planes.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp)]
            L.rosnet_tensordot.argtypes = [vp, vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_Opts), vp,
                                           ctypes.POINTER(vp)]
            L.rosnet_path_greedy.argtypes = [ctypes.POINTER(_Network), i32p, i32p]
            L.rosnet_tensordot_noalloc.argtypes = [vp, vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                                   ctypes.POINTER(ctypes.c_int), vp,
                                                   ctypes.POINTER(_Opts), vp]
            L.rosnet_path_greedy_extents.argtypes = [
                ctypes.c_int32, i32p, ctypes.POINTER(i64p), ctypes.POINTER(i64p), ctypes.c_int32,
                i64p, i32p, i32p]
            L.rosnet_contract.argtypes = [ctypes.POINTER(_Network), ctypes.POINTER(_Path),
                                          ctypes.POINTER(_Opts), vp, ctypes.POINTER(vp)]
            L.rosnet_release_plans.argtypes = []
            dp = ctypes.POINTER(ctypes.c_double)
            L.rosnet_timing_drain.argtypes = [dp, dp, dp, dp, i32p, ctypes.c_int32, i32p]
            L.rosnet_sync.argtypes = [vp]
            L.rosnet_status_string.argtypes = [ctypes.c_int]
            L.rosnet_status_string.restype = ctypes.c_char_p
            L.rosnet_last_error.argtypes = []
            L.rosnet_last_error.restype = ctypes.c_char_p
            L.rosnet_kernel_launches.argtypes = []
            L.rosnet_kernel_launches.restype = ctypes.c_int64
            L.rosnet_tune_export.argtypes = [ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
            L.rosnet_tune_import.argtypes = [ctypes.c_char_p]
            L.rosnet_btensor_download_async.argtypes = [vp, vp, vp]
            L.rosnet_alloc_stats.argtypes = [i64p, i64p]
            L.rosnet_btensor_upload_raw.argtypes = [vp, vp, vp]
            L.rosnet_btensor_download_raw.argtypes = [vp, vp, vp]
            L.rosnet_plan_cache_limit.argtypes = [ctypes.c_int32, i32p]
            for name in EXPORTS:
                f = getattr(L, name)
                if f.restype is ctypes.c_int or name in (
                        "rosnet_set_allocator", "rosnet_btensor_create", "rosnet_btensor_destroy",
                        "rosnet_btensor_upload", "rosnet_btensor_download", "rosnet_btensor_info",
                        "rosnet_btensor_planes", "rosnet_tensordot", "rosnet_path_greedy",
                        "rosnet_contract", "rosnet_release_plans", "rosnet_sync",
                        "rosnet_path_greedy_extents", "rosnet_timing_drain",
                        "rosnet_tensordot_noalloc", "rosnet_btensor_upload_range",
                        "rosnet_btensor_slice", "rosnet_btensor_block", "rosnet_tensordot_ooc",
                        "rosnet_contract_batch", "rosnet_plan_stats", "rosnet_btensor_fix",
                        "rosnet_path_search", "rosnet_slice_search", "rosnet_sum",
                        "rosnet_selftest_timeout", "rosnet_tune_export", "rosnet_tune_import",
                        "rosnet_btensor_download_async", "rosnet_alloc_stats",
                        "rosnet_btensor_upload_raw", "rosnet_btensor_download_raw",
                        "rosnet_plan_cache_limit", "rosnet_probe_peak", "rosnet_plan_release",
                        "rosnet_norm2", "rosnet_tensordot_ooc_host", "rosnet_simplify",
                        "rosnet_plan_spill"):
                    f.restype = ctypes.c_int
            _lib = L
    return _lib


def _check(status, where):
    if status != 0:
        raise RosnetError(status, where)


def _torch():
    import torch
    return torch


def _default_stream():
    torch = _torch()
    if not torch.cuda.is_available():
        raise RosnetError(-7, "no CUDA device available (librosnet has no CPU fallback)")
    return torch.cuda.current_stream().cuda_stream


def _stream(stream):
    if stream is None:
        return _default_stream()
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def use_torch_allocator(enable=True):
    """Route the library's device allocations through torch's caching allocator
    (enable=False restores the built-in cudaMallocAsync pool, the default).
    Only possible while the library holds no device memory (no tensors or
    cached plans alive)."""
    global _alloc_cbs
    L = lib()
    if not enable:
        _check(L.rosnet_set_allocator(_ALLOC_T(), _FREE_T(), None), "rosnet_set_allocator")
        _alloc_cbs = None
        return
    torch = _torch()

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:  # out of memory -> NULL -> ROSNET_ERR_ALLOC
            return None

    def _free(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    _alloc_cbs = (_ALLOC_T(_alloc), _FREE_T(_free))
    _check(L.rosnet_set_allocator(_alloc_cbs[0], _alloc_cbs[1], None), "rosnet_set_allocator")


_init_done = False
_shutting_down = False


def _at_exit():
    """Free cached plans while the Python allocator callbacks still work, then
    stop touching device memory from finalisers."""
    global _shutting_down
    try:
        if _lib is not None and _alloc_cbs is not None:
            _lib.rosnet_release_plans()
    finally:
        _shutting_down = True


def _init():
    global _init_done
    if not _init_done:
        lib()
        torch = _torch()
        if torch.cuda.is_available():
            torch.cuda.init()
            atexit.register(_at_exit)
        _init_done = True


def _i64arr(seq):
    seq = [int(x) for x in seq]
    return (ctypes.c_int64 * max(1, len(seq)))(*seq)


def _rows_i64(rows):
    """Rows of integers for the C ABI's ``const int64_t *const *`` arguments:
    one flat int64 array holding every row, and an array of pointers to the
    rows' starts.  Returns (flat, pointers); keep both alive while the C side
    may read them."""
    rows = [[int(x) for x in r] for r in rows]
    flat = (ctypes.c_int64 * max(1, sum(len(r) for r in rows)))(*[x for r in rows for x in r])
    base, offs, o = ctypes.addressof(flat), [], 0
    for r in rows:
        offs.append(base + 8 * o if r else base)
        o += len(r)
    ptrs = (ctypes.c_void_p * max(1, len(rows)))(*offs)
    return flat, ctypes.cast(ptrs, ctypes.POINTER(ctypes.POINTER(ctypes.c_int64)))


def _i32arr(seq):
    seq = [int(x) for x in seq]
    return (ctypes.c_int * max(1, len(seq)))(*seq)


def _np_dtype(dt):
    return np.complex64 if dt == C64 else np.complex128


class BTensor:
    """Owning handle of a device block tensor."""

    __slots__ = ("_h", "shape", "block_shape", "dtype", "_parent", "__weakref__")

    def __init__(self, handle):
        self._h = ctypes.c_void_p(handle)
        self._parent = None
        L = lib()
        r = ctypes.c_int()
        sh = (ctypes.c_int64 * 64)()
        bl = (ctypes.c_int64 * 64)()
        dt = ctypes.c_int()
        _check(L.rosnet_btensor_info(self._h, ctypes.byref(r), sh, bl, ctypes.byref(dt)), "info")
        self.shape = tuple(sh[i] for i in range(r.value))
        self.block_shape = tuple(bl[i] for i in range(r.value))
        self.dtype = dt.value

    @property
    def handle(self):
        return self._h

    @property
    def rank(self):
        return len(self.shape)

    @property
    def numel(self):
        return int(np.prod(self.shape, dtype=np.int64)) if self.shape else 1

    def planes(self):
        re, im = ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib().rosnet_btensor_planes(self._h, ctypes.byref(re), ctypes.byref(im)), "planes")
        return re.value, im.value

    def upload(self, array, stream=None):
        """Copy a host array (numpy, or a pinned torch CPU tensor) into the tensor."""
        if hasattr(array, "data_ptr"):  # torch CPU tensor (e.g. pinned)
            ptr = array.data_ptr()
            keep = array
        else:
            keep = np.asarray(array, dtype=_np_dtype(self.dtype), order="C")
            if keep.shape != self.shape:
                raise ValueError(f"shape {keep.shape} != tensor shape {self.shape}")
            ptr = keep.ctypes.data
        _check(lib().rosnet_btensor_upload(self._h, ctypes.c_void_p(ptr), _stream(stream)), "upload")
        return keep

    def upload_range(self, array, start, stream=None):
        """Copy host values into the dense row-major entries [start, start + len)."""
        keep = np.ascontiguousarray(np.asarray(array, dtype=_np_dtype(self.dtype)).reshape(-1))
        _check(lib().rosnet_btensor_upload_range(self._h, ctypes.c_void_p(keep.ctypes.data), int(start),
                                                 keep.size, _stream(stream)), "upload_range")
        return keep

    def slice(self, values):
        """View with the leading len(values) (grid) axes fixed; shares storage."""
        h = ctypes.c_void_p()
        _check(lib().rosnet_btensor_slice(self._h, len(values), _i64arr(values), ctypes.byref(h)),
               "rosnet_btensor_slice")
        v = BTensor(h.value)
        v._parent = self
        return v

    def fix(self, axes, values):
        """View with axes[j] fixed to values[j] (any axes); shares storage."""
        h = ctypes.c_void_p()
        _check(lib().rosnet_btensor_fix(self._h, len(axes), _i32arr(axes), _i64arr(values),
                                        ctypes.byref(h)), "rosnet_btensor_fix")
        v = BTensor(h.value)
        v._parent = self
        return v

    def block(self, grid_coords):
        """View of one block (grid coordinates per axis); shares storage."""
        h = ctypes.c_void_p()
        _check(lib().rosnet_btensor_block(self._h, _i64arr(grid_coords), ctypes.byref(h)),
               "rosnet_btensor_block")
        v = BTensor(h.value)
        v._parent = self
        return v

    def download(self, out=None, stream=None):
        """Dense row-major host copy (numpy); synchronises the stream."""
        if out is None:
            out = np.empty(self.shape, dtype=_np_dtype(self.dtype))
        if hasattr(out, "data_ptr"):
            ptr = out.data_ptr()
        else:
            ptr = out.ctypes.data
        _check(lib().rosnet_btensor_download(self._h, ctypes.c_void_p(ptr), _stream(stream)),
               "download")
        return out

    def download_async(self, out, stream=None):
        """Enqueue a dense row-major copy into ``out`` (a page-locked torch
        tensor or numpy array of the right size) on the stream, without
        waiting: ``out`` is complete once the stream reaches this point."""
        ptr = out.data_ptr() if hasattr(out, "data_ptr") else out.ctypes.data
        _check(lib().rosnet_btensor_download_async(self._h, ctypes.c_void_p(ptr), _stream(stream)),
               "download_async")
        return out

    def _raw_ptr(self, buf):
        nbytes = buf.numel() * buf.element_size() if hasattr(buf, "data_ptr") else buf.nbytes
        if nbytes != 2 * self.numel * (4 if self.dtype == C64 else 8):
            raise ValueError("raw buffer must hold 2 * numel real values (real plane, imaginary plane)")
        return buf.data_ptr() if hasattr(buf, "data_ptr") else buf.ctypes.data

    def upload_raw(self, buf, stream=None):
        """Copy the real plane then the imaginary plane (block-major order) from
        ``buf`` (a page-locked or CUDA torch tensor, or a numpy array, of
        2 * numel reals) into the tensor's storage: one enqueued copy, no
        kernel."""
        _check(lib().rosnet_btensor_upload_raw(self._h, ctypes.c_void_p(self._raw_ptr(buf)), _stream(stream)),
               "upload_raw")
        return buf

    def download_raw(self, buf, stream=None):
        """Enqueue a copy of the tensor's storage (real plane, imaginary plane)
        into ``buf`` without waiting."""
        _check(lib().rosnet_btensor_download_raw(self._h, ctypes.c_void_p(self._raw_ptr(buf)), _stream(stream)),
               "download_raw")
        return buf

    def destroy(self):
        if _shutting_down:   # the allocator behind the handle may be gone
            self._h = None
            return
        if self._h is not None and self._h.value:
            lib().rosnet_btensor_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def __repr__(self):
        return f"BTensor(shape={self.shape}, block_shape={self.block_shape}, dtype={'c64' if self.dtype == C64 else 'c128'})"


def empty(shape, block_shape=None, dtype=C64, stream=None):
    _init()
    h = ctypes.c_void_p()
    bl = _i64arr(block_shape) if block_shape is not None else None
    _check(lib().rosnet_btensor_create(len(shape), _i64arr(shape), bl, int(dtype), _stream(stream),
                                       ctypes.byref(h)), "rosnet_btensor_create")
    return BTensor(h.value)


def btensor(array, block_shape=None, dtype=None, stream=None):
    """Create a block tensor from a host array and upload it."""
    array = np.asarray(array)
    if dtype is None:
        dtype = C128 if array.dtype == np.complex128 else C64
    t = empty(array.shape, block_shape, dtype, stream)
    t.upload(array, stream)
    return t


def _opts(precision, flags=0, max_block_entries=0):
    o = _Opts()
    o.precision = int(precision)
    o.flags = int(flags)
    o.max_block_entries = int(max_block_entries)
    return o


def tensordot(A, B, axes_a, axes_b, precision=PREC_DEFAULT, stream=None, flags=0):
    """C = tensordot(A, B, axes=(axes_a, axes_b)) on the GPU (numpy conventions).
    ``flags`` may hold one REDUCE_* mode."""
    _init()
    h = ctypes.c_void_p()
    o = _opts(precision, flags)
    _check(lib().rosnet_tensordot(A.handle, B.handle, len(axes_a), _i32arr(axes_a), _i32arr(axes_b),
                                  ctypes.byref(o), _stream(stream), ctypes.byref(h)),
           "rosnet_tensordot")
    return BTensor(h.value)


def tensordot_noalloc(A, B, axes_a, axes_b, C, precision=PREC_DEFAULT, stream=None, flags=0):
    """tensordot into an existing tensor C without any device allocation (the
    library's fixed scratch array holds the kernels' workspace).  ``flags``
    may hold one REDUCE_* mode."""
    _init()
    o = _opts(precision, flags)
    _check(lib().rosnet_tensordot_noalloc(A.handle, B.handle, len(axes_a), _i32arr(axes_a),
                                          _i32arr(axes_b), C.handle, ctypes.byref(o),
                                          _stream(stream)), "rosnet_tensordot_noalloc")
    return C


def tensordot_ooc(A, B, axes_a, axes_b, nsplit, first_chunk, nchunks, host_out,
                  precision=PREC_DEFAULT, stream=None):
    """Out-of-core tensordot: output chunks along A's first nsplit (grid) axes
    streamed into the pinned host buffer ``host_out`` (a torch CPU tensor or a
    numpy array; chunk c goes to slot (c - first_chunk) % slots, raw
    block-major planar).  Returns when the copies are complete."""
    _init()
    o = _opts(precision)
    if hasattr(host_out, "data_ptr"):
        ptr, nbytes = host_out.data_ptr(), host_out.numel() * host_out.element_size()
    else:
        ptr, nbytes = host_out.ctypes.data, host_out.nbytes
    _check(lib().rosnet_tensordot_ooc(A.handle, B.handle, len(axes_a), _i32arr(axes_a),
                                      _i32arr(axes_b), int(nsplit), int(first_chunk), int(nchunks),
                                      ctypes.byref(o), ctypes.c_void_p(ptr), int(nbytes),
                                      _stream(stream)), "rosnet_tensordot_ooc")


def tensordot_ooc_host(a_host, shape_a, block_a, B, axes_a, axes_b, nsplit, first_chunk, nchunks, host_out,
                       precision=PREC_DEFAULT, stream=None):
    """Out-of-core tensordot with A in host memory: ``a_host`` (a pinned torch
    CPU tensor or a numpy array) holds A raw block-major planar (real plane,
    then imaginary plane) with the given shape and block shape; each chunk's
    slice of A is copied in on a side stream while the previous chunk is
    computed, and output chunks go to ``host_out`` as in tensordot_ooc."""
    _init()
    o = _opts(precision)

    def ptr_bytes(x):
        if hasattr(x, "data_ptr"):
            return x.data_ptr(), x.numel() * x.element_size()
        return x.ctypes.data, x.nbytes
    aptr, _ = ptr_bytes(a_host)
    optr, obytes = ptr_bytes(host_out)
    blk = None if block_a is None else _i64arr(block_a)
    _check(lib().rosnet_tensordot_ooc_host(len(shape_a), _i64arr(shape_a), blk, ctypes.c_void_p(aptr), B.handle,
                                           len(axes_a), _i32arr(axes_a), _i32arr(axes_b), int(nsplit),
                                           int(first_chunk), int(nchunks), ctypes.byref(o), ctypes.c_void_p(optr),
                                           int(obytes), _stream(stream)), "rosnet_tensordot_ooc_host")


class Network:
    """A network prepared for repeated contraction: the ctypes view of its
    tensors, labels and output labels is built once; ``set_tensor`` swaps a
    leaf (e.g. the output-bitstring projectors of an amplitude query) without
    rebuilding it."""

    def __init__(self, tensors, labels, out_labels=()):
        n = len(tensors)
        self.tensors = list(tensors)
        self.labels = [tuple(int(x) for x in l) for l in labels]
        self.out_labels = [int(x) for x in out_labels]
        self.handles = (ctypes.c_void_p * max(1, n))(*[t.handle.value for t in tensors])
        self.ranks = (ctypes.c_int32 * max(1, n))(*[len(l) for l in labels])
        self._lab, self._labp = _rows_i64(self.labels)
        self._out = _i64arr(out_labels)
        self.net = _Network(n, ctypes.cast(self.handles, ctypes.POINTER(ctypes.c_void_p)),
                            ctypes.cast(self.ranks, ctypes.POINTER(ctypes.c_int32)), self._labp,
                            len(out_labels), ctypes.cast(self._out, ctypes.POINTER(ctypes.c_int64)))
        self._path = None
        self._path_key = None
        self._path_src = None

    def set_tensor(self, i, t):
        self.tensors[i] = t
        self.handles[i] = t.handle.value

    def greedy_path(self):
        n = len(self.tensors)
        pairs = (ctypes.c_int32 * max(1, 2 * (n - 1)))()
        ns = ctypes.c_int32()
        _check(lib().rosnet_path_greedy(ctypes.byref(self.net), pairs, ctypes.byref(ns)),
               "rosnet_path_greedy")
        return [(pairs[2 * i], pairs[2 * i + 1]) for i in range(ns.value)]

    def _cpath(self, path):
        if path is self._path_src:        # the same list object as last time
            return self._path
        self._path_src = path
        key = tuple(tuple(p) for p in path)
        if key != self._path_key:
            flat = [int(x) for p in key for x in p]
            self._parr = (ctypes.c_int32 * max(1, len(flat)))(*flat)
            self._path = _Path(len(key), ctypes.cast(self._parr, ctypes.POINTER(ctypes.c_int32)))
            self._path_key = key
        return self._path


def path_greedy(tensors, labels, out_labels=()):
    """The library's greedy min-size path as a list of SSA pairs."""
    return Network(tensors, labels, out_labels).greedy_path()


def path_greedy_extents(labels, extents, out_labels=()):
    """Greedy path from labels and extents alone (host-only, no GPU needed)."""
    n, ranks, labp, extp, out, keep = _label_args(labels, extents, out_labels)
    pairs = (ctypes.c_int32 * max(1, 2 * (n - 1)))()
    ns = ctypes.c_int32()
    _check(lib().rosnet_path_greedy_extents(n, ranks, labp, extp, len(out_labels), out, pairs,
                                            ctypes.byref(ns)), "rosnet_path_greedy_extents")
    return [(pairs[2 * i], pairs[2 * i + 1]) for i in range(ns.value)]


def _label_args(labels, extents, out_labels):
    n = len(labels)
    ranks = (ctypes.c_int32 * max(1, n))(*[len(l) for l in labels])
    lab, labp = _rows_i64(labels)
    ext, extp = _rows_i64(extents)
    out = _i64arr(out_labels)
    return n, ranks, labp, extp, out, (lab, ext)


def path_search(labels, extents, out_labels=(), ntrials=64, seed=0, temperature=0.3):
    """Randomised greedy path search (host-only): (path, total flops)."""
    n, ranks, labp, extp, out, keep = _label_args(labels, extents, out_labels)
    pairs = (ctypes.c_int32 * max(1, 2 * (n - 1)))()
    ns = ctypes.c_int32()
    fl = ctypes.c_double()
    _check(lib().rosnet_path_search(n, ranks, labp, extp, len(out_labels), out, int(ntrials), int(seed),
                                    float(temperature), pairs, ctypes.byref(ns), ctypes.byref(fl)),
           "rosnet_path_search")
    return [(pairs[2 * i], pairs[2 * i + 1]) for i in range(ns.value)], fl.value


def slice_search(labels, extents, out_labels, path, nslice):
    """Greedy choice of bonds to slice for a path: (labels, max entries, total flops)."""
    n, ranks, labp, extp, out, keep = _label_args(labels, extents, out_labels)
    flat = [int(x) for p in path for x in p]
    parr = (ctypes.c_int32 * max(1, len(flat)))(*flat)
    chosen = (ctypes.c_int64 * max(1, nslice))()
    mx, fl = ctypes.c_double(), ctypes.c_double()
    _check(lib().rosnet_slice_search(n, ranks, labp, extp, len(out_labels), out, len(path), parr,
                                     int(nslice), chosen, ctypes.byref(mx), ctypes.byref(fl)),
           "rosnet_slice_search")
    return [chosen[i] for i in range(nslice)], mx.value, fl.value


def sliced_networks(tensors, labels, out_labels, cut):
    """The projections of a network onto every basis assignment of the bonds in
    ``cut`` (Sec. II-B): each tensor carrying cut bonds becomes a view with
    those axes fixed.  Returns [(assignment, Network)] in row-major order of
    the assignments; views of equal projections share storage."""
    import itertools
    ext = {}
    for t, l in zip(tensors, labels):
        for x, e in zip(l, t.shape):
            ext[x] = e
    cut = list(cut)
    out = []
    for vals in itertools.product(*[range(ext[c]) for c in cut]):
        val = dict(zip(cut, vals))
        ts, ls = [], []
        for t, l in zip(tensors, labels):
            axes = [i for i, x in enumerate(l) if x in val]
            if axes:
                ts.append(t.fix(axes, [val[l[i]] for i in axes]))
                ls.append(tuple(x for x in l if x not in val))
            else:
                ts.append(t)
                ls.append(tuple(l))
        out.append((vals, Network(ts, ls, out_labels)))
    return out


def sum_fp64(tensors, stream=None):
    """Elementwise FP64 sum of equal-shape tensors (a complex128 BTensor)."""
    _init()
    arr = (ctypes.c_void_p * len(tensors))(*[t.handle.value for t in tensors])
    h = ctypes.c_void_p()
    _check(lib().rosnet_sum(len(tensors), arr, _stream(stream), ctypes.byref(h)), "rosnet_sum")
    return BTensor(h.value)


def simplify(tensors, labels, out_labels=(), keep=(), max_rank=2, precision=PREC_DEFAULT, stream=None):
    """Rank reduction before path search (rosnet_simplify): tensors of rank
    <= max_rank not in ``keep`` (indices) are absorbed into neighbours by
    tensordots on the device.  Returns (tensors, labels, origin): the
    survivors in input order (the caller's own BTensor where nothing was
    absorbed, a new one otherwise), their labels, and for each the input
    index whose position it holds."""
    _init()
    net = Network(tensors, labels, out_labels)
    n = len(tensors)
    kp = (ctypes.c_uint8 * max(1, n))(*[1 if i in set(keep) else 0 for i in range(n)])
    tout = (ctypes.c_void_p * max(1, n))()
    rout = (ctypes.c_int32 * max(1, n))()
    lout = (ctypes.c_int64 * max(1, sum(len(l) for l in net.labels)))()
    oout = (ctypes.c_int32 * max(1, n))()
    nout = ctypes.c_int32()
    o = _opts(precision)
    _check(lib().rosnet_simplify(ctypes.byref(net.net), kp, int(max_rank), ctypes.byref(o), _stream(stream), tout,
                                 rout, lout, oout, ctypes.byref(nout)), "rosnet_simplify")
    res_t, res_l, origin, pos = [], [], [], 0
    for i in range(nout.value):
        j = oout[i]
        h = tout[i]
        res_t.append(tensors[j] if h == tensors[j].handle.value else BTensor(h))
        res_l.append(tuple(lout[pos:pos + rout[i]]))
        origin.append(j)
        pos += rout[i]
    return res_t, res_l, origin


def cheaper_network(tensors, labels, out_labels=(), keep=(), ntrials=16, seed=0, max_rank=2, stream=None):
    """The network as given or simplified (``simplify``), whichever has the
    cheaper path found by ``path_search`` with the same trials and seed:
    (tensors, labels, path, flops).  Simplification leaves fewer, larger
    tensors, on which the randomised greedy search can find better or worse
    paths than on the raw network, so both are searched."""
    ext = [t.shape for t in tensors]
    path, fl = path_search(labels, ext, out_labels, ntrials=ntrials, seed=seed)
    st, sl, _ = simplify(tensors, labels, out_labels, keep=keep, max_rank=max_rank, stream=stream)
    if len(st) == len(tensors):
        return list(tensors), [tuple(l) for l in labels], path, fl
    p2, f2 = path_search(sl, [t.shape for t in st], out_labels, ntrials=ntrials, seed=seed)
    if f2 < fl:
        return st, sl, p2, f2
    return list(tensors), [tuple(l) for l in labels], path, fl


def contract(tensors, labels=None, out_labels=None, path=None, precision=PREC_DEFAULT, flags=0,
             max_block_entries=0, stream=None):
    """Contract a network along an SSA path on the GPU.

    ``tensors`` is either a prepared ``Network`` (then ``labels`` and
    ``out_labels`` are ignored) or a list of BTensors with their labels."""
    _init()
    net = tensors if isinstance(tensors, Network) else Network(tensors, labels, out_labels or ())
    if path is None:
        path = net.greedy_path()
    pth = net._cpath(path)
    o = _opts(precision, flags, max_block_entries)
    h = ctypes.c_void_p()
    _check(lib().rosnet_contract(ctypes.byref(net.net), ctypes.byref(pth), ctypes.byref(o),
                                 _stream(stream), ctypes.byref(h)), "rosnet_contract")
    return BTensor(h.value)


def _batch_args(networks, paths):
    nets = [n if isinstance(n, Network) else Network(*n) for n in networks]
    arr = (_Network * len(nets))(*[n.net for n in nets])
    cps = [n._cpath(p) for n, p in zip(nets, paths)]
    parr = (_Path * len(nets))(*cps)
    return nets, arr, parr


def contract_batch(networks, paths, precision=PREC_DEFAULT, flags=0, max_block_entries=0,
                   stream=None):
    """Contract several networks in one plan (common steps computed once);
    ``networks``: Network objects or (tensors, labels, out_labels) tuples."""
    _init()
    nets, arr, parr = _batch_args(networks, paths)
    o = _opts(precision, flags, max_block_entries)
    outs = (ctypes.c_void_p * len(nets))()
    _check(lib().rosnet_contract_batch(len(nets), arr, parr, ctypes.byref(o), _stream(stream), outs),
           "rosnet_contract_batch")
    return [BTensor(outs[i]) for i in range(len(nets))]


def plan_stats(networks, paths, precision=PREC_DEFAULT, flags=0, max_block_entries=0, stream=None):
    """(steps requested, distinct steps planned, launches per call, operands
    gathered into a packed workspace per call) of a planned batch."""
    return plan_info(networks, paths, precision, flags, max_block_entries, stream)[:4]


def plan_info(networks, paths, precision=PREC_DEFAULT, flags=0, max_block_entries=0, stream=None):
    """plan_stats plus the device bytes the cached plan holds between calls."""
    nets, arr, parr = _batch_args(networks, paths)
    o = _opts(precision, flags, max_block_entries)
    v = [ctypes.c_int64() for _ in range(5)]
    _check(lib().rosnet_plan_stats(len(nets), arr, parr, ctypes.byref(o), _stream(stream),
                                   *[ctypes.byref(x) for x in v]), "rosnet_plan_stats")
    return tuple(x.value for x in v)


def plan_release(networks, paths, precision=PREC_DEFAULT, flags=0, max_block_entries=0, stream=None):
    """Free the cached plan of these arguments (rosnet_plan_release)."""
    nets, arr, parr = _batch_args(networks, paths)
    o = _opts(precision, flags, max_block_entries)
    _check(lib().rosnet_plan_release(len(nets), arr, parr, ctypes.byref(o), _stream(stream)),
           "rosnet_plan_release")


def plan_spill(networks, paths, precision=PREC_DEFAULT, flags=0, max_block_entries=0, stream=None):
    """Move the cached plan of these arguments to pinned host memory
    (rosnet_plan_spill); the next contraction restores it.  Returns the
    page-locked bytes it holds."""
    nets, arr, parr = _batch_args(networks, paths)
    o = _opts(precision, flags, max_block_entries)
    hb = ctypes.c_int64()
    _check(lib().rosnet_plan_spill(len(nets), arr, parr, ctypes.byref(o), _stream(stream), ctypes.byref(hb)),
           "rosnet_plan_spill")
    return hb.value


def norm2(t, stream=None):
    """Sum of |x|^2 over the tensor, accumulated in FP64 on the GPU."""
    _init()
    out = ctypes.c_double()
    _check(lib().rosnet_norm2(t.handle, _stream(stream), ctypes.byref(out)), "rosnet_norm2")
    return out.value


def sync(stream=None):
    _check(lib().rosnet_sync(_stream(stream)), "rosnet_sync")


def kernel_launches():
    return int(lib().rosnet_kernel_launches())


PROBE_FFMA, PROBE_DFMA, PROBE_TF32, PROBE_BF16 = 0, 1, 2, 3


def probe_peak(kind, stream=None):
    """Measured peak of one kind of arithmetic (PROBE_*): (TFLOP/s, flops, ms)."""
    _init()
    fl, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib().rosnet_probe_peak(int(kind), _stream(stream), ctypes.byref(fl), ctypes.byref(ms)),
           "rosnet_probe_peak")
    return fl.value / (ms.value * 1e-3) / 1e12, fl.value, ms.value


def timing_drain(max_entries=4096):
    """[(ms, flops, bytes, kind, ms_whole)] of the heaviest launch of each
    timed contract call: ms covers its GEMM kernel (for packed-operand
    launches after the operand packs), ms_whole the whole launch."""
    ms = (ctypes.c_double * max_entries)()
    mw = (ctypes.c_double * max_entries)()
    fl = (ctypes.c_double * max_entries)()
    by = (ctypes.c_double * max_entries)()
    kd = (ctypes.c_int32 * max_entries)()
    n = ctypes.c_int32()
    _check(lib().rosnet_timing_drain(ms, mw, fl, by, kd, max_entries, ctypes.byref(n)), "rosnet_timing_drain")
    return [(ms[i], fl[i], by[i], kd[i], mw[i]) for i in range(n.value)]


def release_plans():
    _check(lib().rosnet_release_plans(), "rosnet_release_plans")


def plan_cache_limit(max_plans=-1):
    """Set the most contraction plans kept cached (0: no limit; least recently
    used freed first); a negative value only queries.  Returns the number of
    plans cached after the call."""
    n = ctypes.c_int32()
    _check(lib().rosnet_plan_cache_limit(int(max_plans), ctypes.byref(n)), "rosnet_plan_cache_limit")
    return n.value


def alloc_stats():
    """(device blocks requested since load, blocks still live)."""
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().rosnet_alloc_stats(ctypes.byref(a), ctypes.byref(b)), "rosnet_alloc_stats")
    return a.value, b.value


def tune_export():
    """The autotuner's decisions as text (one line per tuned problem shape)."""
    L = lib()
    n = ctypes.c_size_t()
    _check(L.rosnet_tune_export(None, 0, ctypes.byref(n)), "rosnet_tune_export")
    buf = ctypes.create_string_buffer(n.value)
    _check(L.rosnet_tune_export(buf, n.value, ctypes.byref(n)), "rosnet_tune_export")
    return buf.value.decode()


def tune_import(text):
    """Merge decisions written by tune_export (checked against their shapes)."""
    _check(lib().rosnet_tune_import(text.encode()), "rosnet_tune_import")
