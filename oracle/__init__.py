"""CPU oracle for the blocked pairwise tensordot -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the GPU library
``paper_2201_06620_b300`` and never imports it; both sides take their inputs
from the seeded generators in ``workloads``.

Functions (all complex128):

* ``tensordot(a, b, axes_a, axes_b)`` -- plain loop contraction of Sec. II-A,
  numpy tensordot conventions (C loops in ``oracle.c``).
* ``block_tensordot(a, block_a, b, block_b, axes_a, axes_b)`` -- the same
  result computed block by block with the four steps of Sec. II-C.
* ``contract(network, path)`` -- a tensor network contracted pairwise along
  ``path`` (SSA pairs: step t joins ids i, j and creates id ntensors + t), each
  step one call of ``tensordot`` (Sec. II-A: a contraction is a sequence of
  pairwise operations between neighbouring tensors).
* ``greedy_path(network)`` -- the oracle's own contraction order (any order
  gives the same result up to rounding).
* ``sliced_contract(network, path, cut)`` -- Sec. II-B slicing: the sum over
  all basis assignments of the cut bonds of the projected networks.
* ``statevector(circuit)`` / ``amplitude_sv`` -- |psi> = C|0^n> by applying each
  gate to the 2^n state vector (Sec. II-A), an independent check of network
  contraction.

Every function here is pinned by ``tests/test_oracle.py`` against numpy,
closed forms, brute force, invariants and the paper's equations.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile ``oracle.c`` into ``_oracle.so`` with gcc (plain C, OpenMP)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            i64p = ctypes.POINTER(ctypes.c_int64)
            ip = ctypes.POINTER(ctypes.c_int)
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_tensordot.argtypes = [ctypes.c_int, i64p, dp, ctypes.c_int, i64p, dp,
                                             ctypes.c_int, ip, ip, dp, ctypes.c_int]
            lib.oracle_block_tensordot.argtypes = [ctypes.c_int, i64p, i64p, dp,
                                                   ctypes.c_int, i64p, i64p, dp,
                                                   ctypes.c_int, ip, ip, dp]
            lib.oracle_apply_gate1.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp]
            lib.oracle_apply_gate2.argtypes = [ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, dp]
            for f in (lib.oracle_tensordot, lib.oracle_block_tensordot,
                      lib.oracle_apply_gate1, lib.oracle_apply_gate2):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _i64(seq):
    arr = (ctypes.c_int64 * max(1, len(seq)))(*[int(x) for x in seq])
    return arr


def _i32(seq):
    return (ctypes.c_int * max(1, len(seq)))(*[int(x) for x in seq])


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _as_c128(a):
    """complex128, C-contiguous, rank preserved (rank-0 stays a scalar)."""
    a = np.asarray(a, dtype=np.complex128)
    return a if a.flags.c_contiguous else a.copy(order="C")


def _out_shape(sa, sb, axes_a, axes_b):
    fa = [i for i in range(len(sa)) if i not in set(axes_a)]
    fb = [i for i in range(len(sb)) if i not in set(axes_b)]
    return tuple(sa[i] for i in fa) + tuple(sb[i] for i in fb)


def tensordot(a, b, axes_a, axes_b, nthreads=None):
    """C[fA, fB] = sum_k A[fA, k] B[k, fB] in complex128 (plain loops)."""
    lib = _load()
    a = _as_c128(a)
    b = _as_c128(b)
    axes_a = [int(x) % max(1, a.ndim) for x in axes_a]
    axes_b = [int(x) % max(1, b.ndim) for x in axes_b]
    oshape = _out_shape(a.shape, b.shape, axes_a, axes_b)
    c = np.zeros(oshape, dtype=np.complex128)
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    rc = lib.oracle_tensordot(a.ndim, _i64(a.shape), _dptr(a), b.ndim, _i64(b.shape), _dptr(b),
                              len(axes_a), _i32(axes_a), _i32(axes_b), _dptr(c), int(nthreads))
    if rc:
        raise ValueError("oracle_tensordot: invalid arguments")
    return c


def block_tensordot(a, block_a, b, block_b, axes_a, axes_b):
    """tensordot computed with the block steps of Sec. II-C (same result)."""
    lib = _load()
    a = _as_c128(a)
    b = _as_c128(b)
    oshape = _out_shape(a.shape, b.shape, axes_a, axes_b)
    c = np.zeros(oshape, dtype=np.complex128)
    rc = lib.oracle_block_tensordot(a.ndim, _i64(a.shape), _i64(block_a), _dptr(a),
                                    b.ndim, _i64(b.shape), _i64(block_b), _dptr(b),
                                    len(axes_a), _i32(axes_a), _i32(axes_b), _dptr(c))
    if rc:
        raise ValueError("oracle_block_tensordot: invalid arguments")
    return c


# ---------------------------------------------------------------------------
# networks
# ---------------------------------------------------------------------------
def _pair_axes(la, lb, keep):
    """Contracted axes of a pair: labels shared by both and not kept open."""
    shared = [x for x in la if x in lb and x not in keep]
    return [la.index(x) for x in shared], [lb.index(x) for x in shared], shared


def contract(network, path, nthreads=None):
    """Contract ``network`` pairwise along the SSA ``path``; returns the result
    with its axes in ``network.out_labels`` order.

    A label shared by the two operands of a step is summed over unless it is
    an output label or still appears on another live tensor (it then stays
    open on the intermediate).
    """
    tensors = {i: _as_c128(t) for i, t in enumerate(network.tensors)}
    labels = {i: list(l) for i, l in enumerate(network.labels)}
    out = list(network.out_labels)
    nxt = len(network.tensors)
    for i, j in path:
        a, la = tensors.pop(i), labels.pop(i)
        b, lb = tensors.pop(j), labels.pop(j)
        still = set(out)
        for l in labels.values():
            still.update(l)
        ax_a, ax_b, shared = _pair_axes(la, lb, still)
        c = tensordot(a, b, ax_a, ax_b, nthreads)
        lc = [x for x in la if x not in shared] + [x for x in lb if x not in shared]
        tensors[nxt], labels[nxt] = c, lc
        nxt += 1
    if len(tensors) != 1:
        raise ValueError("path does not reduce the network to one tensor")
    (k,) = tensors.keys()
    res, lres = tensors[k], labels[k]
    if sorted(lres) != sorted(out):
        raise ValueError("open labels of the result do not match out_labels")
    perm = [lres.index(x) for x in out]
    return np.transpose(res, perm) if perm else res


def greedy_path(network):
    """The oracle's own pairwise order: repeatedly join the connected pair whose
    result has the fewest entries, ties to the smaller (result entries - entries
    of the two operands), then to the lowest ids; disconnected pieces are
    joined last.  Any order gives the same result up to rounding."""
    labels = {i: list(l) for i, l in enumerate(network.labels)}
    ext = {}
    for t, l in zip(network.tensors, network.labels):
        for x, e in zip(l, np.shape(t)):
            ext[x] = e
    out = set(network.out_labels)
    nxt = len(labels)
    path = []

    def size(ls):
        p = 1
        for x in ls:
            p *= ext[x]
        return p

    while len(labels) > 1:
        best = None
        ids = sorted(labels)
        count = {}
        for l in labels.values():
            for x in l:
                count[x] = count.get(x, 0) + 1
        for ai, i in enumerate(ids):
            for j in ids[ai + 1:]:
                shared = set(labels[i]) & set(labels[j])
                if not shared:
                    continue
                summed = {x for x in shared if x not in out and count[x] == 2}
                res = [x for x in labels[i] if x not in summed] + [x for x in labels[j] if x not in summed]
                key = (size(res), size(res) - size(labels[i]) - size(labels[j]), i, j)
                if best is None or key < best[0]:
                    best = (key, i, j, summed)
        if best is None:  # disconnected: outer product of the two lowest ids
            i, j = ids[0], ids[1]
            summed = set()
        else:
            _, i, j, summed = best
        lc = [x for x in labels[i] if x not in summed] + [x for x in labels[j] if x not in summed]
        del labels[i], labels[j]
        labels[nxt] = lc
        path.append((i, j))
        nxt += 1
    return path


def sliced_contract(network, path, cut):
    """Sec. II-B slicing: the sum, over every basis assignment of the bonds in
    ``cut``, of the network projected onto that assignment (each tensor that
    carries a cut bond is indexed at the assigned value and loses that axis),
    each contracted along the same ``path``; summed in complex128."""
    import itertools
    ext = {}
    for t, l in zip(network.tensors, network.labels):
        for x, e in zip(l, np.shape(t)):
            ext[x] = e
    total = None
    for vals in itertools.product(*[range(ext[c]) for c in cut]):
        val = dict(zip(cut, vals))
        ts, ls = [], []
        for t, l in zip(network.tensors, network.labels):
            t = _as_c128(t)
            idx = tuple(val[x] if x in val else slice(None) for x in l)
            ts.append(_as_c128(t[idx]) if any(x in val for x in l) else t)
            ls.append(tuple(x for x in l if x not in val))
        part = contract(type(network)(tensors=ts, labels=ls, out_labels=list(network.out_labels)), path)
        total = part if total is None else total + part
    return total


def circuit_order_path(network):
    """Absorb tensors one by one in network order into a running tensor (the
    state-vector-like order)."""
    n = len(network.tensors)
    path = []
    cur = 0
    for t in range(1, n):
        path.append((cur, t))
        cur = n + t - 1
    return path


# ---------------------------------------------------------------------------
# state vector
# ---------------------------------------------------------------------------
def statevector(circ):
    """C|0^n> as a flat complex128 vector (qubit 0 = most significant bit)."""
    lib = _load()
    n = circ.n
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    for _name, qs, mat in circ.gates:
        g = np.ascontiguousarray(np.asarray(mat, dtype=np.complex128).reshape(-1))
        if len(qs) == 1:
            rc = lib.oracle_apply_gate1(n, _dptr(psi), int(qs[0]), _dptr(g))
        else:
            rc = lib.oracle_apply_gate2(n, _dptr(psi), int(qs[0]), int(qs[1]), _dptr(g))
        if rc:
            raise ValueError("bad gate")
    return psi


def bitstring_index(bits):
    idx = 0
    for b in bits:
        idx = (idx << 1) | int(b)
    return idx


def amplitude_sv(circ, bits=None):
    """<x|C|0^n> from the state vector."""
    if bits is None:
        bits = circ.bitstring
    return statevector(circ)[bitstring_index(bits)]


# ---------------------------------------------------------------------------
# memory model of the reduction strategies (Sec. IV-A, Eq. 1 and Eq. 2)
# ---------------------------------------------------------------------------
def mem_sequential(B_k, m_b, n_b, k_b):
    """Elements held by a sequential-reduction task: all B_k pairs of input
    blocks plus the accumulator (Eq. 1)."""
    return B_k * k_b * (m_b + n_b) + m_b * n_b


def mem_pair(m_b, n_b, k_b):
    """Elements held by a one-pair task (tree or commutative reduction, Eq. 2)."""
    return k_b * (m_b + n_b) + m_b * n_b


def rel_frobenius(x, ref):
    """||x - ref||_F / ||ref||_F."""
    x = np.asarray(x, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    den = np.linalg.norm(ref.ravel())
    num = np.linalg.norm((x - ref).ravel())
    return float(num / den) if den > 0 else float(num)
