"""Seeded synthetic inputs for the blocked tensordot and circuit contractions.

This module is shared by the CPU oracle (``oracle/``) and the GPU library
(``paper_2201_06620_b300``).  It only *generates inputs*: random complex
tensors, random grid circuits (gate lists with their matrices), the tensor
network that describes an amplitude of such a circuit (tensors plus index
labels), and the fixed problem definitions of the benchmark workloads.  It
contains no contraction arithmetic of any kind: no tensordot, no gate
application, no sums over indices.

Conventions (the paper's statement of the problem, Sec. II-A):

* a quantum state of n qubits is an order-n tensor over C^2; qubit q is axis q
  of that tensor, so the row-major flat index of a basis state has qubit 0 as
  its most significant bit;
* a one-qubit gate is the order-2 tensor ``G[out, in]``;
* a two-qubit gate on qubits (q1, q2) is the order-4 tensor
  ``G[o1, o2, i1, i2]`` (the 4x4 matrix with row ``2*o1+o2`` and column
  ``2*i1+i2``).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "complex_normal", "complex_normal_range", "SQRT_X", "SQRT_Y", "SQRT_W", "HADAMARD", "CNOT",
    "fsim", "grid_shape", "grid_sites", "coupler_layer", "PATTERN",
    "Circuit", "random_circuit", "ghz_circuit", "hadamard_circuit",
    "circuit_network", "Network",
    "tensordot_single_config", "precision_sweep_config", "rqc20_config",
]


# ---------------------------------------------------------------------------
# random tensors
# ---------------------------------------------------------------------------
def complex_normal(shape, seed, scale=1.0, dtype=np.complex128):
    """i.i.d. standard complex normal entries: re, im ~ N(0, 1/2), E|z|^2 = 1.

    Drawn from numpy's PCG64 ``default_rng(seed)``: first all real parts,
    then all imaginary parts, in row-major order of ``shape``.
    """
    rng = np.random.default_rng(seed)
    shape = tuple(int(s) for s in shape)
    s = math.sqrt(0.5) * scale
    re = rng.standard_normal(shape) * s
    im = rng.standard_normal(shape) * s
    return (re + 1j * im).astype(dtype)


def complex_normal_range(seed, start, count, scale=1.0, dtype=np.complex64):
    """Entries [start, start + count) of a counter-addressable stream of i.i.d.
    complex normals (re, im ~ N(0, 1/2)), so that any piece of a tensor too
    large for host memory can be generated on its own.

    Entry e uses the 64-bit draws 2e and 2e+1 of numpy's PCG64(seed) as the
    doubles u1, u2 in [0, 1) (Generator.random) and the Box-Muller map
    z = sqrt(-ln(1 - u1)) * exp(2 pi i u2), so |z|^2 ~ Exp(1).
    """
    bg = np.random.PCG64(seed)
    bg.advance(2 * int(start))
    u = np.random.Generator(bg).random(2 * int(count))
    r = np.sqrt(-np.log1p(-u[0::2])) * scale
    th = 2.0 * np.pi * u[1::2]
    return (r * np.cos(th) + 1j * (r * np.sin(th))).astype(dtype)


# ---------------------------------------------------------------------------
# gate set (Sycamore-style random circuits, Sec. V)
# ---------------------------------------------------------------------------
_I2 = np.eye(2, dtype=np.complex128)
_X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_W = (_X + _Y) / math.sqrt(2.0)

#: (I - iP)/sqrt(2) = R_P(pi/2) for P in {X, Y, W}; each squares to -iP.
SQRT_X = (_I2 - 1j * _X) / math.sqrt(2.0)
SQRT_Y = (_I2 - 1j * _Y) / math.sqrt(2.0)
SQRT_W = (_I2 - 1j * _W) / math.sqrt(2.0)
HADAMARD = np.array([[1, 1], [1, -1]], dtype=np.complex128) / math.sqrt(2.0)
#: control = first qubit, target = second, as a G[o1,o2,i1,i2] 4x4 matrix
CNOT = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]],
                dtype=np.complex128)

_ONE_QUBIT = (("sqrt_x", SQRT_X), ("sqrt_y", SQRT_Y), ("sqrt_w", SQRT_W))


def fsim(theta, phi):
    """fSim(theta, phi) as a 4x4 matrix in the basis |00>,|01>,|10>,|11>."""
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[1, 0, 0, 0],
                     [0, c, -1j * s, 0],
                     [0, -1j * s, c, 0],
                     [0, 0, 0, complex(math.cos(phi), -math.sin(phi))]],
                    dtype=np.complex128)


FSIM = fsim(math.pi / 2, math.pi / 6)

#: coupler layer used by cycle t is PATTERN[t % 8]
PATTERN = "ABCDCDAB"


def grid_shape(n):
    """(rows, cols) of the grid for n qubits: rows = floor(sqrt n), cols = ceil(n/rows)."""
    rows = max(1, int(math.isqrt(n)))
    cols = -(-n // rows)
    return rows, cols


def grid_sites(n, rows, cols):
    """Qubit index of each (r, c) site, row-major; sites beyond n are absent."""
    return {(r, c): r * cols + c for r in range(rows) for c in range(cols)
            if r * cols + c < n}


def coupler_layer(letter, n, rows, cols):
    """Qubit pairs coupled by layer A, B, C or D on a rows x cols grid.

    A: horizontal (r,c)-(r,c+1) with c even;  B: horizontal with c odd;
    C: vertical (r,c)-(r+1,c) with r even;    D: vertical with r odd.
    """
    site = grid_sites(n, rows, cols)
    pairs = []
    for (r, c), q in sorted(site.items(), key=lambda kv: kv[1]):
        if letter in "AB":
            if (c % 2 == 0) == (letter == "A") and (r, c + 1) in site:
                pairs.append((q, site[(r, c + 1)]))
        else:
            if (r % 2 == 0) == (letter == "C") and (r + 1, c) in site:
                pairs.append((q, site[(r + 1, c)]))
    return pairs


@dataclass
class Circuit:
    """A gate list acting on |0...0>, plus the output bitstring of interest."""
    n: int
    gates: list = field(default_factory=list)   # (name, qubits tuple, matrix)
    bitstring: np.ndarray | None = None
    rows: int = 0
    cols: int = 0
    depth: int = 0
    seed: int | None = None


def random_circuit(n, depth, seed, rows=None, cols=None):
    """Random grid circuit: per cycle, a random gate from {sqrt X, sqrt Y, sqrt W}
    on every qubit (never the one that qubit had in the previous cycle), then
    fSim(pi/2, pi/6) on the couplers of layer PATTERN[t % 8].  The bitstring is
    drawn from the same generator after the gates.
    """
    if rows is None or cols is None:
        rows, cols = grid_shape(n)
    rng = np.random.default_rng(seed)
    circ = Circuit(n=n, rows=rows, cols=cols, depth=depth, seed=seed)
    prev = [-1] * n
    for t in range(depth):
        for q in range(n):
            while True:
                g = int(rng.integers(0, 3))
                if g != prev[q]:
                    break
            prev[q] = g
            name, mat = _ONE_QUBIT[g]
            circ.gates.append((name, (q,), mat.copy()))
        for q1, q2 in coupler_layer(PATTERN[t % 8], n, rows, cols):
            circ.gates.append(("fsim", (q1, q2), FSIM.reshape(2, 2, 2, 2).copy()))
    circ.bitstring = rng.integers(0, 2, n).astype(np.int64)
    return circ


def ghz_circuit(n):
    """H on qubit 0, then CNOT(q, q+1) down the chain: (|0..0> + |1..1>)/sqrt 2."""
    circ = Circuit(n=n)
    circ.gates.append(("h", (0,), HADAMARD.copy()))
    for q in range(n - 1):
        circ.gates.append(("cnot", (q, q + 1), CNOT.reshape(2, 2, 2, 2).copy()))
    circ.bitstring = np.zeros(n, dtype=np.int64)
    return circ


def hadamard_circuit(n):
    """H on every qubit: every amplitude is 2^(-n/2)."""
    circ = Circuit(n=n)
    for q in range(n):
        circ.gates.append(("h", (q,), HADAMARD.copy()))
    circ.bitstring = np.zeros(n, dtype=np.int64)
    return circ


# ---------------------------------------------------------------------------
# circuit -> tensor network (Sec. II-A)
# ---------------------------------------------------------------------------
@dataclass
class Network:
    """Tensors with integer index labels.

    A label that appears on two tensors is a bond (contracted); labels listed
    in ``out_labels`` stay open, in that order, in the result.  Every index
    has extent 2.
    """
    tensors: list
    labels: list
    out_labels: list


def circuit_network(circ, bitstring=None, open_output=False):
    """The network whose full contraction is <x|C|0^n> (or C|0^n> if open).

    Tensors, in order: the |0> vector of each qubit (rank 1), each gate in
    circuit order (rank 2 or rank 4, as ``G[out..., in...]``), then the <x_q|
    projector of each qubit (rank 1), unless ``open_output`` is set, in which
    case the final wire of qubit q is left open as output label number q.
    """
    n = circ.n
    if bitstring is None:
        bitstring = circ.bitstring
    next_label = 0
    wire = []
    tensors, labels = [], []
    for q in range(n):
        wire.append(next_label)
        tensors.append(np.array([1.0, 0.0], dtype=np.complex128))
        labels.append((next_label,))
        next_label += 1
    for _name, qs, mat in circ.gates:
        ins = [wire[q] for q in qs]
        outs = list(range(next_label, next_label + len(qs)))
        next_label += len(qs)
        tensors.append(np.asarray(mat, dtype=np.complex128).reshape((2,) * (2 * len(qs))))
        labels.append(tuple(outs + ins))
        for q, o in zip(qs, outs):
            wire[q] = o
    out_labels = []
    if open_output:
        out_labels = list(wire)
    else:
        for q in range(n):
            v = np.zeros(2, dtype=np.complex128)
            v[int(bitstring[q])] = 1.0
            tensors.append(v)
            labels.append((wire[q],))
    return Network(tensors=tensors, labels=labels, out_labels=out_labels)


# ---------------------------------------------------------------------------
# fixed benchmark problems
# ---------------------------------------------------------------------------
def _block_tensordot_problem(seed_a, seed_b, free_a, contracted, free_b,
                             grid_free_a, grid_contracted, grid_free_b,
                             perm_seed=None, scale=1.0, dtype=np.complex128,
                             materialise=True):
    """A pairwise problem on [2]^r tensors with a block grid.

    Logical axes before permutation: A = (free_a | contracted),
    B = (contracted | free_b).  The first ``grid_free_a`` free axes of A, the
    first ``grid_contracted`` contracted axes and the first ``grid_free_b``
    free axes of B get block extent 1 (they are grid axes of extent 2); every
    other axis has block extent 2.  With ``perm_seed`` both operands' axis
    orders are shuffled by a seeded permutation.
    """
    ra = free_a + contracted
    rb = contracted + free_b
    a_kind = [("f", i) for i in range(free_a)] + [("c", i) for i in range(contracted)]
    b_kind = [("c", i) for i in range(contracted)] + [("g", i) for i in range(free_b)]

    def blk(kind):
        t, i = kind
        if t == "f":
            return 1 if i < grid_free_a else 2
        if t == "g":
            return 1 if i < grid_free_b else 2
        return 1 if i < grid_contracted else 2

    if perm_seed is not None:
        rng = np.random.default_rng(perm_seed)
        pa = rng.permutation(ra)
        pb = rng.permutation(rb)
    else:
        pa = np.arange(ra)
        pb = np.arange(rb)
    a_kind = [a_kind[i] for i in pa]
    b_kind = [b_kind[i] for i in pb]
    axes_a = [a_kind.index(("c", i)) for i in range(contracted)]
    axes_b = [b_kind.index(("c", i)) for i in range(contracted)]
    prob = {
        "shape_a": (2,) * ra, "shape_b": (2,) * rb,
        "block_a": tuple(blk(k) for k in a_kind),
        "block_b": tuple(blk(k) for k in b_kind),
        "axes_a": axes_a, "axes_b": axes_b,
        "seed_a": seed_a, "seed_b": seed_b, "scale": scale,
    }
    if materialise:
        prob["a"] = complex_normal(prob["shape_a"], seed_a, scale, dtype)
        prob["b"] = complex_normal(prob["shape_b"], seed_b, scale, dtype)
    return prob


def tensordot_single_config(perm_seed=7, grid_free=2, grid_contracted=2):
    """Single blocked tensordot, complex128: A, B of shape [2]^14 in blocks of
    2^10 entries, 6 contracted indices, [2]^16 output.

    Each operand has 8 free and 6 contracted axes; ``grid_free`` free and
    ``grid_contracted`` contracted axes per operand are grid axes (block
    extent 1), so each operand block holds 2^10 entries and there are
    B_k = 2^grid_contracted block pairs per output block.  A seeded
    permutation shuffles both operands' axis orders.  Seeds 1 (A), 2 (B).
    """
    return _block_tensordot_problem(1, 2, 8, 6, 8, grid_free, grid_contracted,
                                    grid_free, perm_seed=perm_seed)


def precision_sweep_config(materialise=False, dtype=np.complex64):
    """One large pairwise contraction in the form U_mk V_nk: A, B of shape [2]^30,
    axes (20 free | 10 contracted) each, contracting the last 10 axes of both
    into a [2]^40 output; entries complex normal times 2^-15 (seeds 3, 4).

    Blocks hold 2^12 entries: block extent 2 on the last 6 free and the last 6
    contracted axes of each operand, extent 1 on the rest, so B_k = 16 and the
    output blocks hold 2^12 entries.  The output is produced in chunks of 2^30
    entries, one per value of A's first 10 free axes.
    """
    ra = 30
    block = tuple([1] * 14 + [2] * 6 + [1] * 4 + [2] * 6)
    prob = {
        "shape_a": (2,) * ra, "shape_b": (2,) * ra,
        "block_a": block, "block_b": block,
        "axes_a": list(range(20, 30)), "axes_b": list(range(20, 30)),
        "seed_a": 3, "seed_b": 4, "scale": 2.0 ** -15,
    }
    if materialise:
        prob["a"] = complex_normal(prob["shape_a"], 3, 2.0 ** -15, dtype)
        prob["b"] = complex_normal(prob["shape_b"], 4, 2.0 ** -15, dtype)
    return prob


def rqc20_config(seed=2022):
    """The 20-qubit 4x5 depth-12 random circuit of the amplitude workload."""
    return random_circuit(20, 12, seed, rows=4, cols=5)
