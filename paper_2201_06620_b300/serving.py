"""Amplitude serving with continuous batching on one GPU.

A query asks for amplitudes <x|C|0^n> of one registered circuit for 1 to
1024 bitstrings x that share their first n - k bits (k <= 10): the network
keeps the last k output wires open, so one contraction gives all 2^k
amplitudes of the query (its intermediates serve every requested bitstring)
and the requested ones are read from that result.  Everything that runs on
the device is rosnet_contract (librosnet's kernels); this module schedules.

Scheduling: queries wait in arrival order; a query is admitted as soon as a
stream slot is free and the device memory it needs fits the budget next to
what is already held.  Each stream keeps one plan per (circuit, k) (offset
tables, intermediate arena, captured CUDA graph) and a device buffer of
projectors, so a query costs one small host-to-device copy (its prefix), one
graph launch and one device-to-host copy (its amplitudes).  The budget
counts every resident plan (its device bytes as the library reports them;
before a plan exists, its predicted footprint: input tensors plus the peak
of live intermediates along the path -- the analogue of the paper's
per-task memory, Eq. 1 / Eq. 2) and the outputs of running queries.  When a
query needs a new plan that does not fit, resident plans that no running
query uses are spilled to pinned host memory, least recently used first
(rosnet_plan_spill: their device memory is released and their offset tables
kept in page-locked host memory, so a later query restores the plan instead
of planning it anew; spilled plans beyond a host budget are freed, oldest
first); if it still does not fit it waits for running queries to retire (a
query alone is always admitted).
Admitted queries run concurrently on separate streams, so a query that
arrives while others are on the GPU starts as soon as a slot and memory free
up, and its kernels overlap theirs.  Latency runs from a query's arrival to
the moment its amplitudes are on the host.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass

import numpy as np

from . import (C64, OPT_GRAPH, PREC_DEFAULT, Network, btensor, contract, empty, path_search, plan_info,
               plan_release, plan_spill, simplify)


@dataclass
class _Plan:
    tensors: list      # circuit tensors (as given or simplified); projectors follow
    labels: list
    out: list
    path: list
    flops: float
    footprint: float
    sig: tuple = ()    # what the library keys its cached plan by (with the slot's stream):
                       # equal signatures share one plan

__all__ = ["Query", "AmplitudeServer", "predict_footprint"]


@dataclass
class Query:
    circuit: int
    prefix: tuple            # bits of qubits 0 .. n-k-1
    k: int                   # open (trailing) qubits
    suffixes: list           # requested values of the open qubits (ints < 2^k)
    arrival: float = 0.0
    started: float | None = None
    done: float | None = None
    result: np.ndarray | None = None
    qid: int = 0


def predict_footprint(labels, extents, out_labels, path, elem_bytes=8):
    """Device bytes of a contraction: inputs plus the largest total of live
    intermediates along the path (each lives from its step to its use)."""
    ext = {}
    for l, e in zip(labels, extents):
        for x, v in zip(l, e):
            ext[x] = v
    n = len(labels)
    live = {i: list(l) for i, l in enumerate(labels)}
    size = {i: math.prod(ext[x] for x in l) for i, l in enumerate(labels)}
    inputs = sum(size.values())
    nxt, cur, peak = n, 0, 0
    for a, b in path:
        la, lb = live.pop(a), live.pop(b)
        sh = set(la) & set(lb)
        lc = [x for x in la if x not in sh] + [x for x in lb if x not in sh]
        s = math.prod(ext[x] for x in lc) if lc else 1
        cur += s
        peak = max(peak, cur)
        for o in (a, b):
            if o >= n:
                cur -= size[o]
        live[nxt], size[nxt] = lc, s
        nxt += 1
    return elem_bytes * (inputs + peak)


class _Circuit:
    """Device-resident tensors of one circuit and its per-k paths.  The
    circuit part (|0> vectors and gates, final wires open) is also simplified
    once on registration: every rank-1 and rank-2 tensor absorbed into a
    neighbour on the device (rosnet_simplify), about one tensor per two-qubit
    gate.  For each k the path is searched on both forms, with the query's
    projectors on the closed wires, and the cheaper one is used."""

    def __init__(self, cid, circ):
        self.cid, self.n = cid, circ.n
        zero = np.array([1, 0], dtype=np.complex64)
        self.tensors = [btensor(zero) for _ in range(circ.n)]
        self.labels = [(q,) for q in range(circ.n)]
        wire, nl = list(range(circ.n)), circ.n
        for _, qs, mat in circ.gates:
            outs = list(range(nl, nl + len(qs)))
            nl += len(qs)
            self.tensors.append(btensor(np.asarray(mat, dtype=np.complex64)))
            self.labels.append(tuple(outs + [wire[q] for q in qs]))
            for q, o in zip(qs, outs):
                wire[q] = o
        self.wire = wire
        st, sl, _ = simplify(self.tensors, self.labels, out_labels=wire)
        self.forms = [(self.tensors, self.labels)] + ([(st, sl)] if len(st) < len(self.tensors) else [])
        self.per_k = {}

    def plan_for(self, k):
        if k not in self.per_k:
            closed = self.n - k
            out = [self.wire[q] for q in range(closed, self.n)]
            best = None
            for tensors, labels in self.forms:
                labels = list(labels) + [(self.wire[q],) for q in range(closed)]
                ext = [t.shape for t in tensors] + [(2,)] * closed
                path, flops = path_search(labels, ext, out, ntrials=16, seed=self.cid)
                if best is None or flops < best.flops:
                    best = _Plan(tensors, labels, out, path, flops, predict_footprint(labels, ext, out, path))
            best.sig = (tuple(map(tuple, best.labels)), tuple(tuple(t.shape) for t in best.tensors),
                        tuple(tuple(t.block_shape) for t in best.tensors), tuple(best.out),
                        tuple(map(tuple, best.path)))
            self.per_k[k] = best
        return self.per_k[k]


class _Slot:
    """One stream with its projector buffer (views per qubit) and networks."""

    def __init__(self, torch, nmax):
        self.stream = torch.cuda.Stream()
        self.buf = empty((nmax, 2), None, C64, stream=self.stream)
        self.views = [self.buf.fix([0], [q]) for q in range(nmax)]
        self.nets = {}
        self.host = np.zeros((nmax, 2), dtype=np.complex64)


class AmplitudeServer:
    """Continuous-batching amplitude server over a pool of stream slots."""

    def __init__(self, circuits, slots=4, memory_budget=160e9, precision=PREC_DEFAULT, use_graph=True,
                 spill=True, host_budget=64e9):
        import torch
        self.torch = torch
        self.circuits = [_Circuit(i, c) for i, c in enumerate(circuits)]
        nmax = max(c.n for c in self.circuits)
        self.slots = [_Slot(torch, nmax) for _ in range(slots)]
        self.free = list(range(slots))
        self.budget = memory_budget
        # resident plans: (slot, plan signature) -> device bytes, least recently
        # used first.  Circuits of equal structure and path share one plan in
        # the library's cache, so it is counted and released once
        self.resident = collections.OrderedDict()
        self.resident_bytes = 0.0
        self.in_use = 0.0          # outputs of running queries
        self.evictions = 0
        # plans spilled to pinned host memory: (slot, signature) -> host bytes, oldest first
        self.spill, self.host_budget = spill, host_budget
        self.spilled = collections.OrderedDict()
        self.spilled_bytes = 0.0
        self.restores = 0
        self.precision = precision
        self.flags = OPT_GRAPH if use_graph else 0
        self.waiting = collections.deque()
        self.running = []
        self.finished = []
        self._qid = 0

    @property
    def device_bytes(self):
        """Device memory the server accounts for: resident plans and running outputs."""
        return self.resident_bytes + self.in_use

    def submit(self, q: Query, now=None):
        q.arrival = time.perf_counter() if now is None else now
        q.qid = self._qid
        self._qid += 1
        self.waiting.append(q)

    def step(self):
        """Retire finished queries, then admit waiting ones while a slot is
        free and the memory they need fits the budget (freeing idle resident
        plans, least recently used first, to make room)."""
        self._retire()
        while self.waiting and self.free:
            q = self.waiting[0]
            si = self.free[-1]
            key = self._key(si, q)
            need = 8.0 * 2 ** q.k + (0.0 if key in self.resident else self.circuits[q.circuit].plan_for(q.k).footprint)
            if self.device_bytes + need > self.budget:
                busy = {self._key(r[1], r[0]) for r in self.running}
                for victim in [k for k in self.resident if k not in busy and k != key]:
                    if self.device_bytes + need <= self.budget:
                        break
                    self._evict(victim)
            if self.running and self.device_bytes + need > self.budget:
                break
            self.waiting.popleft()
            self._launch(q, key)

    def drain(self):
        while self.waiting or self.running:
            self.step()
            if self.running:
                self.running[0][2].synchronize()
        self._retire()

    def _key(self, si, q):
        return (si, self.circuits[q.circuit].plan_for(q.k).sig)

    def _users(self, key):
        si, sig = key
        return [ck for ck in self.slots[si].nets if self.circuits[ck[0]].plan_for(ck[1]).sig == sig]

    def _evict(self, key):
        """Free the device memory of an idle resident plan: spill it to
        pinned host memory (or release it when spilling is off)."""
        si, _ = key
        sl = self.slots[si]
        ci, k = self._users(key)[0]
        self.resident_bytes -= self.resident.pop(key)
        self.evictions += 1
        if not self.spill:
            self._release(key)
            return
        hb = plan_spill([sl.nets[(ci, k)]], [self.circuits[ci].plan_for(k).path], precision=self.precision,
                        flags=self.flags, stream=sl.stream)
        self.spilled[key] = float(hb)
        self.spilled_bytes += float(hb)
        while self.spilled_bytes > self.host_budget and self.spilled:
            old = next(iter(self.spilled))
            self.spilled_bytes -= self.spilled.pop(old)
            self._release(old)

    def _release(self, key):
        si, _ = key
        sl = self.slots[si]
        users = self._users(key)
        nets = [sl.nets.pop(ck) for ck in users]
        ci, k = users[0]
        plan_release([nets[0]], [self.circuits[ci].plan_for(k).path], precision=self.precision, flags=self.flags,
                     stream=sl.stream)

    def _launch(self, q, key):
        torch = self.torch
        si = key[0]
        self.free.remove(si)
        sl = self.slots[si]
        c = self.circuits[q.circuit]
        pl = c.plan_for(q.k)
        path = pl.path
        closed = c.n - q.k
        if (q.circuit, q.k) not in sl.nets:
            sl.nets[(q.circuit, q.k)] = Network(list(pl.tensors) + sl.views[:closed], pl.labels, pl.out)
        net = sl.nets[(q.circuit, q.k)]
        pre = np.asarray(q.prefix, dtype=np.float32)
        sl.host[:closed, 0] = 1.0 - pre
        sl.host[:closed, 1] = pre
        q.started = time.perf_counter()
        sl.buf.upload(sl.host, stream=sl.stream)
        res = contract(net, path=path, precision=self.precision, flags=self.flags, stream=sl.stream)
        if key in self.resident:
            self.resident.move_to_end(key)
        else:   # the plan now exists (built, or restored from host memory): account for it
            if key in self.spilled:
                self.spilled_bytes -= self.spilled.pop(key)
                self.restores += 1
            nbytes = float(plan_info([net], [path], precision=self.precision, flags=self.flags,
                                     stream=sl.stream)[4])
            self.resident[key] = nbytes
            self.resident_bytes += nbytes
        ev = torch.cuda.Event()
        ev.record(sl.stream)
        out_bytes = 8.0 * 2 ** q.k
        self.in_use += out_bytes
        self.running.append((q, si, ev, res, out_bytes))
        # a plan larger than predicted: free idle plans until the budget holds
        if self.device_bytes > self.budget:
            busy = {self._key(r[1], r[0]) for r in self.running}
            for victim in [k for k in self.resident if k not in busy]:
                if self.device_bytes <= self.budget:
                    break
                self._evict(victim)

    def _retire(self):
        keep = []
        for q, si, ev, res, out_bytes in self.running:
            if ev.query():
                amps = res.download(stream=self.slots[si].stream).reshape(-1)
                q.result = amps[np.asarray(q.suffixes, dtype=np.int64)]
                q.done = time.perf_counter()
                self.in_use -= out_bytes
                self.free.append(si)
                self.finished.append(q)
            else:
                keep.append((q, si, ev, res, out_bytes))
        self.running = keep
