#!/usr/bin/env python3
"""Benchmark: amplitudes/s of a 20-qubit random circuit on one B300.

Workload (one step = one amplitude): the 4x5 grid, depth-12 random circuit
(sqrt X / sqrt Y / sqrt W layers, fSim(pi/2, pi/6) on couplers ABCDCDAB),
|0>^20 in, a seeded output bitstring per step, complex64, the library's greedy
min-size path, blocks of 2^8 entries on every intermediate of rank > 8,
contracted by rosnet_contract (grouped wave launches replayed as a CUDA
graph).  The circuit's gate tensors stay resident on the device; each step
binds the 20 projector tensors of its own bitstring.

Timing: W warm-up steps, then K steps each bracketed by CUDA events on the
launching stream, with a 256 MiB buffer rewritten between steps to flush the
126 MB L2; barrier + synchronize before and after.  Under torchrun every
rank runs its own replica on different bitstrings (no data-path collective);
rank 0 prints one JSON line with the whole-job value (sum over ranks of the
amplitudes over the slowest rank's time).

--impl reference runs the CPU oracle (plain complex128 loop contraction,
its own greedy path) on the same workload, on rank 0 only.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

N_QUBITS = 20
MAX_BLOCK = 256           # 2^8-entry blocks on every intermediate of rank > 8
WORKLOAD = "rqc20_4x5_d12_amplitude"
METRIC = "amplitudes/s"


def _env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def _bitstrings(seed, count):
    rng = np.random.default_rng(seed)
    return [rng.integers(0, 2, N_QUBITS) for _ in range(count)]


def _config(extra=None):
    cfg = {"workload": WORKLOAD, "qubits": N_QUBITS, "grid": "4x5", "depth": 12,
           "circuit_seed": 2022, "dtype": "complex64", "path": "greedy min-size",
           "max_block_entries": MAX_BLOCK, "per_step": "1 amplitude (1 bitstring)",
           "l2": "256 MiB buffer rewritten between timed steps"}
    if extra:
        cfg.update(extra)
    return cfg


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_rosnet(args):
    import torch
    import torch.distributed as dist

    import paper_2201_06620_b300 as R

    rank, world, local = _env_rank()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    circ = W.rqc20_config()
    net0 = W.circuit_network(circ)
    ngates = len(net0.tensors) - N_QUBITS
    # resident circuit: |0> vectors and gates; projectors per step
    leaves = [R.btensor(np.asarray(t, dtype=np.complex64)) for t in net0.tensors]
    net = R.Network(leaves, net0.labels, net0.out_labels)
    path = net.greedy_path()
    steps = args.warmup + args.steps
    bits = _bitstrings(1000 + rank, steps)
    proj = [[R.btensor(np.eye(2, dtype=np.complex64)[int(b)]) for b in bs] for bs in bits]
    flags = R.OPT_GRAPH | R.OPT_TIMING

    def bind(i):
        for q in range(N_QUBITS):
            net.set_tensor(ngates + q, proj[i][q])

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    outs = []
    for i in range(args.warmup):
        bind(i)
        outs.append(R.contract(net, path=path, flags=flags, max_block_entries=MAX_BLOCK))
    torch.cuda.synchronize()
    R.timing_drain()
    launches0 = R.kernel_launches()
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")
    wall0 = time.perf_counter()
    for i in range(args.warmup, steps):
        flush.random_(0, 255) if i == args.warmup else flush.fill_(i & 0xff)
        bind(i)
        starts[i].record(stream)
        outs.append(R.contract(net, path=path, flags=flags, max_block_entries=MAX_BLOCK))
        ends[i].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    torch.cuda.nvtx.range_pop()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    launches = R.kernel_launches() - launches0
    step_ms = [starts[i].elapsed_time(ends[i]) for i in range(args.warmup, steps)]
    heavy = R.timing_drain()
    amps = [complex(o.download()) for o in outs[args.warmup:]]
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * args.steps / (total_ms / 1e3)

    # roofline of the heaviest launch (FP32 FFMA, plain ALU bound)
    peaks = _measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    fp32_peak = 148 * 128 * 2 * sm_max * 1e6 / 1e12   # TFLOP/s: SMs x FP32 lanes x FMA
    hms = [h[0] for h in heavy]
    hflops = heavy[0][1] if heavy else 0.0
    hbytes = heavy[0][2] if heavy else 0.0
    h_avg = statistics.mean(hms) if hms else float("nan")
    achieved = hflops / (h_avg * 1e-3) / 1e12 if hms else None
    traffic = _profiled_traffic()
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": (achieved / fp32_peak) if achieved else None, "traffic": traffic,
                "kernel": "gett_tiled (heaviest grouped launch)", "launch_ms": h_avg,
                "flops_per_launch": hflops, "bytes_per_launch": hbytes,
                "peak_source": "148 SMs x 128 FP32 lanes x 2 flop x sm_max_mhz (MEASURED_PEAKS.json)"}

    e2e = run_e2e(args, R, torch, circ, net, path, ngates, stream) if not args.no_e2e else None
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(circ, bits[args.warmup:], args.cpu_seconds)
    # check: oracle-independent sanity (amplitudes are finite and not all equal)
    assert all(np.isfinite(a.real) and np.isfinite(a.imag) for a in amps)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "amplitudes/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64 (fp32)",
            "data": "synthetic (seeded random circuit and bitstrings)",
            "config": _config({"parallelism": f"replicas x{world}" if world > 1 else "single GPU"}),
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                           "p99": float(np.percentile(step_ms, 99))},
            "tensordot_tflops": achieved,
            "gpu_launches": launches,
            "wall_s": wall,
            "clocks": clk,
            "roofline": roofline,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_e2e(args, R, torch, circ, net, path, ngates, stream):
    """Same metric through the public API with host buffers: every step copies
    its 20 projector vectors from pinned host memory into device tensors,
    contracts, and reads the amplitude back to the host."""
    steps = args.warmup + args.steps
    bits = _bitstrings(5000, steps)
    host = []
    for bs in bits:
        hs = []
        for b in bs:
            t = torch.zeros(2, dtype=torch.complex64).pin_memory()
            t[int(b)] = 1.0
            hs.append(t)
        host.append(hs)
    dev_proj = [R.empty((2,), None, R.C64) for _ in range(N_QUBITS)]
    for q in range(N_QUBITS):
        net.set_tensor(ngates + q, dev_proj[q])
    out_host = torch.empty((), dtype=torch.complex64).pin_memory()
    flags = R.OPT_GRAPH
    h2d = N_QUBITS * 2 * 8
    t0 = None
    for i in range(steps):
        if i == args.warmup:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
        for q in range(N_QUBITS):
            dev_proj[q].upload(host[i][q])
        C = R.contract(net, path=path, flags=flags, max_block_entries=MAX_BLOCK)
        C.download(out_host)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return {"value": args.steps / dt, "unit": "amplitudes/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": 8,
            "what": "per step: 20 projector uploads from pinned host, rosnet_contract, amplitude download"}


# ---------------------------------------------------------------------------
# CPU baseline / reference arm: the oracle as it stands
# ---------------------------------------------------------------------------
def cpu_baseline(circ, bits, seconds):
    import oracle
    net = W.circuit_network(circ, bitstring=bits[0])
    path = oracle.greedy_path(net)
    n = 0
    t0 = time.perf_counter()
    while n < len(bits) and (n == 0 or time.perf_counter() - t0 < seconds):
        oracle.contract(W.circuit_network(circ, bitstring=bits[n]), path)
        n += 1
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "amplitudes/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{n} amplitudes of the same circuit (oracle complex128 loop contraction, "
                      f"oracle greedy path), {dt:.1f} s"}


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    import oracle
    circ = W.rqc20_config()
    bits = _bitstrings(1000, args.warmup + args.steps)
    net = W.circuit_network(circ, bitstring=bits[0])
    path = oracle.greedy_path(net)
    for i in range(args.warmup):
        oracle.contract(W.circuit_network(circ, bitstring=bits[i]), path)
    t0 = time.perf_counter()
    for i in range(args.warmup, args.warmup + args.steps):
        oracle.contract(W.circuit_network(circ, bitstring=bits[i]), path)
    dt = time.perf_counter() - t0
    value = args.steps / dt
    line = {"metric": METRIC, "value": value, "unit": "amplitudes/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128 (fp64)",
            "data": "synthetic (seeded random circuit and bitstrings)", "impl": "reference",
            "config": _config({"parallelism": "host cores"}),
            "cpu_baseline": {"value": value, "unit": "amplitudes/s", "cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": f"{args.steps} timed amplitudes after {args.warmup} warm-up"},
            "e2e": {"value": value, "unit": "amplitudes/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _profiled_traffic():
    """DRAM bytes per launch of the heaviest kernel from the committed ncu
    summary, or None when the kernel source changed since that capture."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)
        with open(os.path.join(ROOT, "paper_2201_06620_b300", "csrc", "gett.cu"), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
    except (OSError, ValueError):
        return None
    if not sha.startswith(rec.get("kernel_source_sha256_prefix", "-")):
        return None
    return rec.get("gett_tiled_rqc20_bytes_per_launch")


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["rosnet", "reference"], default="rosnet")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_rosnet(args)


if __name__ == "__main__":
    main()
