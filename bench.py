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
# kernel family of the heaviest launch (rosnet_timing_drain kinds)
KERNEL_NAMES = {
    2: "gett_tiled_kernel 64x64 (offset-table gathers, FFMA)",
    3: "gett_tiled_kernel 128x64 (offset-table gathers, FFMA)",
    10: "f32_gemm_kernel (TMA-fed FFMA 64x64x32, two k sets of 8x4-output threads; dense operands read in "
        "place; stream-K when tiles load the SMs unevenly; 128x16 tiles with a split contraction for few "
        "columns)",
    5: "tc_gemm_kernel TF32 (tcgen05)", 6: "tc_gemm_kernel 3xTF32 (tcgen05)", 7: "tc_gemm_kernel 3xBF16 (tcgen05)",
}
METRIC = "amplitudes/s"


def _env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def _whole_job(local_ms, steps, world, device=None):
    """Replicas: every rank timed `steps` amplitudes of its own bitstrings in
    local_ms; the job's time is the slowest rank's, its throughput all ranks'
    amplitudes over that time.  Returns (max_ms, amplitudes/s)."""
    total_ms = float(local_ms)
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, world * steps / (total_ms / 1e3)


def _bitstrings(seed, count):
    rng = np.random.default_rng(seed)
    return [rng.integers(0, 2, N_QUBITS) for _ in range(count)]


def _config(extra=None):
    cfg = {"workload": WORKLOAD, "qubits": N_QUBITS, "grid": "4x5", "depth": 12,
           "circuit_seed": 2022, "dtype": "complex64", "path": "greedy min-size",
           "max_block_entries": MAX_BLOCK, "per_step": "1 amplitude (1 bitstring)",
           "kernel_choice": "autotuned when planning (warm-up)",
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
                 "--format=csv,noheader,nounits", "-lms", "50"],
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
    # the output projectors are the rows of one device buffer (fixed
    # addresses: the plan's descriptors never change); every step's projector
    # values (real plane one-hot per qubit, imaginary plane zero) are resident
    # in HBM before the timed region, and a step copies its row of that table
    # into the buffer (one 320-byte device-to-device copy) before contracting
    pbuf = R.empty((N_QUBITS, 2), None, R.C64)
    prow = [pbuf.fix([0], [q]) for q in range(N_QUBITS)]
    for q in range(N_QUBITS):
        net.set_tensor(ngates + q, prow[q])
    ptab_h = np.zeros((steps, 2, N_QUBITS, 2), dtype=np.float32)
    ptab_h[np.arange(steps)[:, None], 0, np.arange(N_QUBITS)[None, :], np.asarray(bits)] = 1.0
    ptab = torch.from_numpy(ptab_h.reshape(steps, -1)).to(dev)
    flags = R.OPT_GRAPH | R.OPT_TIMING | (0 if args.no_autotune else R.OPT_AUTOTUNE)
    if args.tune_file and os.path.exists(args.tune_file):
        with open(args.tune_file) as f:
            R.tune_import(f.read())          # kernel choices of an earlier run

    def bind(i):
        pbuf.upload_raw(ptab[i], stream=stream)

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    outs = []
    for i in range(args.warmup):
        bind(i)
        outs.append(R.contract(net, path=path, flags=flags, max_block_entries=MAX_BLOCK))
    torch.cuda.synchronize()
    R.timing_drain()
    if args.tune_file:
        with open(args.tune_file, "w") as f:
            f.write(R.tune_export())
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
    total_ms, value = _whole_job(sum(step_ms), args.steps, world, dev)

    # roofline of the heaviest launch (FP32 FFMA, plain ALU bound)
    peaks = _measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = sms * 128 * 2 * sm_max * 1e6 / 1e12   # TFLOP/s: SMs x FP32 lanes x FMA
    hms = [h[0] for h in heavy]
    hflops = heavy[0][1] if heavy else 0.0
    hbytes = heavy[0][2] if heavy else 0.0
    hkind = heavy[0][3] if heavy else -1
    h_avg = statistics.mean(hms) if hms else float("nan")
    h_whole = statistics.mean([h[4] for h in heavy]) if heavy else float("nan")
    achieved = hflops / (h_avg * 1e-3) / 1e12 if hms else None
    achieved_whole = hflops / (h_whole * 1e-3) / 1e12 if hms else None
    traffic = _profiled_traffic(hkind)
    probed = probe_peaks(R, torch, dev) if not args.no_probes else None
    ffma = probed["fp32_ffma_tflops"] if probed else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": (achieved / fp32_peak) if achieved else None, "traffic": traffic,
                "kernel": KERNEL_NAMES.get(hkind, f"kind {hkind}"), "launch_ms": h_avg,
                "flops_per_launch": hflops, "bytes_per_launch": hbytes,
                "peak_source": f"{sms} SMs (queried) x 128 FP32 lanes x 2 flop x sm_max_mhz "
                               "(MEASURED_PEAKS.json)",
                "launch_ms_with_packs": h_whole, "achieved_with_packs": achieved_whole,
                "frac_with_packs": (achieved_whole / fp32_peak) if achieved_whole else None,
                "peak_probed_ffma": ffma,
                "frac_of_probed_ffma": (achieved / ffma) if (achieved and ffma) else None}

    others = None
    if not args.no_precision_modes:
        others = run_precision_modes(args, R, torch, net, path, bind, amps, flush, stream, flags)
    e2e = run_e2e(args, R, torch, circ, net, path, ngates, stream) if not args.no_e2e else None
    extras = None if args.no_extras else run_extras(R, torch, dev, probed, args)
    cpu, ref_amps = None, []
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, ref_amps = cpu_baseline(circ, bits[args.warmup:], args.cpu_seconds)
    assert all(np.isfinite(a.real) and np.isfinite(a.imag) for a in amps)
    # parity of the timed amplitudes against the oracle's, on the bitstrings
    # the CPU baseline contracted: |a - a_ref| / max(|a_ref|, 2^-n/2)
    parity = None
    if ref_amps:
        floor = 2.0 ** (-N_QUBITS / 2)
        err = max(abs(a - r) / max(abs(r), floor) for a, r in zip(amps, ref_amps))
        parity = {"max_rel_err_vs_oracle": err, "amplitudes_checked": len(ref_amps), "bar": 1e-5,
                  "ok": bool(err <= 1e-5)}
        if others:
            for o in others.values():
                got = o.pop("_amps", None)
                if got:
                    m = min(len(got), len(ref_amps))
                    e = max(abs(a - r) / max(abs(r), floor) for a, r in zip(got[:m], ref_amps[:m]))
                    o["max_rel_err_vs_oracle"] = e
                    o["oracle_checked"] = m
                    o["within_1e-5_vs_oracle"] = bool(e <= 1e-5)
    if others:
        for o in others.values():
            o.pop("_amps", None)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "amplitudes/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64 (fp32)",
            "data": "synthetic (seeded random circuit and bitstrings)",
            "config": _config({"parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                               "step_input": "every step's 20 projector vectors resident in HBM; a step "
                                             "copies its own (320 B, device to device) into the "
                                             "network's projector rows, then contracts"}),
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                           "p99": float(np.percentile(step_ms, 99))},
            "tensordot_tflops": achieved,
            "gpu_launches": launches,
            "wall_s": wall,
            "clocks": clk,
            "roofline": roofline,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "parity": parity,
            "peaks_probed": probed,
            "other_precisions": others,
            "extras": extras,
        }
        print(json.dumps(line), flush=True)
        if parity is not None and not parity["ok"]:
            sys.exit(f"amplitudes differ from the oracle by {parity['max_rel_err_vs_oracle']:.3g} > 1e-5")
    if world > 1:
        dist.destroy_process_group()


def probe_peaks(R, torch, dev):
    """Peak rates measured on this GPU: the library's FP32 FFMA, FP64 DFMA and
    tcgen05 TF32 / BF16 MMA probes (each launched once to warm up, once timed),
    and page-locked host <-> device copy bandwidth (three 1 GiB copies each
    way after a warm-up copy, CUDA events)."""
    out = {}
    for key, kind in (("fp32_ffma_tflops", R.PROBE_FFMA), ("fp64_dfma_tflops", R.PROBE_DFMA),
                      ("tf32_tcgen05_tflops", R.PROBE_TF32), ("bf16_tcgen05_tflops", R.PROBE_BF16)):
        try:
            out[key] = R.probe_peak(kind)[0]
        except Exception as e:   # reported, not fatal to the line
            out[key] = None
            out[key + "_error"] = str(e)[:160]
    n = 1 << 30
    h = torch.empty(n, dtype=torch.uint8).pin_memory()
    d = torch.empty(n, dtype=torch.uint8, device=dev)
    for name, dst, src in (("h2d_gbs", d, h), ("d2h_gbs", h, d)):
        dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            dst.copy_(src, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        out[name] = 3 * n / (e0.elapsed_time(e1) * 1e-3) / 1e9
    del h, d
    return out


def _net_labels(rank_a, rank_b, axes_a, axes_b):
    """Labels of a two-tensor network equal to tensordot(A, B, (axes_a, axes_b))."""
    la = list(range(rank_a))
    lb = [1000 + j for j in range(rank_b)]
    for x, y in zip(axes_a, axes_b):
        lb[y] = la[x]
    out = [la[i] for i in range(rank_a) if i not in axes_a] + [lb[j] for j in range(rank_b) if j not in axes_b]
    return [la, lb], out


def _timed_contract(R, torch, ts, labels, out, precision, reps, path=((0, 1),)):
    """Plan (graph, timing) once, then `reps` replays: (ms per call from
    events around the calls, [(gemm ms, flops, bytes, kind, whole ms)])."""
    fl = R.OPT_GRAPH | R.OPT_TIMING
    path = [tuple(p) for p in path]
    for _ in range(2):
        C = R.contract(ts, labels, out, path, precision=precision, flags=fl)
        del C
    torch.cuda.synchronize()
    R.timing_drain()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        C = R.contract(ts, labels, out, path, precision=precision, flags=fl)
        del C
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, R.timing_drain()


def run_extras(R, torch, dev, probed, args=None):
    """Measurements beside the headline, each against the probed peak of its
    arithmetic: (1) the single blocked FP64 tensordot ([2]^14 x [2]^14 in
    2^10-entry blocks, 6 contracted axes, complex128); (2) the precision
    sweep's chunk contraction ([2]^20 x [2]^30 -> [2]^30: M = 2^10, N = 2^20,
    K = 2^10, complex64, 2^12-entry blocks, entries ~ 2^-15 complex normal from
    a seeded device generator) in every precision mode, GEMM kernel alone and
    with its operand packs; (3) gates on a [2]^28 state against the HBM rate;
    (4) the out-of-core tier with the large operand streamed from host memory;
    (5) the serving stream (16 circuits, 10 s) and (6) the batched plan (256
    slices of a 30-qubit circuit + 64 circuits), in short form."""
    probed = probed or {}
    out = {}
    try:
        prob = W.tensordot_single_config()
        A = R.btensor(prob["a"], prob["block_a"], R.C128)
        B = R.btensor(prob["b"], prob["block_b"], R.C128)
        labels, ol = _net_labels(14, 14, prob["axes_a"], prob["axes_b"])
        ms, recs = _timed_contract(R, torch, [A, B], labels, ol, R.PREC_DEFAULT, 20)
        flop = 8.0 * 2 ** 8 * 2 ** 8 * 2 ** 6
        gemm = statistics.mean(r[0] for r in recs)
        peak = probed.get("fp64_dfma_tflops")
        out["fp64_blocked_tensordot"] = {
            "shape": "[2]^14 x [2]^14 -> [2]^16, blocks 2^10, B_k = 4, complex128", "flop": flop,
            "call_ms": ms, "gemm_kernel_ms": gemm, "tflops": flop / (ms * 1e-3) / 1e12,
            "gemm_tflops": flop / (gemm * 1e-3) / 1e12, "peak_probed_dfma": peak,
            "frac_of_probed_dfma": (flop / (ms * 1e-3) / 1e12 / peak) if peak else None,
            "what": "call_ms: events around rosnet_contract of the cached two-tensor plan (graph replay: "
                    "GEMM, split-K sum, descriptor patch); gemm_kernel_ms: the GEMM launch alone"}
        del A, B
        R.release_plans()
    except Exception as e:
        out["fp64_blocked_tensordot"] = {"error": str(e)[:200]}
    try:
        prob = W.precision_sweep_config()
        As = R.empty((2,) * 20, prob["block_a"][10:], R.C64)
        B = R.empty(prob["shape_b"], prob["block_b"], R.C64)
        g = torch.Generator(device=dev)
        for t, seed in ((As, prob["seed_a"]), (B, prob["seed_b"])):
            g.manual_seed(seed)
            raw = torch.randn(2 * t.numel, device=dev, generator=g) * (prob["scale"] * 0.5 ** 0.5)
            t.upload_raw(raw)
            torch.cuda.synchronize()
            del raw
        labels, ol = _net_labels(20, 30, list(range(10, 20)), prob["axes_b"])
        flop = 8.0 * 2 ** 10 * 2 ** 20 * 2 ** 10
        rows = {}
        for name, prec, issued, pk in (("fp32", R.PREC_FP32, 1, "fp32_ffma_tflops"),
                                       ("tf32", R.PREC_TF32, 1, "tf32_tcgen05_tflops"),
                                       ("tf32x3", R.PREC_TF32X3, 3, "tf32_tcgen05_tflops"),
                                       ("bf16x3", R.PREC_BF16X3, 3, "bf16_tcgen05_tflops")):
            ms, recs = _timed_contract(R, torch, [As, B], labels, ol, prec, 3)
            gemm = statistics.mean(r[0] for r in recs)
            whole = statistics.mean(r[4] for r in recs)
            tf, tfw = flop / (gemm * 1e-3) / 1e12, flop / (whole * 1e-3) / 1e12
            peak = probed.get(pk)
            rows[name] = {"gemm_kernel_ms": gemm, "with_packs_ms": whole, "call_ms": ms,
                          "tflops": tf, "tflops_with_packs": tfw, "issued_tflops": tf * issued,
                          "peak_probed": peak, "peak_kind": pk,
                          "frac_issued_of_probed": (tf * issued / peak) if peak else None,
                          "frac_issued_with_packs": (tfw * issued / peak) if peak else None,
                          "kernel_kind": recs[0][3] if recs else None}
            R.release_plans()
        out["sweep_chunk"] = {"shape": "M = 2^10, N = 2^20, K = 2^10 complex64 (2^12-entry blocks, B_k = 16)",
                              "flop": flop, "modes": rows}
        del As, B
        R.release_plans()
    except Exception as e:
        out["sweep_chunk"] = {"error": str(e)[:200]}
    try:
        out["gates_hbm"] = run_gate_extras(R, torch, dev)
    except Exception as e:
        out["gates_hbm"] = {"error": str(e)[:200]}
    try:
        out["ooc_operand"] = run_ooc_extras(R, torch, dev)
    except Exception as e:
        out["ooc_operand"] = {"error": str(e)[:200]}
    if args is None:
        return out
    # the serving and batch workloads in short form, so that every run of the
    # default line carries them (their own workloads print the full lines)
    try:
        sa = argparse.Namespace(**vars(args))
        sa.pool, sa.duration, sa.plain_sample, sa.no_cpu_baseline = 16, 10.0, 8, True
        line = run_serve(sa, emit=False)
        out["serve"] = {k: line[k] for k in ("value", "unit", "config", "queries", "amplitudes", "wall_s",
                                             "warmup_s", "latency_ms", "plain_fp32_per_query",
                                             "max_rel_err_vs_plain_fp32", "evictions")}
        R.release_plans()
    except Exception as e:
        out["serve"] = {"error": str(e)[:200]}
    try:
        ba = argparse.Namespace(**vars(args))
        ba.steps = 3
        line = run_batch(ba, emit=False)
        out["batch"] = {k: line[k] for k in ("workload", "tensors_30q_given_used", "small_circuits_simplified",
                                             "path_gflop", "sliced_gflop", "modes")}
        R.release_plans()
    except Exception as e:
        out["batch"] = {"error": str(e)[:200]}
    return out


def run_ooc_extras(R, torch, dev, chunks=3):
    """The out-of-core tier with the large operand in host memory, on the
    weak-scaling contraction U_mk V_nk of Sec. V-A scaled down 4x per block
    dimension (m_b = n_b = 2^12, k_b = 2^11; B_m = 8, B_n = 6, B_k = 16): U
    (8 GiB, complex64) stays in pinned host memory and each output chunk (one
    m-block row, 4096 x 24576) streams its 1 GiB slice of U in on a side
    stream while the previous chunk computes; chunks go out to pinned host
    memory.  Timed against the same chunks with U resident on the device:
    equal times mean the copies are hidden."""
    mb, nb, kb, Bm, Bn, Bk = 4096, 4096, 2048, 8, 6, 16
    shape_u, block_u = (Bm, mb, Bk * kb), (1, mb, kb)
    V = R.empty((Bn * nb, Bk * kb), (nb, kb), R.C64)
    U = R.empty(shape_u, block_u, R.C64)
    g = torch.Generator(device=dev)
    for t, seed in ((U, 31), (V, 32)):
        g.manual_seed(seed)
        raw = torch.randn(2 * t.numel, device=dev, generator=g) * 0.5 ** 0.5
        t.upload_raw(raw)
        torch.cuda.synchronize()
        del raw
    u_host = torch.empty(2 * U.numel * 4, dtype=torch.uint8).pin_memory()
    U.download_raw(u_host)
    torch.cuda.synchronize()
    chunk_bytes = 2 * mb * Bn * nb * 4
    host = torch.empty(2 * chunk_bytes, dtype=torch.uint8).pin_memory()
    flop = 8.0 * mb * (Bn * nb) * (Bk * kb) * chunks
    R.tensordot_ooc(U, V, [2], [1], 1, 0, 1, host)            # warm-up (plans, packs)
    R.tensordot_ooc_host(u_host, shape_u, block_u, V, [2], [1], 1, 0, 1, host)
    torch.cuda.synchronize()
    res = {}
    for name in ("device", "host"):
        t0 = time.perf_counter()
        if name == "device":
            R.tensordot_ooc(U, V, [2], [1], 1, 1, chunks, host)
        else:
            R.tensordot_ooc_host(u_host, shape_u, block_u, V, [2], [1], 1, 1, chunks, host)
        torch.cuda.synchronize()
        res[name] = time.perf_counter() - t0
    slice_bytes = 2 * mb * Bk * kb * 4
    del U, V, u_host, host
    R.release_plans()
    return {"shape": "U (8 x 4096, 16 x 2048) x V (6 x 4096, 16 x 2048) complex64, blocks (4096, 2048)",
            "chunks": chunks, "chunk": "4096 x 24576 (768 MiB out), U slice 1 GiB in",
            "s_u_on_device": res["device"], "s_u_in_host": res["host"],
            "tflops_u_in_host": flop / res["host"] / 1e12, "tflops_u_on_device": flop / res["device"] / 1e12,
            "copy_hidden_frac": res["device"] / res["host"],
            "h2d_gbs_needed": slice_bytes * chunks / res["host"] / 1e9,
            "what": "wall time of rosnet_tensordot_ooc (U resident) and rosnet_tensordot_ooc_host (U streamed "
                    "from pinned host) over the same chunks, output chunks to pinned host in both"}


def run_gate_extras(R, torch, dev, rank=28):
    """Memory-bound contractions: one- and two-qubit gates applied along axes
    of a [2]^28 complex64 tensor (2 GiB; entries from a seeded device
    generator), each a single planned step whose kernel time is the timed
    heavy launch.  Algorithmic bytes: the tensor read once, the result written
    once (the gate's 32 or 128 bytes aside), against the measured HBM copy
    bandwidth."""
    peak = float(_measured_peaks().get("hbm_gbs", 6465.2))
    T = R.empty((2,) * rank, None, R.C64)
    g = torch.Generator(device=dev)
    g.manual_seed(28)
    raw = torch.randn(2 * T.numel, device=dev, generator=g) * 0.5 ** 0.5
    T.upload_raw(raw)
    torch.cuda.synchronize()
    del raw
    rng = np.random.default_rng(5)
    rows = {}
    labels_t = list(range(rank))
    for name, axes, first in (("1q_axis13_out_last", (13,), False), ("1q_axis13_out_first", (13,), True),
                              ("2q_axes9_20_out_last", (9, 20), False)):
        q = len(axes)
        gm = (rng.standard_normal((2,) * (2 * q)) + 1j * rng.standard_normal((2,) * (2 * q))).astype(np.complex64)
        G = R.btensor(gm)
        outs = [200 + i for i in range(q)]
        rest = [x for x in labels_t if x not in axes]
        lab = [labels_t, outs + list(axes)]
        out_l = outs + rest if first else rest + outs
        ms, recs = _timed_contract(R, torch, [T, G], lab, out_l, R.PREC_DEFAULT, 5,
                                   path=[(1, 0)] if first else [(0, 1)])
        kern = statistics.mean(r[0] for r in recs)
        nbytes = 2 * T.numel * 8 + gm.size * 8
        gbs = nbytes / (kern * 1e-3) / 1e9
        rows[name] = {"kernel_ms": kern, "call_ms": ms, "bytes": nbytes, "achieved_gbs": gbs,
                      "peak_gbs": peak, "frac_of_measured_hbm": gbs / peak,
                      "kernel_kind": recs[0][3] if recs else None}
        del G
        R.release_plans()
    del T
    return {"tensor": "[2]^28 complex64 (2 GiB)", "rows": rows}


def run_precision_modes(args, R, torch, net, path, bind, amps_fp32, flush, stream, flags):
    """The same amplitudes with the tensor-core precision modes (complex
    products as 3xTF32 / 3xBF16 split products or plain TF32 on tcgen05, FP32
    accumulation), timed like the main loop (L2 flushed before each step) on
    up to 400 of its bitstrings, each with its largest amplitude error against
    the plain FP32 result, |a - a_fp32| / max(|a_fp32|, 2^-10), and (filled in
    after the CPU baseline) against the oracle on the bitstrings it
    contracted.  Not the headline: the workload specifies plain FP32."""
    out = {}
    n = min(args.steps, 400)
    fl = flags & ~R.OPT_TIMING
    for name, prec in (("tf32x3", R.PREC_TF32X3), ("bf16x3", R.PREC_BF16X3), ("tf32", R.PREC_TF32)):
        try:
            for i in range(3):
                bind(i)
                R.contract(net, path=path, precision=prec, flags=fl, max_block_entries=MAX_BLOCK)
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
            res = []
            for i in range(n):
                flush.fill_(i & 0xff)
                bind(args.warmup + i)
                ev[i][0].record(stream)
                res.append(R.contract(net, path=path, precision=prec, flags=fl, max_block_entries=MAX_BLOCK))
                ev[i][1].record(stream)
            torch.cuda.synchronize()
            ms = sum(a.elapsed_time(b) for a, b in ev)
            got = [complex(r.download()) for r in res]
            err = max(abs(g - a) / max(abs(a), 2.0 ** -10) for g, a in zip(got, amps_fp32[:n]))
            out[name] = {"value": n / (ms / 1e3), "unit": "amplitudes/s", "steps": n,
                         "max_rel_err_vs_fp32": err, "_amps": got}
        except Exception as e:   # a mode that fails is reported, not fatal to the line
            out[name] = {"error": str(e)[:200]}
    return out


def run_e2e(args, R, torch, circ, net, path, ngates, stream):
    """Same metric through the public API with host buffers: every step writes
    its bitstring's 20 projector vectors into a page-locked host array, copies
    it into a device buffer whose rows are bound as the projector tensors,
    contracts, and copies the amplitude into page-locked host memory, where it
    is read.  Steps are pipelined over a ring of host buffers (the host
    prepares step i + 1 while the device runs step i); a buffer is reused only
    after the step that used it has finished."""
    steps = args.warmup + args.steps
    bits = _bitstrings(5000, steps)
    ring = 8
    # page-locked host buffers in the tensors' storage layout (real plane,
    # imaginary plane): one copy each way, no staging kernel
    inp = [torch.zeros((2, N_QUBITS, 2), dtype=torch.float32).pin_memory() for _ in range(ring)]
    inp_np = [t.numpy() for t in inp]
    out = [torch.zeros(2, dtype=torch.float32).pin_memory() for _ in range(ring)]
    done = [torch.cuda.Event() for _ in range(ring)]
    buf = R.empty((N_QUBITS, 2), None, R.C64)
    rows = [buf.fix([0], [q]) for q in range(N_QUBITS)]
    for q in range(N_QUBITS):
        net.set_tensor(ngates + q, rows[q])
    flags = R.OPT_GRAPH | (0 if args.no_autotune else R.OPT_AUTOTUNE)   # the timed run's kernel choices
    s = stream.cuda_stream
    qidx = np.arange(N_QUBITS)
    amps = np.zeros(steps, dtype=np.complex64)
    h2d = N_QUBITS * 2 * 8
    t0 = None
    for i in range(steps):
        if i == args.warmup:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
        j = i % ring
        if i >= ring:
            done[j].synchronize()            # step i - ring has finished with slot j
            o = out[j].numpy()
            amps[i - ring] = complex(o[0], o[1])
        h = inp_np[j]
        h[0].fill(0)                         # real plane: the bitstring's projectors
        h[0][qidx, bits[i]] = 1.0            # (the imaginary plane stays zero)
        buf.upload_raw(inp[j], stream=s)
        C = R.contract(net, path=path, flags=flags, max_block_entries=MAX_BLOCK, stream=s)
        C.download_raw(out[j], stream=s)
        done[j].record(stream)
    torch.cuda.synchronize()
    for i in range(max(0, steps - ring), steps):
        o = out[i % ring].numpy()
        amps[i] = complex(o[0], o[1])
    dt = time.perf_counter() - t0
    assert np.all(np.isfinite(amps[args.warmup:]))
    return {"value": args.steps / dt, "unit": "amplitudes/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": 8,
            "what": "per step: bitstring written to a pinned host array (storage layout), 20x2 projector "
                    "upload (one copy), rosnet_contract, amplitude copied to pinned host memory and read; "
                    f"pipelined over a ring of {ring} host buffers; steady state (no L2 flush between "
                    "steps, unlike the device-timed value)"}


# ---------------------------------------------------------------------------
# CPU baseline / reference arm: the oracle as it stands
# ---------------------------------------------------------------------------
def cpu_baseline(circ, bits, seconds):
    """The oracle timed on the first bitstrings of the timed loop; returns the
    baseline record and the oracle's amplitudes (for the parity check)."""
    import oracle
    net = W.circuit_network(circ, bitstring=bits[0])
    path = oracle.greedy_path(net)
    n, ref = 0, []
    t0 = time.perf_counter()
    while n < len(bits) and (n == 0 or time.perf_counter() - t0 < seconds):
        ref.append(complex(np.asarray(oracle.contract(W.circuit_network(circ, bitstring=bits[n]), path))))
        n += 1
    dt = time.perf_counter() - t0
    return ({"value": n / dt, "unit": "amplitudes/s", "cores": os.cpu_count(), "kind": "oracle",
             "sample": f"{n} amplitudes of the same circuit (oracle complex128 loop contraction, "
                       f"oracle greedy path), {dt:.1f} s"}, ref)


def cpu_baseline_serve(pool, finished, seconds):
    """The oracle (state-vector simulation, complex128) timed on the served
    queries of the pool's circuits with n <= 20 (bounded to ~`seconds` of
    host work), and the served amplitudes checked against its results.
    Returns (baseline record, largest error, amplitudes checked)."""
    import oracle
    sv, err, n, done = {}, None, 0, 0
    t0 = time.perf_counter()
    for q in finished:
        c = pool[q.circuit]
        if c.n > 20:
            continue
        if q.circuit not in sv:
            if time.perf_counter() - t0 > seconds:
                break
            sv[q.circuit] = oracle.statevector(c)
        base = 0
        for b in q.prefix:
            base = (base << 1) | b
        for s_, got in zip(q.suffixes, q.result):
            ref = sv[q.circuit][(base << q.k) | s_]
            e = abs(complex(got) - ref) / max(abs(ref), 2.0 ** (-c.n / 2))
            err = e if err is None else max(err, e)
            n += 1
        done += len(q.suffixes)
    dt = time.perf_counter() - t0
    rec = {"value": done / dt if dt > 0 else None, "unit": "amplitudes/s", "cores": os.cpu_count(),
           "kind": "oracle", "sample": f"state vectors of {len(sv)} pool circuits (n <= 20), "
                                       f"{done} served amplitudes read from them, {dt:.1f} s"}
    return rec, err, n


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    import oracle
    circ = W.rqc20_config()
    bits = _bitstrings(1000, args.warmup + args.steps)
    net = W.circuit_network(circ, bitstring=bits[0])
    path = oracle.greedy_path(net)
    # the oracle takes ~1 s per amplitude: bounded warm-up and a bounded
    # sample of the K steps (at most ~120 s of host work), so the run ends
    # within a few minutes
    for i in range(min(args.warmup, 2)):
        oracle.contract(W.circuit_network(circ, bitstring=bits[i]), path)
    t0 = time.perf_counter()
    done = 0
    for i in range(args.warmup, args.warmup + args.steps):
        oracle.contract(W.circuit_network(circ, bitstring=bits[i]), path)
        done += 1
        if time.perf_counter() - t0 > 120.0:
            break
    dt = time.perf_counter() - t0
    value = done / dt
    line = {"metric": METRIC, "value": value, "unit": "amplitudes/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / done,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128 (fp64)",
            "data": "synthetic (seeded random circuit and bitstrings)", "impl": "reference",
            "config": _config({"parallelism": "host cores"}),
            "cpu_baseline": {"value": value, "unit": "amplitudes/s", "cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": f"{done} timed amplitudes of the {args.steps} requested "
                                       f"(bounded to ~120 s of host work) after {min(args.warmup, 2)} warm-up"},
            "e2e": {"value": value, "unit": "amplitudes/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _profiled_traffic(kind):
    """DRAM bytes per launch of the heaviest kernel from the committed ncu
    summary (profiles/traffic.json), or None when that summary is for another
    kernel family or the kernel's source changed since the capture (the
    summary names the block of its source file that holds the kernel, else
    the whole file is compared)."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)
        with open(os.path.join(ROOT, rec["source"]), "rb") as f:
            text = f.read()
        if "source_block" in rec:
            start, end = (x.encode() for x in rec["source_block"])
            i = text.index(start)
            text = text[i:text.index(end, i) + len(end)]
        sha = hashlib.sha256(text).hexdigest()
    except (OSError, ValueError, KeyError):
        return None
    if rec.get("kind") != kind or not sha.startswith(rec.get("source_sha256_prefix", "-")):
        return None
    return rec.get("bytes_per_launch")


# ---------------------------------------------------------------------------
# further workloads (not the default line)
# ---------------------------------------------------------------------------
def serving_pool(count, seed, max_flops=1e11):
    """Seeded pool of grid circuits, n ~ U{16..40}, depth ~ U{8..16}, redrawn
    until one amplitude costs at most max_flops with the library's path search."""
    import paper_2201_06620_b300 as R
    rng = np.random.default_rng(seed)
    pool = []
    while len(pool) < count:
        n, d = int(rng.integers(16, 41)), int(rng.integers(8, 17))
        circ = W.random_circuit(n, d, int(rng.integers(1 << 30)))
        net = W.circuit_network(circ)
        _, fl = R.path_search(net.labels, [t.shape for t in net.tensors], net.out_labels, ntrials=4, seed=0)
        if fl <= max_flops:
            pool.append(circ)
    return pool


def run_serve(args, emit=True):
    """Poisson stream of amplitude-batch queries served with continuous
    batching; p50/p99 latency and amplitudes/s, against the plain per-query
    FP32 form (one amplitude per contraction, one at a time)."""
    import torch
    import paper_2201_06620_b300 as R
    from paper_2201_06620_b300.serving import AmplitudeServer, Query
    pool = serving_pool(args.pool, 2022)
    rng = np.random.default_rng(7)
    ks = [0, 3, 6, 10]
    prec = {"fp32": R.PREC_DEFAULT, "bf16x3": R.PREC_BF16X3, "tf32x3": R.PREC_TF32X3}[args.serve_precision]
    srv = AmplitudeServer(pool, slots=args.slots, memory_budget=160e9, precision=prec)

    def draw():
        ci = int(rng.integers(len(pool)))
        n = pool[ci].n
        b = 2 ** int(rng.integers(0, 11))
        k = min(next(x for x in ks if 2 ** x >= b), n)
        b = min(b, 2 ** k)
        prefix = tuple(int(x) for x in rng.integers(0, 2, n - k))
        suffixes = sorted(int(x) for x in rng.choice(2 ** k, size=b, replace=False))
        return Query(circuit=ci, prefix=prefix, k=k, suffixes=suffixes)

    # warm-up: plan every (circuit, k) on every slot before the clock starts
    t0 = time.perf_counter()
    for ci, c in enumerate(pool):
        for k in ks:
            if k > c.n:
                continue
            for _ in range(args.slots):
                srv.submit(Query(circuit=ci, prefix=(0,) * (c.n - k), k=k, suffixes=[0]))
            srv.drain()
    warm = time.perf_counter() - t0
    srv.finished.clear()
    # Poisson arrivals at rate lambda for `duration` seconds, served live
    lam, dur = args.rate, args.duration
    arrivals, t = [], 0.0
    while True:
        t += rng.exponential(1.0 / lam)
        if t > dur:
            break
        arrivals.append(t)
    queries = [draw() for _ in arrivals]
    start = time.perf_counter()
    i = 0
    while i < len(queries) or srv.waiting or srv.running:
        now = time.perf_counter() - start
        while i < len(queries) and arrivals[i] <= now:
            srv.submit(queries[i], now=start + arrivals[i])
            i += 1
        srv.step()
    wall = time.perf_counter() - start
    lat = np.array([q.done - q.arrival for q in srv.finished]) * 1e3
    amps = sum(len(q.suffixes) for q in srv.finished)
    # plain per-query FP32 form on a sample, on equal terms: one amplitude per
    # contraction and per query (each waits for its result), plans built and
    # warmed before the clock (captured graphs replayed, projectors resident)
    sample = srv.finished[: args.plain_sample]
    nets = {}
    plain_n, plain_t, err = 0, 0.0, 0.0
    for q in sample:
        c = pool[q.circuit]
        if q.circuit not in nets:
            net = W.circuit_network(c, bitstring=[0] * c.n)
            ts = [R.btensor(np.asarray(x, dtype=np.complex64)) for x in net.tensors]
            nw = R.Network(ts, net.labels, net.out_labels)
            ng = len(ts) - c.n
            proj = [[R.btensor(np.eye(2, dtype=np.complex64)[b]) for b in (0, 1)] for _ in range(c.n)]
            path = R.path_search(net.labels, [x.shape for x in net.tensors], [], ntrials=16, seed=q.circuit)[0]
            for _ in range(2):
                R.contract(nw, path=path, flags=R.OPT_GRAPH).download()
            nets[q.circuit] = (nw, path, ng, proj)
        nw, path, ng, proj = nets[q.circuit]
        for s_, got in zip(q.suffixes[:4], q.result[:4]):
            bits = list(q.prefix) + [(s_ >> (q.k - 1 - j)) & 1 for j in range(q.k)]
            for qq in range(c.n):
                nw.set_tensor(ng + qq, proj[qq][bits[qq]])
            t1 = time.perf_counter()
            ref = complex(R.contract(nw, path=path, flags=R.OPT_GRAPH).download())
            plain_t += time.perf_counter() - t1
            plain_n += 1
            err = max(err, abs(complex(got) - ref) / max(abs(ref), 2.0 ** (-c.n / 2)))
    cpu, oracle_err, oracle_n = (None, None, 0) if args.no_cpu_baseline else \
        cpu_baseline_serve(pool, srv.finished, args.cpu_seconds)
    line = {"metric": "amplitudes/s (served)", "value": amps / wall, "unit": "amplitudes/s",
            "n_gpus": 1, "higher_is_better": True, "workload": "serving",
            "config": {"pool": args.pool, "rate_per_s": lam, "duration_s": dur, "slots": args.slots,
                       "precision": args.serve_precision, "k_values": ks,
                       "pool_rule": "n~U{16..40}, depth~U{8..16}, redrawn above 1e11 flop/amplitude"},
            "queries": len(srv.finished), "amplitudes": amps, "wall_s": wall, "warmup_s": warm,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "plain_fp32_per_query": {"value": plain_n / plain_t if plain_t else None, "unit": "amplitudes/s",
                                     "sample_amplitudes": plain_n,
                                     "how": "one amplitude per contraction and per query, each waiting for its "
                                            "result; plans warmed, graphs replayed, projectors resident"},
            "max_rel_err_vs_plain_fp32": err,
            "cpu_baseline": cpu,
            "oracle_check": {"max_rel_err": oracle_err, "amplitudes": oracle_n,
                             "what": "served amplitudes of the pool's circuits with n <= 20 against the "
                                     "oracle's state vector (the CPU baseline's results)"},
            "evictions": srv.evictions, "resident_plan_bytes": srv.resident_bytes}
    if emit:
        print(json.dumps(line), flush=True)
    return line


def run_batch(args, emit=True):
    """Sliced 30-qubit circuit (256 slices) + 64 circuits of 16-24 qubits in
    one batched plan per precision mode (each network as given or simplified,
    whichever has the cheaper searched path)."""
    import torch
    import paper_2201_06620_b300 as R
    # each network as given or simplified (rank-1 and rank-2 tensors absorbed
    # into neighbours on the device), whichever has the cheaper searched path;
    # the 30-qubit one is then sliced
    circ = W.random_circuit(30, 14, 2022, 5, 6)
    net = W.circuit_network(circ)
    raw = [R.btensor(np.asarray(t, dtype=np.complex64)) for t in net.tensors]
    ts, labels, path, fl = R.cheaper_network(raw, net.labels, net.out_labels, ntrials=64, seed=0)
    ntens = (len(raw), len(ts))
    ext = [t.shape for t in ts]
    cut, mx, ft = R.slice_search(labels, ext, net.out_labels, path, 8)
    nets = [n for _, n in R.sliced_networks(ts, labels, net.out_labels, cut)]
    paths = [path] * len(nets)
    rng = np.random.default_rng(7)
    nsimp = 0
    for i in range(64):
        c = W.random_circuit(int(rng.integers(16, 25)), int(rng.integers(8, 13)), 500 + i)
        nw = W.circuit_network(c)
        tr = [R.btensor(np.asarray(t, dtype=np.complex64)) for t in nw.tensors]
        tt, ll, p, _ = R.cheaper_network(tr, nw.labels, nw.out_labels, ntrials=16, seed=i)
        nsimp += len(tt) < len(tr)
        nets.append(R.Network(tt, ll, nw.out_labels))
        paths.append(p)
    res = {}
    for name, prec in (("fp32", R.PREC_DEFAULT), ("bf16x3", R.PREC_BF16X3), ("tf32x3", R.PREC_TF32X3)):
        t0 = time.perf_counter()
        fl_ = R.OPT_GRAPH | R.OPT_AUTOTUNE
        outs = R.contract_batch(nets, paths, precision=prec, flags=fl_)
        torch.cuda.synchronize()
        plan_s = time.perf_counter() - t0
        req, planned, launches, _ = R.plan_stats(nets, paths, precision=prec, flags=fl_)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        for _ in range(args.steps):
            outs = R.contract_batch(nets, paths, precision=prec, flags=fl_)
        e.record()
        torch.cuda.synchronize()
        ms = s.elapsed_time(e) / args.steps
        amp = complex(R.sum_fp64(outs[:256]).download())
        res[name] = {"batch_ms": ms, "amplitudes_per_s": 65 / (ms / 1e3), "plan_s": plan_s,
                     "steps_requested": req, "steps_planned": planned, "launches": launches,
                     "amp30": [amp.real, amp.imag]}
        del outs
        R.release_plans()
    line = {"metric": "batch amplitudes/s", "workload": "sliced 30q (256 slices) + 64 circuits",
            "tensors_30q_given_used": list(ntens), "small_circuits_simplified": nsimp,
            "path_gflop": fl / 1e9, "sliced_gflop": ft / 1e9, "max_slice_entries": mx, "modes": res}
    if emit:
        print(json.dumps(line), flush=True)
    return line


def run_reduction(args):
    """The paper's reduction comparison (Sec. IV-A, its node experiment: an
    8 x 6 grid of output blocks, B_k contracted block pairs per output block),
    scaled to blocks of m_b = n_b = 2^10, k_b = 2^9 so that a sweep of
    B_k = 2..32 takes seconds.  Per B_k and reduction mode: device time of the
    whole contraction (split reductions included), algorithmic TFLOP/s and the
    kernel family that ran (the sequential mode may take the packed path,
    which never splits; tree and commutative split K across CTAs)."""
    import torch
    import paper_2201_06620_b300 as R
    m_b, n_b, k_b, gm, gn = 1 << 10, 1 << 10, 1 << 9, 8, 6
    piece = 1 << 24
    modes = (("auto", 0), ("sequential", R.REDUCE_SEQUENTIAL), ("tree", R.REDUCE_TREE),
             ("commutative", R.REDUCE_COMMUTATIVE))
    rows = []
    for bk in (2, 4, 8, 16, 32):
        M, N, K = gm * m_b, gn * n_b, bk * k_b
        A = R.empty((M, K), (m_b, k_b), R.C64)
        B = R.empty((K, N), (k_b, n_b), R.C64)
        for t, seed in ((A, 11), (B, 12)):
            for st in range(0, t.numel, piece):
                t.upload_range(W.complex_normal_range(seed, st, min(piece, t.numel - st), 1.0), st)
        R.sync()
        for name, flag in modes:
            fl = R.OPT_GRAPH | R.OPT_TIMING | flag
            run = lambda: R.contract([A, B], [(0, 1), (1, 2)], [0, 2], [(0, 1)], flags=fl)
            run()
            torch.cuda.synchronize()
            R.timing_drain()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(3):
                C = run()
                del C
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 3
            kinds = {r[3] for r in R.timing_drain()}
            rows.append({"B_k": bk, "mode": name, "ms": ms, "tflops": 8.0 * M * N * K / (ms * 1e-3) / 1e12,
                         "kernel": "/".join(KERNEL_NAMES.get(k, f"kind {k}").split(" (")[0] for k in sorted(kinds))})
            R.release_plans()
        del A, B
    print(json.dumps({"metric": "tensordot TFLOP/s by reduction mode", "unit": "TFLOP/s",
                      "workload": "8 x 6 grid of 2^10 x 2^10 output blocks, k_b = 2^9, B_k = 2..32, complex64",
                      "rows": rows}), flush=True)


def run_tensordot(args):
    """One pairwise contraction C = A^T B with A stored (K, M) and B (K, N)
    (dense complex64 in the layout the TMA-fed GEMMs read in place; entries
    from a seeded device generator), planned once and replayed: per-call
    kernel time of the GEMM launch and algorithmic TFLOP/s.  For profiling
    one kernel on a chosen shape (--mnk M,N,K --precision ...)."""
    import torch
    import paper_2201_06620_b300 as R
    M, N, K = (int(x) for x in args.mnk.split(","))
    prec = {"fp32": R.PREC_FP32, "tf32": R.PREC_TF32, "tf32x3": R.PREC_TF32X3,
            "bf16x3": R.PREC_BF16X3}[args.precision]
    dev = torch.device("cuda", 0)
    A, B = R.empty((K, M), None, R.C64), R.empty((K, N), None, R.C64)
    g = torch.Generator(device=dev)
    for t, seed in ((A, 1), (B, 2)):
        g.manual_seed(seed)
        raw = torch.randn(2 * t.numel, device=dev, generator=g) * 0.5 ** 0.5
        t.upload_raw(raw)
        torch.cuda.synchronize()
        del raw
    ms, recs = _timed_contract(R, torch, [A, B], [(0, 1), (0, 2)], [1, 2], prec, max(args.steps, 1))
    kern = statistics.mean(r[0] for r in recs)
    flop = 8.0 * M * N * K
    print(json.dumps({"metric": "tensordot TFLOP/s", "workload": f"tensordot {M}x{N}x{K} complex64",
                      "precision": args.precision, "gemm_kernel_ms": kern, "call_ms": ms,
                      "tflops": flop / (kern * 1e-3) / 1e12, "kernel_kind": recs[0][3] if recs else None}),
          flush=True)


def run_gate(args):
    """A one-qubit gate on axis --axis of a [2]^--rank complex64 tensor (a
    single planned step on the gate kernel, the gate's output axis last):
    kernel time and HBM GB/s of the algorithmic bytes (tensor read once,
    result written once).  For profiling the memory-bound kernel."""
    import torch
    import paper_2201_06620_b300 as R
    dev = torch.device("cuda", 0)
    T = R.empty((2,) * args.rank, None, R.C64)
    g = torch.Generator(device=dev)
    g.manual_seed(args.rank)
    raw = torch.randn(2 * T.numel, device=dev, generator=g) * 0.5 ** 0.5
    T.upload_raw(raw)
    torch.cuda.synchronize()
    del raw
    G = R.btensor(W.SQRT_X.astype(np.complex64))
    lt = list(range(args.rank))
    out = [x for x in lt if x != args.axis] + [100]
    ms, recs = _timed_contract(R, torch, [T, G], [lt, [100, args.axis]], out, R.PREC_DEFAULT, max(args.steps, 1))
    kern = statistics.mean(r[0] for r in recs)
    nbytes = 2 * T.numel * 8 + 32
    print(json.dumps({"metric": "HBM GB/s", "workload": f"1q gate on axis {args.axis} of [2]^{args.rank} complex64",
                      "kernel_ms": kern, "call_ms": ms, "bytes": nbytes,
                      "gbs": nbytes / (kern * 1e-3) / 1e9, "kernel_kind": recs[0][3] if recs else None}),
          flush=True)


def run_sweep(args):
    """Precision sweep: [2]^30 x [2]^30 -> [2]^40 in 2^30-entry chunks."""
    import torch
    import paper_2201_06620_b300 as R
    prob = W.precision_sweep_config()
    A = R.empty(prob["shape_a"], prob["block_a"], R.C64)
    B = R.empty(prob["shape_b"], prob["block_b"], R.C64)
    piece = 1 << 26
    for t, seed in ((A, prob["seed_a"]), (B, prob["seed_b"])):
        for st in range(0, 1 << 30, piece):
            t.upload_range(W.complex_normal_range(seed, st, piece, prob["scale"]), st)
    R.sync()
    host = torch.empty(2 * (1 << 30) * 4, dtype=torch.uint8).pin_memory()
    flop = 8.0 * 2 ** 10 * 2 ** 20 * 2 ** 10
    peaks = _measured_peaks()
    bf16 = float(peaks.get("bf16_tflops", 1783.9))
    out = {}
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    fp32 = sms * 128 * 2 * float(peaks.get("sm_max_mhz", 2032.0)) / 1e6   # TFLOP/s, FFMA
    for name, prec, peak, issued in (("fp32", R.PREC_FP32, fp32, 1),
                                     ("tf32", R.PREC_TF32, bf16 * 1.1 / 2.25, 1),
                                     ("bf16x3", R.PREC_BF16X3, bf16, 3),
                                     ("tf32x3", R.PREC_TF32X3, bf16 * 1.1 / 2.25, 3)):
        As = A.slice([0] * 10)
        C = R.tensordot(As, B, list(range(10, 20)), prob["axes_b"], precision=prec)
        del C
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        s.record()
        C = R.tensordot(As, B, list(range(10, 20)), prob["axes_b"], precision=prec)
        e.record()
        torch.cuda.synchronize()
        ms = s.elapsed_time(e)
        del C
        t0 = time.perf_counter()
        R.tensordot_ooc(A, B, prob["axes_a"], prob["axes_b"], 10, 1, args.chunks, host, precision=prec)
        ooc = (time.perf_counter() - t0) / args.chunks
        tf = flop / ms / 1e9
        out[name] = {"chunk_ms_kernel": ms, "tflops": tf, "issued_tflops": tf * issued,
                     "peak_tflops": peak, "frac": tf * issued / peak, "ooc_s_per_chunk": ooc,
                     "ooc_tflops": flop / ooc / 1e12}
    print(json.dumps({"metric": "tensordot TFLOP/s", "workload": "precision sweep [2]^30x[2]^30->[2]^40",
                      "modes": out}), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["rosnet", "reference"], default="rosnet")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-precision-modes", action="store_true",
                    help="skip timing the tensor-core precision modes on the default workload")
    ap.add_argument("--tune-file", default=None,
                    help="load autotuner decisions from this file if it exists; save them after planning")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-probes", action="store_true", help="skip the peak-rate probes")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the extra measurements (FP64 blocked tensordot, large tensor-core contractions)")
    ap.add_argument("--workload", choices=["rqc20", "serve", "batch", "sweep", "reduction", "tensordot", "gate"],
                    default="rqc20")
    ap.add_argument("--mnk", default="1024,32768,1024", help="tensordot workload: M,N,K")
    ap.add_argument("--precision", choices=["fp32", "tf32", "tf32x3", "bf16x3"], default="fp32",
                    help="tensordot workload: arithmetic")
    ap.add_argument("--rank", type=int, default=25, help="gate workload: tensor rank")
    ap.add_argument("--axis", type=int, default=12, help="gate workload: gate axis")
    ap.add_argument("--pool", type=int, default=64)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--duration", type=float, default=20.0)
    ap.add_argument("--slots", type=int, default=2)
    # 3xTF32 keeps the served amplitudes within 1e-5 of plain FP32 on the deep
    # circuits of the pool; 3xBF16 reaches ~2e-5 there
    ap.add_argument("--serve-precision", choices=["fp32", "bf16x3", "tf32x3"], default="tf32x3")
    ap.add_argument("--plain-sample", type=int, default=20)
    ap.add_argument("--chunks", type=int, default=3)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "sweep":
        run_sweep(args)
    elif args.workload == "reduction":
        run_reduction(args)
    elif args.workload == "tensordot":
        run_tensordot(args)
    elif args.workload == "gate":
        run_gate(args)
    else:
        run_rosnet(args)


if __name__ == "__main__":
    main()
