"""Benchmark: GPU Huffman encoding pipeline (histogram -> codebook -> encode
with fused deflate) on the HPC quantisation-code field, 512^3 u16 symbols.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload hpc_field|small_field]

One step = one pass of the whole path over one field already resident in
HBM.  `value` is GB/s of input (all ranks' input bytes / max rank time).
`e2e` measures the same pass through the public binding from pinned host
memory, host->device input copy and device->host copy of the encoded stream
included.  With --gpus N > 1 (under torchrun) every rank encodes its own
replica field: the encoder has no cross-GPU exchange.
`--impl reference` times the CPU oracle (test infrastructure, single thread)
on a bounded prefix of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (n, nbins, generator description)
    "hpc_field": (512 ** 3, 1024, "u16 Laplace(512, b=2) + 1% uniform outliers over 1024 bins, seed 1"),
    "small_field": (1 << 20, 1024, "u16 Gaussian(512, sigma=8) over 1024 bins, seed 0"),
    "served": (None, None, "Poisson arrivals at --rate req/s for --duration s; half u8 Zipf(1.2) over 256 ids, "
                           "half u16 Gaussian/Laplace(512, scale log-uniform in [1, 64]) over 1024 bins; n log-uniform "
                           "in [16384, 67108864]; payloads drawn on the device before arrival; seed 5"),
    "large_alphabet": (1 << 26, 65536, "u32 Zipf(s=1.1) over 8,192, 65,536, 262,144 and 1,048,576 ids (--alphabets) "
                                       "mapped through a seeded permutation, 67,108,864 symbols per alphabet, seed 3"),
    "batched_fields": (None, 1024, "512 u16 fields, n log-uniform in [65536, 16777216], Laplace(512, b ~ U[0.5, 16]) "
                                   "over 1024 bins, seed 4 (field j: stream j, size/scale from stream 10000+j)"),
}
BATCH_FIELDS = 512
SUB_SERVED_SECONDS = 5.0      # open-loop seconds of the served sub-record of the default line
NOMINAL_HBM_GBPS = 8000.0     # GB300 HBM3e, nominal (the measured copy peak is the headline denominator)


def make_input(name: str, n: int | None = None, rank: int = 0) -> np.ndarray:
    from paper_2010_10039_gb300 import synth
    if name == "hpc_field":
        return synth.laplace_field(n or 512 ** 3, seed=1, stream=rank)
    if name == "small_field":
        return synth.gaussian_field(n or (1 << 20), seed=0)
    if name == "large_alphabet":
        return synth.zipf_field(n or (1 << 26), 65536)
    raise ValueError(name)


def load_traffic(kernel: str):
    """DRAM bytes (read + write) per launch of `kernel` from the committed ncu
    summary, or None when the kernel's source changed since the capture."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[kernel]
        h = hashlib.sha256()
        for src in rec["sources"]:
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
        if h.hexdigest() != rec["sha256"]:
            return None
        return int(rec["dram_bytes_read"]) + int(rec["dram_bytes_write"])
    except Exception:
        return None


def load_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = max(smax, float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------- CPU oracle leg

LAST_ORACLE_PARTS = {}


def oracle_leg(name: str, n_full: int, nbins: int, max_seconds: float = 15.0):
    """Times the oracle (single thread) on a prefix of the workload; returns
    (GB/s of input, sample description, symbols, seconds).  The last run's
    histogram, codebook and encode times are left in LAST_ORACLE_PARTS."""
    import oracle
    oracle.build()

    def once(n):
        sym = make_input(name, n)
        t0 = time.perf_counter()
        h = oracle.histogram(sym, nbins)
        t1 = time.perf_counter()
        book = oracle.codebook(h)
        t2 = time.perf_counter()
        oracle.encode(sym, book, chunk_log2=10)
        t3 = time.perf_counter()
        LAST_ORACLE_PARTS.clear()
        LAST_ORACLE_PARTS.update({"histogram_GBps": round(sym.nbytes / (t1 - t0) / 1e9, 4),
                                  "codebook_ms": round((t2 - t1) * 1e3, 3),
                                  "encode_GBps": round(sym.nbytes / (t3 - t2) / 1e9, 4)})
        return sym, t3 - t0

    n = min(n_full, 1 << 24)
    sym, dt = once(n)
    # grow the sample while the whole leg stays within the time bound
    while n < n_full and dt * (min(n_full, 4 * n) / n) < max_seconds:
        n = min(n_full, 4 * n)
        sym, dt = once(n)
    gbs = n * sym.itemsize / dt / 1e9
    return gbs, f"first {n} symbols of the workload, histogram+codebook+encode, 1 thread", n, dt


def multithreaded_leg(sym_np: np.ndarray, nbins: int, chunk_log2: int, gpu_words: np.ndarray, gpu_bits: int):
    """The multithreaded CPU encoder (the paper's Table VI measurement) on the
    whole field at 1, 2, 4, ... threads up to the host's cores; its stream at
    all cores is compared with the GPU's."""
    import cpu_baseline
    cores = cpu_baseline.default_threads()
    counts = sorted({1, cores} | {1 << k for k in range(1, 9) if (1 << k) < cores})
    rows = cpu_baseline.scaling(sym_np, nbins, counts, chunk_log2)
    book = cpu_baseline.codebook(cpu_baseline.histogram(sym_np, nbins, cores), cores)
    words, _, bits = cpu_baseline.encode(sym_np, book, chunk_log2, cores)
    equal = bits == gpu_bits and np.array_equal(words, gpu_words)
    if not equal:
        raise RuntimeError("the multithreaded CPU stream differs from the GPU stream")
    best = rows[-1]
    return {"value": best["hist_codebook_encode_GBps"], "unit": "GB/s", "cores": cores,
            "kind": "multithreaded C, POSIX threads (histogram + codebook + encode)",
            "sample": f"the whole field ({sym_np.size} symbols), best of 2 runs per thread count",
            "stream_equal_to_gpu": equal, "scaling": rows}


def run_reference(args, world, rank):
    name = args.workload
    n_full, nbins, desc = WORKLOADS[name]
    if rank != 0:
        return
    vals = []
    samp = None
    for i in range(args.warmup + args.steps):
        bound = max(2.0, 60.0 / max(1, args.steps + args.warmup))
        if name in ("batched_fields", "served"):
            t0 = time.perf_counter()
            leg = oracle_batched_leg if name == "batched_fields" else oracle_served_leg
            gbs, samp = leg(max_seconds=bound)
            dt = time.perf_counter() - t0
        else:
            gbs, samp, n, dt = oracle_leg(name, n_full, nbins, max_seconds=bound)
        if i >= args.warmup:
            vals.append((gbs, dt))
    value = statistics.median(v[0] for v in vals)
    ms = statistics.median(v[1] for v in vals) * 1e3
    line = {
        "impl": "reference",
        "metric": {"batched_fields": "huffman_batched_encode_input_GBps",
                   "served": "huffman_served_encode_input_GBps"}.get(name, "huffman_encode_input_GBps"), "value": round(value, 4), "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32" if name == "large_alphabet" else "u16", "data": "synthetic",
        "config": {"workload": name, "n": n_full, "nbins": nbins, "input": desc},
        "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": samp, "value": round(value, 4), "unit": "GB/s"},
        "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU leg

def run_ours(args, world, rank, local):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2010_10039_gb300 as huff

    torch.cuda.set_device(local)
    name = args.workload
    n, nbins, desc = WORKLOADS[name]
    sym_np = make_input(name, n, rank)
    sym = torch.from_numpy(sym_np.view(np.int16)).cuda()
    params = {"chunk_log2": args.chunk_log2, "merge": {"scan": 1, "shuffle": 2}[args.merge]}
    pipe = huff.Pipeline(n, nbins, params)
    stream = torch.cuda.current_stream()

    # warm-up
    for _ in range(args.warmup):
        pipe.run(sym)
    st = pipe.status()
    if st != 0:
        raise RuntimeError(f"device status {huff.STATUS.get(st, st)}")
    torch.cuda.synchronize()
    total_bits = int(pipe.total_bits.item())

    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    l0 = huff.huff_launch_count()
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for k in range(K):
        ev[k][0].record(stream)
        pipe.run(sym, stages=("hist",))
        ev[k][1].record(stream)
        pipe.run(sym, stages=("codebook",))
        ev[k][2].record(stream)
        pipe.run(sym, stages=("encode",))
        ev[k][3].record(stream)
    stop.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = huff.huff_launch_count() - l0
    clk = clocks.stop()
    total_ms = start.elapsed_time(stop)
    ms_step = max_over_ranks(total_ms / K, world)
    st = pipe.status()
    if st != 0:
        raise RuntimeError(f"device status {huff.STATUS.get(st, st)}")

    stage_lists = {"histogram": [ev[k][0].elapsed_time(ev[k][1]) for k in range(K)],
                   "codebook": [ev[k][1].elapsed_time(ev[k][2]) for k in range(K)],
                   "encode": [ev[k][2].elapsed_time(ev[k][3]) for k in range(K)]}
    hist_ms = statistics.mean(stage_lists["histogram"])
    cb_ms = statistics.mean(stage_lists["codebook"])
    enc_ms = statistics.mean(stage_lists["encode"])
    in_bytes = n * 2
    out_bytes = (total_bits + 31) // 32 * 4
    nch = (n + (1 << args.chunk_log2) - 1) >> args.chunk_log2
    off_bytes = (nch + 1) * 8
    enc_alg = in_bytes + out_bytes + off_bytes
    hist_alg = in_bytes + nbins * 4
    peak, peak_kind = load_peak()
    value = world * in_bytes / (ms_step * 1e-3) / 1e9

    # the decoder on the stream just written (outside the timed step): event
    # timed on the launching stream, output checked against the input
    dec = None
    if args.merge == "scan":
        dec_out = torch.empty_like(sym)
        for _ in range(2):
            huff.huff_decode(pipe.out, total_bits, pipe.offsets, args.chunk_log2, n, 2, pipe.codebook, nbins,
                             dec_out, pipe.ws)
        d0 = torch.cuda.Event(enable_timing=True)
        d1 = torch.cuda.Event(enable_timing=True)
        reps = 5
        d0.record(stream)
        for _ in range(reps):
            huff.huff_decode(pipe.out, total_bits, pipe.offsets, args.chunk_log2, n, 2, pipe.codebook, nbins,
                             dec_out, pipe.ws)
        d1.record(stream)
        torch.cuda.synchronize()
        dec_ms = d0.elapsed_time(d1) / reps
        st = pipe.status()
        if st != 0 or not torch.equal(dec_out, sym):
            raise RuntimeError(f"decode: status {huff.STATUS.get(st, st)}, output equal {torch.equal(dec_out, sym)}")
        dec_alg = out_bytes + off_bytes + in_bytes
        dec = {"ms": round(dec_ms, 5), "GBps_of_symbols": round(in_bytes / (dec_ms * 1e-3) / 1e9, 2),
               "roofline": {"bound": "hbm", "achieved": round(dec_alg / (dec_ms * 1e-3) / 1e9, 2), "peak": peak,
                            "unit": "GB/s", "frac": round(dec_alg / (dec_ms * 1e-3) / 1e9 / peak, 4),
                            "algorithmic_bytes": dec_alg},
               "equal_to_input": True}
        del dec_out

    # format ablation: the encode alone in each stream format (Sec. IV-C typed
    # units of W bits; Sec. VI chunks kept unit-aligned instead of gathered
    # densely), on the same field, outside the timed step
    formats = []
    if args.merge == "scan" and 9 <= args.chunk_log2 <= 12:
        for W in (32, 16, 8):
            for layout in (0, 1):
                prm = dict(params, word_bits=W, layout=layout)
                p2 = huff.Pipeline(n, nbins, prm)
                p2.run(sym)
                for _ in range(2):
                    p2.run(sym, stages=("encode",))
                ts = []
                for _ in range(8):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    p2.run(sym, stages=("encode",))
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1) * 1e3)
                st2 = p2.status()
                if st2 != 0:
                    raise RuntimeError(f"format W={W} layout={layout}: device status {huff.STATUS.get(st2, st2)}")
                tb2 = int(p2.total_bits.item())
                formats.append({"word_bits": W, "layout": "chunk_aligned" if layout else "dense",
                                "encode_us_mean": round(statistics.mean(ts), 2), "encode_us_best": round(min(ts), 2),
                                "stream_bytes": (tb2 + W - 1) // W * W // 8,
                                "input_GBps": round(in_bytes / (statistics.mean(ts) * 1e-6) / 1e9, 1)})
                del p2

    # end to end through the binding from pinned host memory: every step copies
    # its input in and its stream and offsets out.  Two buffer sets and two copy
    # streams let step k + 1's input copy overlap step k's compute and read-back.
    # The stream's length is known only on the device: its bit count comes back
    # by an 8-byte copy, and the host reads it one step late (while the device
    # is already busy with the next step) to size the stream's read-back.
    nw = (total_bits + 31) // 32
    ref_words = pipe.out[:nw].cpu()
    ref_offs = pipe.offsets.cpu()
    host_in = torch.from_numpy(sym_np.view(np.int16)).pin_memory()
    pipes = [pipe, huff.Pipeline(n, nbins, params)]
    dev_in = [torch.empty_like(sym), torch.empty_like(sym)]
    host_out = [torch.empty(pipe.out.numel(), dtype=torch.int32).pin_memory() for _ in range(2)]
    host_offs = [torch.empty(pipe.offsets.numel(), dtype=torch.int64).pin_memory() for _ in range(2)]
    host_tb = [torch.zeros(1, dtype=torch.int64).pin_memory() for _ in range(2)]
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event(), torch.cuda.Event()]
    ev_used = [torch.cuda.Event(), torch.cuda.Event()]     # compute on buffer set b finished
    ev_tb = [torch.cuda.Event(), torch.cuda.Event()]       # bit count of buffer set b on the host
    ev_read = [torch.cuda.Event(), torch.cuda.Event()]     # read-back of buffer set b finished
    read_words = [0, 0]

    def read_back(b):
        ev_tb[b].synchronize()
        nw = (int(host_tb[b][0]) + 31) // 32
        read_words[b] = nw
        with torch.cuda.stream(s_out):
            host_out[b][:nw].copy_(pipes[b].out[:nw], non_blocking=True)
            host_offs[b].copy_(pipes[b].offsets, non_blocking=True)
            ev_read[b].record(s_out)

    def e2e_run(steps):
        with torch.cuda.stream(s_in):
            dev_in[0].copy_(host_in, non_blocking=True)
            ev_in[0].record(s_in)
        pending = None
        for k in range(steps):
            b = k % 2
            if k + 1 < steps:
                nb = 1 - b
                with torch.cuda.stream(s_in):
                    if k >= 1:
                        s_in.wait_event(ev_used[nb])           # step k - 1 no longer reads dev_in[nb]
                    dev_in[nb].copy_(host_in, non_blocking=True)
                    ev_in[nb].record(s_in)
            stream.wait_event(ev_in[b])
            if k >= 2:
                stream.wait_event(ev_read[b])                  # step k - 2's stream is off the device
            pipes[b].run(dev_in[b])
            ev_used[b].record(stream)
            with torch.cuda.stream(s_out):
                s_out.wait_event(ev_used[b])
                host_tb[b].copy_(pipes[b].total_bits, non_blocking=True)
                ev_tb[b].record(s_out)
            if pending is not None:
                read_back(pending)                             # step k - 1, while step k computes
            pending = b
        read_back(pending)
        torch.cuda.synchronize()

    e2e_steps = max(8, K)
    torch.cuda.synchronize()
    e2e_run(2)                                                 # untimed: touches both buffer sets
    barrier(world)
    t0 = time.perf_counter()
    e2e_run(e2e_steps)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, world)
    e2e_val = world * in_bytes / e2e_s / 1e9
    for b in range(2):
        st = pipes[b].status()
        if st != 0:
            raise RuntimeError(f"end-to-end run: device status {huff.STATUS.get(st, st)}")
    # both buffer sets encoded the same input: their streams must equal the
    # device-timed run's
    for b in range(2):
        if read_words[b] != nw or not torch.equal(host_out[b][:nw], ref_words) or \
                not torch.equal(host_offs[b], ref_offs):
            raise RuntimeError(f"end-to-end run: buffer set {b} read back a different stream")
    del pipes, dev_in, host_out, host_offs

    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        gbs, samp, _, _ = oracle_leg(name, n, nbins)
        cpu = {"value": round(gbs, 4), "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": samp,
               "parts": dict(LAST_ORACLE_PARTS), "host_cores": os.cpu_count(),
               "multithreaded": multithreaded_leg(sym_np, nbins, args.chunk_log2, ref_words.numpy().view(np.uint32),
                                                  total_bits)}
    enc_s = enc_ms * 1e-3
    line = {
        "metric": "huffman_encode_input_GBps",
        "value": round(value, 3),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": round(ms_step, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u16",
        "data": "synthetic",
        "config": {"workload": name, "n": n, "nbins": nbins, "input": desc, "chunk_log2": args.chunk_log2,
                   "encode_layout": args.merge,
                   "l2": "inputs larger than L2 (268 MB per step)", "parallelism": f"replicas{world}",
                   "avg_bits": round(total_bits / n, 4)},
        "stages_ms": {"histogram": round(hist_ms, 5), "codebook": round(cb_ms, 5), "encode": round(enc_ms, 5)},
        "stages_ms_best": {k: round(min(v), 5) for k, v in stage_lists.items()},
        "stages_ms_median": {k: round(statistics.median(v), 5) for k, v in stage_lists.items()},
        "encode_only_GBps": round(in_bytes / enc_s / 1e9, 3),
        "roofline": {"bound": "hbm", "kernel": "encode (a4-a6)" if args.merge == "scan" else
                     "encode, paper layout: merge + scan + gather kernels", "achieved": round(enc_alg / enc_s / 1e9, 2),
                     "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": round(enc_alg / enc_s / 1e9 / peak, 4),
                     "traffic": load_traffic("encode_kernel") if name == "hpc_field" and args.merge == "scan" else None,
                     "algorithmic_bytes": enc_alg, "peak_nominal": NOMINAL_HBM_GBPS,
                     "frac_nominal": round(enc_alg / enc_s / 1e9 / NOMINAL_HBM_GBPS, 4)},
        "roofline_histogram": {"bound": "hbm", "achieved": round(hist_alg / (hist_ms * 1e-3) / 1e9, 2),
                               "peak": peak, "unit": "GB/s",
                               "frac": round(hist_alg / (hist_ms * 1e-3) / 1e9 / peak, 4),
                               "traffic": load_traffic("hist_kernel") if name == "hpc_field" else None},
        "e2e": {"value": round(e2e_val, 3), "unit": "GB/s", "h2d_bytes_per_step": in_bytes,
                "d2h_bytes_per_step": out_bytes + off_bytes + 8, "steps": e2e_steps,
                "untimed_steps_before": 2, "checked": "both buffer sets' streams equal the timed run's"},
        "gpu_launches": launches,
        "cpu_baseline": cpu,
        "clocks": clk,
        "decode": dec,
        "format_ablation": formats,
    }
    return line


# ----------------------------------------------------------------------------- large alphabets

def run_large_alphabet(args, world, rank, local):
    """The large-alphabet stress: 67,108,864 u32 Zipf(1.1) symbols over each
    alphabet of --alphabets (8,192 to 1,048,576 ids, n-gram sized), each
    through histogram -> codebook -> encode, with every stage timed on its
    own.  A step is all alphabets."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2010_10039_gb300 as huff
    from paper_2010_10039_gb300 import synth

    torch.cuda.set_device(local)
    n = WORKLOADS["large_alphabet"][0]
    alphabets = tuple(args.alphabets)
    params = {"chunk_log2": args.chunk_log2}
    fields = []
    for K in alphabets:
        sym = synth.draw_device(3, rank, n, synth.cdf_table(synth.zipf_pmf(K, 1.1)), 4,
                                mapping=synth.permutation(3, K))
        fields.append((K, sym, huff.Pipeline(n, K, params)))
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        for K, sym, pipe in fields:
            pipe.run(sym)
    torch.cuda.synchronize()
    for K, sym, pipe in fields:
        st = pipe.status()
        if st != 0:
            raise RuntimeError(f"{K} bins: device status {huff.STATUS.get(st, st)}")

    steps = args.steps
    ev = {K: [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)] for K in alphabets}
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    l0 = huff.huff_launch_count()
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for k in range(steps):
        for K, sym, pipe in fields:
            e = ev[K][k]
            e[0].record(stream)
            pipe.run(sym, stages=("hist",))
            e[1].record(stream)
            pipe.run(sym, stages=("codebook",))
            e[2].record(stream)
            pipe.run(sym, stages=("encode",))
            e[3].record(stream)
    stop.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = huff.huff_launch_count() - l0
    clk = clocks.stop()
    ms_step = max_over_ranks(start.elapsed_time(stop) / steps, world)
    peak, peak_kind = load_peak()
    in_bytes = n * 4
    per = {}
    enc_total_ms = 0.0
    for K, sym, pipe in fields:
        st = pipe.status()
        if st != 0:
            raise RuntimeError(f"{K} bins: device status {huff.STATUS.get(st, st)}")
        hist_ms = statistics.mean(ev[K][k][0].elapsed_time(ev[K][k][1]) for k in range(steps))
        cb_ms = statistics.mean(ev[K][k][1].elapsed_time(ev[K][k][2]) for k in range(steps))
        enc_ms = statistics.mean(ev[K][k][2].elapsed_time(ev[K][k][3]) for k in range(steps))
        enc_total_ms += enc_ms
        total_bits = int(pipe.total_bits.item())
        max_len = int(pipe.codebook[4:8].view(torch.int32).item())
        nch = (n + (1 << args.chunk_log2) - 1) >> args.chunk_log2
        enc_alg = in_bytes + (total_bits + 31) // 32 * 4 + (nch + 1) * 8
        per[str(K)] = {
            "codebook_us": round(cb_ms * 1e3, 2),
            "stages_ms": {"histogram": round(hist_ms, 5), "codebook": round(cb_ms, 5), "encode": round(enc_ms, 5)},
            "step_GBps": round(in_bytes / ((hist_ms + cb_ms + enc_ms) * 1e-3) / 1e9, 3),
            "encode_roofline": {"bound": "hbm", "achieved": round(enc_alg / (enc_ms * 1e-3) / 1e9, 2),
                                "peak": peak, "unit": "GB/s",
                                "frac": round(enc_alg / (enc_ms * 1e-3) / 1e9 / peak, 4),
                                "traffic": None, "algorithmic_bytes": enc_alg},
            "avg_bits": round(total_bits / n, 4),
            "max_len": max_len,
        }
    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        ns = 1 << 22
        cpu = {}
        for K in alphabets:
            symh = synth.zipf_field(ns, K)
            t0 = time.perf_counter()
            h = oracle.histogram(symh, K)
            t1 = time.perf_counter()
            book = oracle.codebook(h)
            t2 = time.perf_counter()
            oracle.encode(symh, book, chunk_log2=10)
            t3 = time.perf_counter()
            cpu[str(K)] = {"value": round(ns * 4 / (t3 - t0) / 1e9, 4), "codebook_us": round((t2 - t1) * 1e6, 1)}
        cpu = {"value": round(2 * ns * 4 / sum(ns * 4 / v["value"] / 1e9 for v in cpu.values()) / 1e9, 4),
               "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"first {ns} symbols of each alphabet's field, histogram+codebook+encode, 1 thread",
               "per_alphabet": cpu}
    value = world * len(alphabets) * in_bytes / (ms_step * 1e-3) / 1e9
    line = {
        "metric": "huffman_encode_input_GBps", "value": round(value, 3), "unit": "GB/s", "n_gpus": world,
        "steps": steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "large_alphabet", "n": n, "alphabets": list(alphabets),
                   "input": WORKLOADS["large_alphabet"][2], "chunk_log2": args.chunk_log2,
                   "l2": "inputs larger than L2 (268 MB per field)", "parallelism": f"replicas{world}"},
        "alphabets": per,
        "e2e": None,
        "gpu_launches": launches,
        "cpu_baseline": cpu,
        "clocks": clk,
    }
    return line


# ----------------------------------------------------------------------------- batched form

def batched_fields_params():
    from paper_2010_10039_gb300 import synth
    return [synth.batch_field_params(j) for j in range(BATCH_FIELDS)]


def oracle_batched_leg(max_seconds: float = 15.0):
    """The oracle (single thread) over whole fields of the batched workload,
    taken in field order until the time bound; returns (GB/s, description)."""
    import oracle
    from paper_2010_10039_gb300 import synth
    oracle.build()
    done_bytes, dt, k = 0, 0.0, 0
    for j, (n, b) in enumerate(batched_fields_params()):
        if dt > max_seconds * 0.5 and k:
            break
        sym = synth.batch_field(j)
        t0 = time.perf_counter()
        h = oracle.histogram(sym, 1024)
        book = oracle.codebook(h)
        oracle.encode(sym, book, chunk_log2=10)
        dt += time.perf_counter() - t0
        done_bytes += sym.nbytes
        k += 1
    return done_bytes / dt / 1e9, f"fields 0..{k - 1} of the batched workload ({done_bytes // 2} symbols), " \
                                  "histogram+codebook+encode per field, 1 thread"


def run_batched(args, world, rank, local):
    """512 fields, one plan (graph of histogram, codebooks, planner and one
    persistent encode launch), against 512 separate plain calls per step."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2010_10039_gb300 as huff
    from paper_2010_10039_gb300 import synth

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    prm = batched_fields_params()
    fields = []
    for j, (n, b) in enumerate(prm):
        table = synth.cdf_table(synth.laplace_pmf(1024, 512, b))
        sym = synth.draw_device(4, j + 100000 * rank, n, table, 2)
        fields.append({"sym": sym, "nbins": 1024, "chunk_log2": 10,
                       "out": torch.empty((n * 12 + 31) // 32 + 1, dtype=torch.int32, device="cuda"),
                       "offsets": torch.empty((n >> 10) + 2, dtype=torch.int64, device="cuda"),
                       "total_bits": torch.zeros(1, dtype=torch.int64, device="cuda")})
    torch.cuda.synchronize()
    total_n = sum(n for n, _ in prm)
    in_bytes = 2 * total_n
    t_plan = time.perf_counter()
    plan = huff.BatchPlan(fields, autotune=True)
    t_plan = time.perf_counter() - t_plan
    info = plan.info()

    for _ in range(args.warmup):
        plan.encode()
    st = plan.status()
    if any(st):
        raise RuntimeError(f"device status {[huff.STATUS.get(x, x) for x in st if x][:4]}")
    K = args.steps
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    l0 = huff.huff_launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(K):
        plan.encode()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = huff.huff_launch_count() - l0
    clk = clocks.stop()
    ms_step = max_over_ranks(ev0.elapsed_time(ev1) / K, world)
    stages = plan.profile()
    out_bytes = sum(4 * ((int(f["total_bits"].item()) + 31) // 32) for f in fields)
    off_bytes = sum(8 * (((n + 1023) >> 10) + 1) for n, _ in prm)
    bits = sum(int(f["total_bits"].item()) for f in fields)

    # the same work as 512 separate plain calls (histogram, codebook, encode per field)
    maxn = max(n for n, _ in prm)
    ws = torch.zeros(huff.huff_workspace_bytes(maxn, 1024), dtype=torch.uint8, device="cuda")
    huff.huff_workspace_init(ws)
    hist = torch.empty(1024, dtype=torch.int32, device="cuda")
    book = torch.empty(huff.huff_codebook_bytes(1024), dtype=torch.uint8, device="cuda")

    def per_call():
        for f in fields:
            huff.huff_histogram(f["sym"], 1024, hist, ws)
            huff.huff_build_codebook(hist, 1024, book, ws)
            huff.huff_encode(f["sym"], book, 1024, f["out"], f["offsets"], f["total_bits"], ws)
    for _ in range(max(1, args.warmup)):
        per_call()
    if huff.huff_get_status(ws) != 0:
        raise RuntimeError("per-call path reported an error")
    reps = max(1, min(K, 5))
    ev0.record(stream)
    for _ in range(reps):
        per_call()
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_per_call = ev0.elapsed_time(ev1) / reps

    # end to end: pinned host inputs in, encoded streams and offsets out, every
    # step.  Two buffer sets, each with its own plan (the tuned settings) and
    # its own host result buffers, and a copy stream for each direction: step
    # k + 1's inputs go in while step k encodes and its results come back.
    # Every field's stream length is the one the timed run found (the inputs
    # are the same), so no step waits on the device for it.
    host_in = [f["sym"].cpu().pin_memory() for f in fields]
    nw = [(int(f["total_bits"].item()) + 31) // 32 for f in fields]
    ref_out = [f["out"][:w].cpu() for f, w in zip(fields, nw)]
    ref_off = [f["offsets"].cpu() for f in fields]
    fields2 = [{"sym": torch.empty_like(f["sym"]), "nbins": f["nbins"], "chunk_log2": f["chunk_log2"],
                "out": torch.empty_like(f["out"]), "offsets": torch.empty_like(f["offsets"]),
                "total_bits": torch.zeros_like(f["total_bits"])} for f in fields]
    plan2 = huff.BatchPlan(fields2, autotune=False, reduce_log2=info["reduce_log2"],
                           max_subtiles=info["max_subtiles"], ctas_per_sm=info["ctas_per_sm"],
                           encode_form=info["encode_form"])
    sets = [(fields, plan), (fields2, plan2)]
    host_out = [[torch.empty(max(1, w), dtype=torch.int32).pin_memory() for w in nw] for _ in range(2)]
    host_off = [[torch.empty_like(f["offsets"], device="cpu").pin_memory() for f in fields] for _ in range(2)]
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event(), torch.cuda.Event()]
    ev_used = [torch.cuda.Event(), torch.cuda.Event()]
    ev_read = [torch.cuda.Event(), torch.cuda.Event()]

    def copy_in(b):
        with torch.cuda.stream(s_in):
            for f, h in zip(sets[b][0], host_in):
                f["sym"].copy_(h, non_blocking=True)
            ev_in[b].record(s_in)

    def e2e_run(steps):
        copy_in(0)
        for k in range(steps):
            b = k % 2
            if k + 1 < steps:
                if k >= 1:
                    s_in.wait_event(ev_used[1 - b])          # step k - 1 no longer reads those inputs
                copy_in(1 - b)
            stream.wait_event(ev_in[b])
            if k >= 2:
                stream.wait_event(ev_read[b])                # step k - 2's results are off the device
            sets[b][1].encode()
            ev_used[b].record(stream)
            with torch.cuda.stream(s_out):
                s_out.wait_event(ev_used[b])
                for f, ho, hf, w in zip(sets[b][0], host_out[b], host_off[b], nw):
                    ho[:w].copy_(f["out"][:w], non_blocking=True)
                    hf.copy_(f["offsets"], non_blocking=True)
                ev_read[b].record(s_out)
        torch.cuda.synchronize()

    e2e_steps = max(8, K)
    torch.cuda.synchronize()
    e2e_run(2)                                               # untimed: touches both buffer sets
    barrier(world)
    t0 = time.perf_counter()
    e2e_run(e2e_steps)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, world)
    for fs, pl in sets:
        st = pl.status()
        if any(st):
            raise RuntimeError(f"end-to-end run: device status {[huff.STATUS.get(x, x) for x in st if x][:4]}")
    for b, (fs, _) in enumerate(sets):
        for j, f in enumerate(fs):
            if int(f["total_bits"].item()) != int(fields[j]["total_bits"].item()) or \
                    not torch.equal(host_out[b][j][:nw[j]], ref_out[j]) or not torch.equal(host_off[b][j], ref_off[j]):
                raise RuntimeError(f"end-to-end run: buffer set {b}, field {j} read back a different stream")
    del plan2, fields2

    if rank != 0:
        return
    peak, peak_kind = load_peak()
    enc_alg = in_bytes + out_bytes + off_bytes
    enc_ms = stages["encode"]
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        gbs, samp = oracle_batched_leg()
        cpu = {"value": round(gbs, 4), "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": samp}
    value = world * in_bytes / (ms_step * 1e-3) / 1e9
    line = {
        "metric": "huffman_batched_encode_input_GBps",
        "value": round(value, 3), "unit": "GB/s", "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": round(ms_step, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u16", "data": "synthetic",
        "config": {"workload": "batched_fields", "fields": BATCH_FIELDS, "symbols": total_n, "nbins": 1024,
                   "input": WORKLOADS["batched_fields"][2], "l2": f"inputs larger than L2 ({in_bytes >> 20} MiB per step)",
                   "parallelism": f"replicas{world}", "avg_bits": round(bits / total_n, 4)},
        "per_call_GBps": round(in_bytes / (ms_per_call * 1e-3) / 1e9, 3),
        "per_call_ms": round(ms_per_call, 4),
        "speedup_vs_per_call": round(ms_per_call / ms_step, 3),
        "plan": {k: (round(v, 4) if isinstance(v, float) else v) for k, v in info.items()},
        "plan_create_s": round(t_plan, 3),
        "stages_ms_ungraphed": {k: round(v, 4) for k, v in stages.items()},
        "roofline": {"bound": "hbm", "kernel": {0: "batched encode (one launch, all fields)",
                                                1: "batched encode (one single-field launch per field, concurrent)",
                                                2: "batched encode (segment encoder over the fields it takes, then "
                                                   "the general encoder over the rest)"}[info["encode_form"]],
                     "achieved": round(enc_alg / (enc_ms * 1e-3) / 1e9, 2), "peak": peak, "peak_kind": peak_kind,
                     "unit": "GB/s", "frac": round(enc_alg / (enc_ms * 1e-3) / 1e9 / peak, 4), "traffic": None,
                     "algorithmic_bytes": enc_alg},
        "e2e": {"value": round(world * in_bytes / e2e_s / 1e9, 3), "unit": "GB/s", "h2d_bytes_per_step": in_bytes,
                "d2h_bytes_per_step": out_bytes + off_bytes, "steps": e2e_steps, "untimed_steps_before": 2,
                "checked": "both buffer sets' streams and offsets equal the timed run's"},
        "gpu_launches": launches,
        "cpu_baseline": cpu,
        "clocks": clk,
    }
    return line


# ----------------------------------------------------------------------------- served form

def oracle_served_leg(max_seconds: float = 15.0):
    """The oracle (single thread) over whole served requests, in order, until
    the time bound; returns (GB/s, description)."""
    import oracle
    from paper_2010_10039_gb300 import synth
    oracle.build()
    done, dt, k = 0, 0.0, 0
    i = 0
    while dt < max_seconds * 0.5 or k == 0:
        width, n, nbins, _ = synth.served_request(i)
        i += 1
        if n > (1 << 23):
            continue                      # keep the sample bounded: skip the largest requests
        sym = synth.served_symbols(i - 1)
        t0 = time.perf_counter()
        h = oracle.histogram(sym, nbins)
        book = oracle.codebook(h)
        oracle.encode(sym, book, chunk_log2=10)
        dt += time.perf_counter() - t0
        done += sym.nbytes
        k += 1
    return done / dt / 1e9, f"{k} served requests of at most 2^23 symbols ({done} bytes), 1 thread"


def _pct(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    return xs[min(len(xs) - 1, int(round(q / 100.0 * (len(xs) - 1))))]


def run_served(args, world, rank, local):
    """Open-loop Poisson load through huff_serve_* against the same schedule
    through serial plain calls, then a closed-loop saturation comparison."""
    import queue
    import threading
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2010_10039_gb300 as huff
    from paper_2010_10039_gb300 import synth

    torch.cuda.set_device(local)
    rate, duration = args.rate, args.duration
    arr = synth.served_arrivals(int(rate * duration * 1.3) + 64)
    count = int(np.searchsorted(arr, duration))
    arr = arr[:count]
    gen_stream = torch.cuda.Stream()
    budget = 40 << 30

    def prepare(i):
        width, n, nbins, table = synth.served_request(i)
        with torch.cuda.stream(gen_stream):
            sym = synth.draw_device(5, 100 + i, n, table, width)
            ev = torch.cuda.Event()
            ev.record(gen_stream)
        return i, sym, nbins, ev, n * width

    def producer(q, indices):
        for i in indices:
            q.put(prepare(i))
        q.put(None)

    sample_ids = [i for i in range(min(count, 400)) if synth.served_request(i)[1] <= (1 << 21)][:4]

    # ---------------- served, open loop
    srv = huff.Server(mem_budget_bytes=budget, nstreams=4, max_batch=64, max_inflight=4096)
    for i in range(8):                                  # warm-up (kernels loaded, pools touched)
        _, sym, nb, ev, _ = prepare(10_000_000 + i)
        ev.synchronize()
        t = srv.submit(sym, nb)
        srv.wait(t)
        srv.release(t)
    q_in = queue.Queue(maxsize=512)
    q_done = queue.Queue()
    lat, done_t, bytes_total, statuses, sampled = {}, {}, 0, [], {}
    threading.Thread(target=producer, args=(q_in, range(count)), daemon=True).start()

    def collector():
        while True:
            item = q_done.get()
            if item is None:
                return
            i, t, arrival, sym = item
            res = srv.wait(t)
            statuses.append(res["status"])
            lat[i] = res["t_done"] - arrival
            done_t[i] = res["t_done"]
            if i in sample_ids:
                nw = (res["total_bits"] + 31) // 32
                m = res["chunk_log2"]
                nch = ((sym.numel() + (1 << m) - 1) >> m) + 1
                sampled[i] = (res["total_bits"],
                              huff.device_view(res["d_out"], 4 * max(1, nw)).cpu().numpy().view(np.uint32)[:nw].copy(),
                              huff.device_view(res["d_chunk_bit_offset"], 8 * nch).cpu().numpy().view(np.uint64).copy())
            srv.release(t)
    col = threading.Thread(target=collector, daemon=True)
    col.start()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = huff.huff_launch_count()
    t0 = time.monotonic()
    late = 0.0
    while True:
        item = q_in.get()
        if item is None:
            break
        i, sym, nb, ev, nbytes = item
        arrival = t0 + float(arr[i])
        d = arrival - time.monotonic()
        if d > 0:
            time.sleep(d)
        else:
            late = max(late, -d)
        ev.synchronize()
        t = srv.submit(sym, nb, keep=False)
        bytes_total += nbytes
        q_done.put((i, t, arrival, sym))
    q_done.put(None)
    col.join()
    launches = huff.huff_launch_count() - l0
    clk = clocks.stop()
    t_end = max(done_t.values())
    served_gbps = bytes_total / (t_end - t0) / 1e9
    stats = srv.stats()
    if any(statuses):
        raise RuntimeError(f"served jobs failed: {sorted(set(statuses))}")
    lat_ms = [v * 1e3 for v in lat.values()]

    # ---------------- the same schedule through serial plain calls
    pipes = {256: huff.Pipeline(1 << 26, 256), 1024: huff.Pipeline(1 << 26, 1024)}
    q_in = queue.Queue(maxsize=512)
    threading.Thread(target=producer, args=(q_in, range(count)), daemon=True).start()
    cur = torch.cuda.current_stream()
    slat = []
    t0s = time.monotonic()
    last_done = t0s
    while True:
        item = q_in.get()
        if item is None:
            break
        i, sym, nb, ev, nbytes = item
        arrival = t0s + float(arr[i])
        d = arrival - time.monotonic()
        if d > 0:
            time.sleep(d)
        ev.synchronize()
        pipes[nb].run(sym)
        cur.synchronize()
        last_done = time.monotonic()
        slat.append((last_done - arrival) * 1e3)
    serial_gbps = bytes_total / (last_done - t0s) / 1e9
    for p in pipes.values():
        if p.status() != 0:
            raise RuntimeError("serial path reported an error")

    # ---------------- closed loop: a backlog of requests, served vs serial
    M = min(args.saturation_requests, count)
    items = [prepare(i) for i in range(M)]
    torch.cuda.synchronize()
    sat_bytes = sum(it[4] for it in items)
    ts = time.monotonic()
    tk = [srv.submit(sym, nb, keep=False) for _, sym, nb, _, _ in items]
    for t in tk:
        srv.wait(t)
    te = time.monotonic()
    for t in tk:
        srv.release(t)
    sat_served = sat_bytes / (te - ts) / 1e9
    ts = time.monotonic()
    for _, sym, nb, _, _ in items:
        pipes[nb].run(sym)
    cur.synchronize()
    sat_serial = sat_bytes / (time.monotonic() - ts) / 1e9
    sat_stats = srv.stats()

    # ---------------- rate sweep: open loop over the prepared requests (reused
    # cyclically) at rising rates until the server stops keeping up; at each
    # rate the same arrivals also go through serial plain calls
    def wait_until(t):
        d = t - time.monotonic()
        if d > 3e-4:
            time.sleep(d - 2e-4)
        while time.monotonic() < t:
            pass
        return -d

    def sweep_point(rate, seconds):
        arr_r = synth.served_arrivals(int(rate * seconds * 1.3) + 64, rate=rate)
        cnt = int(np.searchsorted(arr_r, seconds))
        reqs = [items[i % len(items)] for i in range(cnt)]
        nbytes = sum(r[4] for r in reqs)
        st0 = srv.stats()
        tq = queue.Queue()
        lat_r, t_last, bad = [], [0.0], []

        def coll():
            while True:
                x = tq.get()
                if x is None:
                    return
                t, arrival = x
                res = srv.wait(t)
                if res["status"]:
                    bad.append(res["status"])
                lat_r.append((res["t_done"] - arrival) * 1e3)
                t_last[0] = max(t_last[0], res["t_done"])
                srv.release(t)
        th = threading.Thread(target=coll, daemon=True)
        th.start()
        t0r = time.monotonic() + 0.002
        late_r = 0.0
        for (_, sym, nb, _, _), a in zip(reqs, arr_r[:cnt]):
            arrival = t0r + float(a)
            late_r = max(late_r, wait_until(arrival))
            tq.put((srv.submit(sym, nb, keep=False), arrival))
        tq.put(None)
        th.join()
        if bad:
            raise RuntimeError(f"sweep at {rate}/s: jobs failed {sorted(set(bad))}")
        st1 = srv.stats()
        served_r = nbytes / (t_last[0] - t0r) / 1e9
        # serial plain calls on the same arrivals
        slat_r = []
        t0s_r = time.monotonic() + 0.002
        last = t0s_r
        for (_, sym, nb, _, _), a in zip(reqs, arr_r[:cnt]):
            arrival = t0s_r + float(a)
            wait_until(arrival)
            pipes[nb].run(sym)
            cur.synchronize()
            last = time.monotonic()
            slat_r.append((last - arrival) * 1e3)
        serial_r = nbytes / (last - t0s_r) / 1e9
        nb_batches = st1["batches"] - st0["batches"]
        return {"rate_per_s": rate, "requests": cnt, "offered_GBps": round(nbytes / seconds / 1e9, 3),
                "served_GBps": round(served_r, 3), "served_p50_ms": round(_pct(lat_r, 50), 3),
                "served_p99_ms": round(_pct(lat_r, 99), 3),
                "mean_jobs_per_batch": round((st1["completed"] - st0["completed"]) / max(1, nb_batches), 2),
                "serial_GBps": round(serial_r, 3), "serial_p50_ms": round(_pct(slat_r, 50), 3),
                "serial_p99_ms": round(_pct(slat_r, 99), 3), "submit_late_max_ms": round(max(0.0, late_r) * 1e3, 3)}

    sweep = []
    for rate_r in args.sweep_rates:
        row = sweep_point(rate_r, args.sweep_seconds)
        sweep.append(row)
        if row["served_GBps"] < 0.85 * row["offered_GBps"]:
            break                                       # saturated: the server no longer keeps up
    for p in pipes.values():
        if p.status() != 0:
            raise RuntimeError("serial path reported an error in the sweep")

    # ---------------- end to end: pinned host payloads in, encoded streams out
    E = min(100, M)
    host = [it[1].cpu().pin_memory() for it in items[:E]]
    dev_in = [torch.empty_like(it[1]) for it in items[:E]]
    e2e_in = sum(h.numel() * h.element_size() for h in host)
    e2e_out = 0
    torch.cuda.synchronize()
    ts = time.monotonic()
    tk = []
    for h, d, it in zip(host, dev_in, items[:E]):
        d.copy_(h, non_blocking=True)
        cur.synchronize()
        tk.append(srv.submit(d, it[2], keep=False))
    outs = []
    for t in tk:
        res = srv.wait(t)
        nw = (res["total_bits"] + 31) // 32
        buf = torch.empty(max(1, nw), dtype=torch.int32).pin_memory()
        buf.copy_(huff.device_view(res["d_out"], 4 * max(1, nw)).view(torch.int32))
        e2e_out += 4 * nw
        outs.append(buf)
        srv.release(t)
    e2e_gbps = e2e_in / (time.monotonic() - ts) / 1e9
    srv.close()

    # ---------------- sampled parity against the oracle
    import oracle
    oracle.build()
    checked = 0
    for i, (tb, words, offs) in sampled.items():
        width, n, nbins, _ = synth.served_request(i)
        a = synth.served_symbols(i)
        book = oracle.codebook(oracle.histogram(a, nbins))
        w, o, otb = oracle.encode(a, book, chunk_log2=10)
        if otb != tb or not np.array_equal(words, w) or not np.array_equal(offs, o):
            raise RuntimeError(f"served request {i} differs from the oracle")
        checked += 1

    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        gbs, samp = oracle_served_leg()
        cpu = {"value": round(gbs, 4), "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": samp}
    peak, peak_kind = load_peak()
    line = {
        "metric": "huffman_served_encode_input_GBps",
        "value": round(served_gbps, 3), "unit": "GB/s", "n_gpus": world, "steps": count, "warmup": 8,
        "ms_per_step": round((t_end - t0) / count * 1e3, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8/u16", "data": "synthetic",
        "config": {"workload": "served", "rate_per_s": rate, "duration_s": duration, "requests": count,
                   "input": WORKLOADS["served"][2], "budget_GB": budget >> 30, "nstreams": 4, "max_batch": 64,
                   "parallelism": f"replicas{world}", "l2": "requests stream through (mean 12 MB each)"},
        "latency_ms": {"p50": round(_pct(lat_ms, 50), 3), "p99": round(_pct(lat_ms, 99), 3),
                       "max": round(max(lat_ms), 3), "from": "scheduled arrival to completion on the device"},
        "serial_plain_calls": {"GBps": round(serial_gbps, 3), "p50_ms": round(_pct(slat, 50), 3),
                               "p99_ms": round(_pct(slat, 99), 3), "max_ms": round(max(slat), 3)},
        "saturation": {"requests": M, "bytes": sat_bytes, "served_GBps": round(sat_served, 3),
                       "serial_GBps": round(sat_serial, 3), "speedup": round(sat_served / sat_serial, 3),
                       "batches": sat_stats["batches"] - stats["batches"]},
        "server": {k: stats[k] for k in ("batches", "max_batch_jobs", "max_concurrent_batches", "pool_peak")},
        "submit_late_max_ms": round(late * 1e3, 3),
        "rate_sweep": {"seconds_per_rate": args.sweep_seconds,
                       "requests": f"the {M} closed-loop requests, reused cyclically",
                       "latency_from": "scheduled arrival to completion (server: device completion seen by the "
                                       "server; serial: after the stream synchronises)",
                       "stop": "after the first rate at which the server delivers < 85% of the offered load",
                       "points": sweep},
        "parity_sampled": checked,
        "roofline": {"bound": "hbm", "kernel": "served pipeline at saturation (histogram + codebook + encode)",
                     "achieved": round(sat_served * 2.0, 2), "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": round(sat_served * 2.0 / peak, 4), "traffic": None,
                     "note": "input bytes read twice (histogram, encode); output bytes not counted"},
        "e2e": {"value": round(e2e_gbps, 3), "unit": "GB/s", "h2d_bytes_per_step": e2e_in // E,
                "d2h_bytes_per_step": e2e_out // E, "requests": E},
        "gpu_launches": launches,
        "cpu_baseline": cpu,
        "clocks": clk,
    }
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="hpc_field", choices=sorted(WORKLOADS))
    ap.add_argument("--chunk-log2", dest="chunk_log2", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--merge", default="scan", choices=["scan", "shuffle"],
                    help="encode layout: fused single pass (scan) or the paper's three kernels (shuffle)")
    ap.add_argument("--rate", type=float, default=2000.0, help="served: arrivals per second")
    ap.add_argument("--duration", type=float, default=60.0, help="served: seconds of arrivals")
    ap.add_argument("--saturation-requests", type=int, default=1000, help="served: closed-loop requests")
    ap.add_argument("--sweep-rates", type=lambda v: [float(x) for x in v.split(",")],
                    default=[2000.0, 4000.0, 8000.0, 16000.0, 32000.0, 64000.0, 128000.0],
                    help="served: open-loop rates of the sweep (req/s, comma separated)")
    ap.add_argument("--sweep-seconds", type=float, default=1.0, help="served: seconds of arrivals per sweep rate")
    ap.add_argument("--alphabets", type=lambda v: [int(x) for x in v.split(",")],
                    default=[8192, 65536, 262144, 1048576], help="large_alphabet: alphabet sizes")
    ap.add_argument("--no-sub-records", action="store_true",
                    help="hpc_field: leave out the batched and served sub-records")
    args = ap.parse_args()
    world, rank, local = dist_setup(args)
    line = None
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == "batched_fields":
        line = run_batched(args, world, rank, local)
    elif args.workload == "served":
        line = run_served(args, world, rank, local)
    elif args.workload == "large_alphabet":
        line = run_large_alphabet(args, world, rank, local)
    else:
        line = run_ours(args, world, rank, local)
        if args.workload == "hpc_field" and not args.no_sub_records:
            # the batched and served forms, each with its own timing, as
            # sub-records of the same line (no CPU leg of their own)
            import torch
            torch.cuda.empty_cache()
            sub = argparse.Namespace(**vars(args))
            sub.no_cpu_baseline = True
            sub.duration = SUB_SERVED_SECONDS
            b = run_batched(sub, world, rank, local)
            torch.cuda.empty_cache()
            sv = run_served(sub, world, rank, local)
            torch.cuda.empty_cache()
            if line is not None:
                drop = ("n_gpus", "higher_is_better", "scaling", "vs_baseline", "data", "cpu_baseline", "warmup")
                line["batched"] = {k: v for k, v in b.items() if k not in drop}
                line["served"] = {k: v for k, v in sv.items() if k not in drop}
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
