"""Benchmark of the batched AES-CTR offload on GB300 (one JSON line on stdout).

Workload (the batched varlen case): 4096 requests, each with its own random
key (AES-128 / AES-256, 50/50) and IV, lengths log-uniform on [1 KiB, 8 MiB],
25% with a 1..15-byte tail; about 3.8 GB of payload per step.  A step is one
launch of the persistent batch kernel over all 4096 requests (a CUDA-graph
plan: counter reset + kernel).  Inputs (3.8 GB) are far larger than L2
(129 MB), so no L2 flush is needed between steps.

Also reported: the same requests as 4096 single-buffer launches (per-call),
p50/p99 latency of a 1 MiB offload through the per-call path (aes_ctr +
cudaEventQuery polling) and the served path (offload_submit + offload_poll),
the end-to-end figure with payloads in pinned host memory, the roofline of
the dominant kernel, SM clocks sampled during the timed region, and the CPU
oracle timed on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs its own replica of the workload on
its own GPU (independent requests, no data-path collective: weak scaling).
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

from paper_2607_02630_gb300 import replicas as R  # noqa: E402
from paper_2607_02630_gb300 import workloads as W  # noqa: E402

METRIC = "AES-CTR GB/s (% roofline) batched vs per-call; p50/p99 1 MiB offload µs"
UNIT = "GB/s"
WORKLOAD = "batched varlen AES-CTR: 4096 requests, own key (AES-128/256 50/50) and IV each, " \
           "lengths log-uniform 1 KiB..8 MiB, 25% with 1..15-byte tails"


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except OSError:
            self.proc = None
        time.sleep(0.25)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(2)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons, pw = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                pw.append(float(parts[3]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        loaded = [s for s, p in zip(sm, pw)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(pw) if pw else None}


def dist_env():
    return R.world_from_env()


KERNEL_SOURCES = ["paper_2607_02630_gb300/csrc/batch.cu", "paper_2607_02630_gb300/csrc/tile.cuh",
                  "paper_2607_02630_gb300/csrc/aes_ttable.cuh", "paper_2607_02630_gb300/csrc/common.cuh"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "batch_ttable_kernel.traffic.txt")


def kernel_source_hash() -> str:
    import hashlib

    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def captured_traffic(step_bytes: int):
    """DRAM bytes (read + write) per launch of the batch kernel from the
    committed ncu capture, scaled from the captured case to this launch by
    payload bytes; None if the kernel changed since the capture."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.loads(f.readline())
    except (OSError, ValueError):
        return None
    if rec.get("kernel_src_sha") != kernel_source_hash():
        return None
    per_byte = rec["dram_bytes"] / rec["payload_bytes"]
    return int(per_byte * step_bytes)


def ttable_lookups(w) -> int:
    """Shared-memory lookups the T-table method needs for workload w: 16*Nr
    per 16-byte block, except that counter-mode caching replaces the 32
    lookups of rounds 1-2 by 5 per block plus 27 per 256-block counter group."""
    total = 0
    for n, b, iv in zip(w.lengths, w.bits, w.ivs):
        nb = (int(n) + 15) // 16
        if nb == 0:
            continue
        nr = int(b) // 32 + 6
        v0 = int(iv[15])
        groups = ((v0 + nb - 1) >> 8) + 1
        total += nb * (16 * nr - 27) + 27 * groups
    return total


def bitslice_ops(w) -> float:
    """Logic ops the bitsliced method needs for workload w: per 32 blocks
    (one thread's planes) 16 S-box circuits of 113 gates per round,
    MixColumns' 416 xors per full round and 128 key xors per round key."""
    total = 0.0
    for n, b in zip(w.lengths, w.bits):
        nb = (int(n) + 15) // 16
        nr = int(b) // 32 + 6
        total += nb * (16 * 113 * nr + 416 * (nr - 1) + 128 * (nr + 1)) / 32.0
    return total


def measured_rates(A):
    """aes_measure_peaks on this GPU (per-SM issue rates from clock64, link
    bandwidths from CUDA events); None if the probe fails."""
    try:
        return A.measure_peaks()
    except Exception as e:  # reported, not fatal: the roofline then says so
        return {"error": str(e)}


# --------------------------------------------------------------------- oracle leg

def oracle_sample(w, budget_s: float, nthreads: int):
    """Time the CPU oracle on a prefix of the requests of `w` sized to take
    about budget_s seconds (calibrated on a 4 MiB probe)."""
    import oracle

    oracle.build()
    probe = w.payload[: 4 << 20]
    key = w.key_of(0)
    t0 = time.perf_counter()
    oracle.ctr_mt(key, int(w.bits[0]), w.ivs[0], probe, nthreads)
    rate = probe.size / max(time.perf_counter() - t0, 1e-6)
    target = rate * budget_s
    idx, acc = [], 0
    for i in range(w.n):
        if acc >= target:
            break
        idx.append(i)
        acc += int(w.lengths[i])
    return idx, acc


def run_oracle(w, idx, nthreads: int) -> float:
    import oracle

    t0 = time.perf_counter()
    for i in idx:
        o, n = int(w.offsets[i]), int(w.lengths[i])
        oracle.ctr_mt(w.key_of(i), int(w.bits[i]), w.ivs[i], w.payload[o: o + n], nthreads)
    return time.perf_counter() - t0


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine
    type), reported beside the oracle timings."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=5).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform

    return platform.machine()


def workload_name(requests: int) -> str:
    return WORKLOAD if requests == 4096 else f"{requests} requests of: " + WORKLOAD


def cpu_study(nthreads: int) -> dict:
    """The oracle on single buffers of the configs' sizes, one thread and all
    cores, AES-128 and AES-256 (payload GB/s; one timed run after a warm-up)."""
    import oracle

    oracle.build()
    g = W.rng(W.SEED_BASE + 14)
    rows = []
    for n, threads in ((1 << 20, 1), (8 << 20, 1), (1 << 20, nthreads), (8 << 20, nthreads), (64 << 20, nthreads)):
        data = W.random_bytes(g, n)
        for bits in (128, 256):
            key, iv = W.random_bytes(g, bits // 8), W.random_bytes(g, 16)
            oracle.ctr_mt(key, bits, iv, data[: 1 << 16], threads)
            t0 = time.perf_counter()
            oracle.ctr_mt(key, bits, iv, data, threads)
            secs = time.perf_counter() - t0
            rows.append({"bytes": n, "bits": bits, "threads": threads, "gbs": round(n / secs / 1e9, 6)})
    return {"cpu": cpu_model(), "cores": nthreads, "rows": rows}


def reference_arm(args, ws, rank):
    if rank != 0:
        return 0
    if args.cpu_study:
        print(json.dumps({"impl": "reference", "cpu_study": cpu_study(os.cpu_count() or 1)}), flush=True)
        return 0
    nthreads = os.cpu_count() or 1
    w = W.batch_varlen(n=args.requests, seed=W.SEED_BASE + 3)
    per_step_s = args.reference_step_seconds
    if per_step_s is None:
        per_step_s = max(0.25, min(8.0, 150.0 / max(1, args.steps + args.warmup)))
    idx, nbytes = oracle_sample(w, per_step_s, nthreads)
    for _ in range(args.warmup):
        run_oracle(w, idx[:1], nthreads)
    times = [run_oracle(w, idx, nthreads) for _ in range(args.steps)]
    total = sum(times)
    value = nbytes * args.steps / total / 1e9
    sample = f"first {len(idx)} of {w.n} requests ({nbytes / 1e6:.1f} MB) per step, oracle_ctr_mt"
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic", "config": {"workload": workload_name(args.requests),
                                        "global_batch": args.requests * args.gpus, "seq_len": None,
                                        "parallelism": f"replicas{args.gpus}"},
        "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": nthreads, "cpu": cpu_model(),
                         "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def sweep(args, rank, local):
    """Single-buffer sweep: for every size, key size and cipher variant the
    median of --sweep-reps aes_ctr launches (CUDA events on the launch
    stream), counter low word starting at 2^32 - 8.  Buffers rotate through
    a pool, and L2 is flushed (a write of twice its size) before every timed
    launch, so every launch reads its input from HBM."""
    import torch

    from paper_2607_02630_gb300 import aesoffload as A
    from paper_2607_02630_gb300 import build as libbuild

    torch.cuda.set_device(local)
    libbuild.build()
    A.lib()
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    sh = int(stream.cuda_stream)
    props = torch.cuda.get_device_properties(dev)
    nsm, l2 = props.multi_processor_count, props.L2_cache_size
    pk, pk_kind = peaks()
    mhz = float(pk.get("sm_max_mhz", 2070.0))
    sizes = [int(x) for x in args.sweep_sizes.split(",")]
    bits_list = [int(x) for x in args.sweep_bits.split(",")]
    variants = {"ttable": dict(variant=1, threads=512, blocks_per_thread=1),
                "bitslice": dict(variant=2, threads=128), "auto": {}}
    chosen = [v for v in args.sweep_variants.split(",")]
    pool_bytes = max(2 * l2 + (64 << 20), max(sizes))
    flush = torch.empty(2 * l2, dtype=torch.uint8, device=dev)
    rows = []
    with ClockSampler(local) as clk:
        for n in sizes:
            nbuf = min(max(1, -(-pool_bytes // n)), args.sweep_reps + 3)
            src = torch.empty(nbuf * n, dtype=torch.uint8, device=dev).random_(0, 256)
            dst = torch.empty_like(src)
            for bits in bits_list:
                w = W.single_buffer(16, bits, seed=W.SEED_BASE + 2, low32=0xFFFFFFF8)
                ctx = A.Context(w.key.tobytes(), bits)
                iv = w.iv.tobytes()
                nblocks = (n + 15) // 16
                nr = bits // 32 + 6
                for name in chosen:
                    shape = variants[name]
                    for k in range(3):
                        A.ctr(ctx, iv, src.data_ptr() + (k % nbuf) * n, dst.data_ptr() + (k % nbuf) * n, n,
                              stream=sh, **shape)
                    times = []
                    for k in range(args.sweep_reps):
                        a = torch.cuda.Event(enable_timing=True)
                        b = torch.cuda.Event(enable_timing=True)
                        o = (k % nbuf) * n
                        with torch.cuda.stream(stream):
                            flush.fill_(k & 255)
                        a.record(stream)
                        A.ctr(ctx, iv, src.data_ptr() + o, dst.data_ptr() + o, n, stream=sh, **shape)
                        b.record(stream)
                        stream.synchronize()
                        times.append(a.elapsed_time(b) / 1e3)
                    t = statistics.median(times)
                    gbs = n / t / 1e9
                    if name == "bitslice":
                        # ALU-bound: logic ops at 64 lanes/clk/SM; floor per 32 blocks:
                        # 16 Boyar-Peralta S-boxes (113 gates) per round, MixColumns
                        # (416 xors) per full round, AddRoundKey (128 xors) per key
                        ops = (16 * 113 * nr + 416 * (nr - 1) + 128 * (nr + 1)) / 32.0
                        roof = nsm * mhz * 1e6 * 64.0 / ops * 16 / 1e9
                        bound = "alu (LOP3, 64/clk/SM)"
                    else:
                        groups = ((255 + nblocks - 1) >> 8) + 1
                        lookups = nblocks * (16 * nr - 27) + 27 * groups
                        roof = n / (lookups / (32.0 * nsm * mhz * 1e6)) / 1e9
                        bound = "shared-memory wavefronts (32 lookups/clk/SM)"
                    rows.append({"bytes": n, "bits": bits, "variant": name, "us": round(t * 1e6, 3),
                                 "gbs": round(gbs, 2), "roofline_gbs": round(min(roof, float(pk.get("hbm_gbs", 6784.5)) / 2), 1),
                                 "frac": round(gbs / min(roof, float(pk.get("hbm_gbs", 6784.5)) / 2), 4),
                                 "bound": bound,
                                 "hbm_gbs_moved": round(2 * n / t / 1e9, 1)})
                ctx.close()
            del src, dst
            torch.cuda.empty_cache()
    if rank == 0:
        print(json.dumps({"metric": "AES-CTR single-buffer sweep GB/s (% roofline)", "unit": UNIT,
                          "l2_bytes": l2, "peak_kind": pk_kind, "sm_max_mhz": mhz,
                          "clocks": clk.summary(), "rows": rows}), flush=True)
    return 0


def _pct(x, q):
    x = [v for v in x if v >= 0]
    return round(float(np.percentile(x, q)), 2) if x else None


def served(args, rank, local):
    """Served-mode studies through the native open-loop drivers.

    Open loop: the saturated request rate R_sat of the served path is
    measured first (all arrivals at t = 0); then Poisson arrivals at 0.2, 0.4,
    0.6, 0.8 and 1.0 x R_sat, split over 8 submitter threads, for the served
    path and, on the same schedule, for per-call aes_ctr launches polled with
    cudaEventQuery.  Sizes: 70% 1 MiB, 10% 8 MiB, 20% log-uniform 4-64 KiB;
    64 resident keys (AES-128/256 50/50), one drawn per request.
    Stream: AES-256, 2048 x 8 MiB (16 GiB), at most 512 in flight, an HBM
    budget of 20 GiB and then 2 GiB (back-pressure), a new random key every
    1024 requests; sustained GB/s and p50/p99 (the same stream is checked
    against the oracle by tests/test_server_gpu.py)."""
    import torch

    from paper_2607_02630_gb300 import aesoffload as A
    from paper_2607_02630_gb300 import build as libbuild

    torch.cuda.set_device(local)
    libbuild.build()
    A.lib()
    dev = torch.device("cuda", local)
    MiB = 1 << 20
    out = {"metric": "served AES-CTR: open-loop p50/p99 and GB/s vs per-call; 8 MiB stream", "unit": UNIT}

    # ---------------- open loop
    n = args.served_requests
    sizes = W.served_sizes(n, seed=W.SEED_BASE + 4)
    kbits, kbytes = W.key_set(64, seed=W.SEED_BASE + 5)
    g = W.rng(W.SEED_BASE + 6)
    key_idx = g.integers(0, 64, n)
    ivs = W.random_bytes(g, 16 * n).reshape(n, 16)
    pool_n, ring_n = 64, 2048
    gen = torch.Generator(device=dev).manual_seed(W.SEED_BASE + 4)
    pool = torch.randint(0, 256, (pool_n * 8 * MiB,), dtype=torch.uint8, device=dev, generator=gen)
    ring = torch.empty(ring_n * 8 * MiB, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize(dev)  # the served kernel runs on its own stream
    ctxs = [A.Context(kbytes[i, : kbits[i] // 8].tobytes(), int(kbits[i])) for i in range(64)]
    cm = args.claim_mode

    # The resident kernel holds all but 4 SMs while it runs, so the per-call
    # baseline must never run beside it: every served run gets its own
    # server, closed (resident kernel stopped) before the per-call run.
    def new_server(**kw):
        srv = A.Server(slots=1024, max_keys=64, idle_timeout_us=2_000_000, claim_mode=cm, **kw)
        sl = [srv.key_register(kbytes[i, : kbits[i] // 8].tobytes(), int(kbits[i])) for i in range(64)]
        return srv, np.array(sl)

    reqs = np.zeros(n, dtype=A.drive_dtype())
    reqs["iv"] = ivs
    reqs["inp"] = pool.data_ptr() + (np.arange(n) % pool_n) * 8 * MiB
    reqs["out"] = ring.data_ptr() + (np.arange(n) % ring_n) * 8 * MiB
    reqs["len"] = sizes
    served_reqs = reqs.copy()
    pc_reqs = reqs.copy()
    pc_reqs["key_slot"] = key_idx
    total = int(sizes.sum())
    one_mib = sizes == MiB

    def run_served(arrivals, **kw):
        srv, sl = new_server(**kw)
        try:
            served_reqs["key_slot"] = sl[key_idx]
            served_reqs["arrival_s"] = 0.0
            A.drive_served(srv, served_reqs[: min(n, 2000)], 8)  # warm-up (launch, key pages)
            served_reqs["arrival_s"] = arrivals
            return A.drive_served(srv, served_reqs, 8)
        finally:
            srv.close()

    def run_per_call(arrivals):
        pc_reqs["arrival_s"] = 0.0
        A.drive_per_call(ctxs, pc_reqs[: min(n, 2000)], 8)  # warm-up
        pc_reqs["arrival_s"] = arrivals
        return A.drive_per_call(ctxs, pc_reqs, 8)

    zeros = np.zeros(n)
    lat, res = run_served(zeros)
    r_sat = n / res["elapsed_s"]
    sat = {"req_per_s": round(r_sat, 1), "gbs": round(total / res["elapsed_s"] / 1e9, 2),
           "p50_us": _pct(lat, 50), "p99_us": _pct(lat, 99), "errors": res["errors"]}
    lat_pc, res_pc = run_per_call(zeros)
    sat_pc = {"req_per_s": round(n / res_pc["elapsed_s"], 1), "gbs": round(total / res_pc["elapsed_s"] / 1e9, 2),
              "errors": res_pc["errors"]}
    rates = []
    for frac in (0.2, 0.4, 0.6, 0.8, 1.0):
        rate = frac * r_sat
        arr = W.poisson_arrivals(n, rate, seed=W.SEED_BASE + 40 + int(frac * 10))
        lat, res = run_served(arr)
        lat_pc, res_pc = run_per_call(arr)
        rates.append({
            "offered_frac_of_rsat": frac, "offered_req_per_s": round(rate, 1),
            "served": {"p50_us": _pct(lat, 50), "p99_us": _pct(lat, 99),
                       "p50_1mib_us": _pct(lat[one_mib], 50), "p99_1mib_us": _pct(lat[one_mib], 99),
                       "gbs": round(res["bytes"] / res["elapsed_s"] / 1e9, 2), "errors": res["errors"],
                       "eagain_retries": res["eagain_retries"]},
            "per_call": {"p50_us": _pct(lat_pc, 50), "p99_us": _pct(lat_pc, 99),
                         "p50_1mib_us": _pct(lat_pc[one_mib], 50), "p99_1mib_us": _pct(lat_pc[one_mib], 99),
                         "gbs": round(res_pc["bytes"] / res_pc["elapsed_s"] / 1e9, 2), "errors": res_pc["errors"]}})
    # the same requests on a server cut for throughput (fixed 1024-block tiles)
    lat_t, res_t = run_served(zeros, tile_blocks=1024)
    sat_t = {"req_per_s": round(n / res_t["elapsed_s"], 1), "gbs": round(total / res_t["elapsed_s"] / 1e9, 2),
             "errors": res_t["errors"], "config": "tile_blocks=1024"}
    out["open_loop"] = {"requests_per_rate": n, "payload_bytes_per_rate": total, "submitter_threads": 8,
                        "claim_mode": cm,
                        "saturation_served": sat, "saturation_served_tile1024": sat_t,
                        "saturation_per_call": sat_pc, "rates": rates}
    del pool, ring, ctxs
    torch.cuda.empty_cache()

    # ---------------- large stream
    n5, big = 2048, 8 * MiB
    gen = torch.Generator(device=dev).manual_seed(W.SEED_BASE + 5)
    src = torch.randint(0, 256, (n5 * big,), dtype=torch.uint8, device=dev, generator=gen)
    dst = torch.empty_like(src)
    torch.cuda.synchronize(dev)
    g = W.rng(W.SEED_BASE + 7)
    keys5 = [W.random_bytes(g, 32) for _ in range(n5 // 1024)]
    ivs5 = W.random_bytes(g, 16 * n5).reshape(n5, 16)
    stream = {}
    for budget in (20 << 30, 2 << 30):
        srv = A.Server(slots=512, max_keys=4, hbm_budget=budget, idle_timeout_us=2_000_000, claim_mode=cm)
        ks = [srv.key_register(k.tobytes(), 256) for k in keys5]
        r5 = np.zeros(n5, dtype=A.drive_dtype())
        r5["key_slot"] = np.array(ks)[np.arange(n5) // 1024]
        r5["iv"] = ivs5
        r5["inp"] = src.data_ptr() + np.arange(n5) * big
        r5["out"] = dst.data_ptr() + np.arange(n5) * big
        r5["len"] = big
        lat, res = A.drive_served(srv, r5, 8)  # closed: everything offered at t = 0
        gbs = res["bytes"] / res["elapsed_s"] / 1e9
        r5["arrival_s"] = np.arange(n5) / (0.9 * n5 / res["elapsed_s"])  # paced at 90% of that rate
        lat_p, res_p = A.drive_served(srv, r5, 8)
        stream[f"budget_{budget >> 30}GiB"] = {
            "sustained_gbs": round(gbs, 2), "eagain_retries": res["eagain_retries"], "errors": res["errors"],
            "paced_90pct": {"p50_us": _pct(lat_p, 50), "p99_us": _pct(lat_p, 99),
                            "gbs": round(res_p["bytes"] / res_p["elapsed_s"] / 1e9, 2)}}
        srv.close()
    roof = None
    try:
        pk, _ = peaks()
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        lookups_per_block = 16 * 14 - 27 + 27 / 256.0
        roof = 32.0 * nsm * float(pk.get("sm_max_mhz", 2070.0)) * 1e6 / lookups_per_block * 16 / 1e9
    except Exception:
        pass
    stream["roofline_gbs_aes256"] = round(roof, 1) if roof else None
    out["stream_8mib_aes256"] = stream
    if rank == 0:
        print(json.dumps(out), flush=True)
    return 0


def reroute_sweep(args, rank, local):
    """The reroute block-size sweep: a single-event-loop asyncio server at 50
    closed-loop clients (a spawned process, 127.0.0.1 TCP), per AES-128 block
    size from 4 KiB to 256 MiB (the paper sweeps 4 KiB to 8 MiB): single-op
    latency of the blocking offload, and
    requests/s when the loop waits for the offload (sync), hands it to a
    32-thread executor, or submits it to the served path and suspends."""
    import torch

    from paper_2607_02630_gb300 import aesoffload as A
    from paper_2607_02630_gb300 import build as libbuild
    from paper_2607_02630_gb300 import reroute as RR

    torch.cuda.set_device(local)
    libbuild.build()
    A.lib()
    dev = torch.device("cuda", local)
    sizes = [int(x) for x in args.reroute_sizes.split(",")]
    srv = A.Server(slots=256, max_keys=64, idle_timeout_us=5_000_000)
    key = bytes(W.random_bytes(W.rng(W.SEED_BASE + 9), 16))
    rows = []
    try:
        for i, n in enumerate(sizes):
            row = RR.run_point(A, torch, dev, n, srv, key, 128, nclients=args.reroute_clients,
                               seconds=args.reroute_seconds, warmup=0.5, executor_threads=32,
                               seed=W.SEED_BASE + 10 + i)
            row.pop("_outputs")
            rows.append(row)
            torch.cuda.empty_cache()
    finally:
        srv.close()
    out = {"metric": "reroute on a single-event-loop server: req/s sync vs executor vs served, by block size",
           "unit": "req/s", "rows": rows,
           "config": {"server": "python asyncio, one event loop", "clients": args.reroute_clients,
                      "executor_threads": 32, "cipher": "AES-128-CTR", "payload": "resident in HBM",
                      "seconds_per_point": args.reroute_seconds}}
    if rank == 0:
        print(json.dumps(out), flush=True)
    return 0


def emulated_study(args, rank, local):
    """Latency under offered load over a controlled emulated offload (the
    paper's one emulated experiment: open-loop Poisson arrivals, 20 us
    offload): per offered rate, p50/p99 latency and achieved rate of a
    blocking server (each of 8 threads waits for its offload before taking
    the next request) and of an overlapping one (threads submit at arrival
    and poll), both through the served path (offload_submit_emulated)."""
    import torch

    from paper_2607_02630_gb300 import aesoffload as A
    from paper_2607_02630_gb300 import build as libbuild

    torch.cuda.set_device(local)
    libbuild.build()
    A.lib()
    rates = [float(x) for x in args.emulated_rates.split(",")]
    srv = A.Server(slots=4096, max_keys=1, idle_timeout_us=2_000_000)
    rows = []
    try:
        warm = np.zeros(2000, dtype=A.drive_dtype())
        A.drive_served(srv, warm, 8, emulated_ns=args.emulated_ns)
        for i, rate in enumerate(rates):
            n = int(min(max(4000, rate * args.emulated_seconds), 400_000))
            reqs = np.zeros(n, dtype=A.drive_dtype())
            reqs["arrival_s"] = W.poisson_arrivals(n, rate, seed=W.SEED_BASE + 60 + i)
            row = {"offered_req_per_s": rate, "requests": n}
            for mode, blocking in (("blocking", True), ("overlap", False)):
                lat, res = A.drive_served(srv, reqs, 8, blocking=blocking, emulated_ns=args.emulated_ns)
                ok = lat[lat >= 0]
                row[mode] = {"p50_us": _pct(ok, 50), "p99_us": _pct(ok, 99),
                             "achieved_req_per_s": round(len(ok) / res["elapsed_s"], 1), "errors": res["errors"]}
            rows.append(row)
    finally:
        srv.close()

    def knee(mode):
        base = rows[0][mode]["p99_us"]
        best = None
        for r in rows:
            m = r[mode]
            if m["achieved_req_per_s"] >= 0.95 * r["offered_req_per_s"] and m["p99_us"] <= 10 * base:
                best = r["offered_req_per_s"]
        return best

    out = {"metric": "latency under offered load over an emulated offload: blocking vs overlapping server",
           "unit": "us", "offload_ns": args.emulated_ns, "threads": 8, "rows": rows,
           "knee_req_per_s": {"blocking": knee("blocking"), "overlap": knee("overlap")},
           "knee_rule": "highest offered rate served at >= 95 % with p99 <= 10x the lowest-rate p99"}
    if rank == 0:
        print(json.dumps(out), flush=True)
    return 0


def conflict_study(args, rank, local):
    """The conflict detector with a real GPU offload: 16 handlers on one
    event loop serve requests that read one of 64 shared counters, park at an
    AES-128-CTR served request (1 MiB and 8 MiB), and write the counter back
    incremented; lost updates, conflicts and requests/s for unprotected
    overlap, a coarse lock, detection only, and enforcement.  Also the cost
    of one guarded write in this (CUDA) process: one handler, no offload,
    detection on vs off."""
    import torch

    from paper_2607_02630_gb300 import aesoffload as A
    from paper_2607_02630_gb300 import build as libbuild

    torch.cuda.set_device(local)
    libbuild.build()
    A.lib()
    dev = torch.device("cuda", local)
    handlers, requests = 16, args.conflict_requests
    sizes = [int(x) for x in args.conflict_bytes.split(",")]
    stride = (max(sizes) + 255) // 256 * 256
    gen = torch.Generator(device=dev).manual_seed(W.SEED_BASE + 11)
    src = torch.randint(0, 256, (handlers * stride,), dtype=torch.uint8, device=dev, generator=gen)
    dst = torch.empty_like(src)
    torch.cuda.synchronize(dev)  # the served kernel runs on its own stream
    srv = A.Server(slots=256, max_keys=1, idle_timeout_us=2_000_000)
    names = {A.CDET_UNPROTECTED: "unprotected", A.CDET_LOCK: "coarse_lock", A.CDET_DETECT: "detect",
             A.CDET_ENFORCE: "enforce"}
    studies = []
    try:
        ks = srv.key_register(bytes(W.random_bytes(W.rng(W.SEED_BASE + 12), 16)), 128)
        for nbytes in sizes:
            # per-handler buffers at `stride` apart: pass views so the stride matches
            def run(mode, n):
                return A.conflict_run(mode, handlers, n, 64, server=srv, key_slot=ks, buf_in=src, buf_out=dst,
                                      nbytes=nbytes, emulate_stores=False)
            run(A.CDET_UNPROTECTED, 500)  # warm-up
            rows = {}
            for mode, name in names.items():
                r = run(mode, requests)
                rows[name] = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in r.items()}
            for mode, name in ((A.CDET_DETECT, "detect_emulated_stores"), (A.CDET_ENFORCE, "enforce_emulated_stores")):
                r = A.conflict_run(mode, handlers, requests, 64, server=srv, key_slot=ks, buf_in=src, buf_out=dst,
                                   nbytes=nbytes, emulate_stores=True)
                rows[name] = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in r.items()}
            studies.append({"offload": f"served AES-128-CTR, {nbytes} bytes per request, payload in HBM",
                            "rows": rows,
                            "enforce_vs_lock": round(rows["enforce"]["req_per_s"] / rows["coarse_lock"]["req_per_s"], 2),
                            "enforce_emulated_vs_lock": round(rows["enforce_emulated_stores"]["req_per_s"]
                                                              / rows["coarse_lock"]["req_per_s"], 2),
                            "enforce_vs_unprotected": round(rows["enforce"]["req_per_s"]
                                                            / rows["unprotected"]["req_per_s"], 3)})
        # the paper's taxonomy of shared state: detection on each pattern,
        # over the 1 MiB served offload (only the shared aggregate is hazardous)
        pats = {A.CDET_PATTERN_SHARED: "shared_unlocked", A.CDET_PATTERN_READONLY: "read_only",
                A.CDET_PATTERN_PER_CONN: "per_connection", A.CDET_PATTERN_LOCKED: "lock_protected"}
        taxonomy = {}
        for pat, name in pats.items():
            r = A.conflict_run(A.CDET_DETECT, handlers, requests, 64, server=srv, key_slot=ks, buf_in=src,
                               buf_out=dst, nbytes=min(sizes), pattern=pat, emulate_stores=False)
            taxonomy[name] = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in r.items()}
        n1 = 5000
        off = A.conflict_run(A.CDET_UNPROTECTED, 1, n1, 1, offload_ns=0)
        on = A.conflict_run(A.CDET_DETECT, 1, n1, 1, offload_ns=0, emulate_stores=False)
        fault_us = (on["elapsed_s"] - off["elapsed_s"]) / n1 * 1e6
        on_e = A.conflict_run(A.CDET_DETECT, 1, n1, 1, offload_ns=0, emulate_stores=True)
        fault_emu_us = (on_e["elapsed_s"] - off["elapsed_s"]) / n1 * 1e6
        selftest = A.store_selftest(6000)
    finally:
        srv.close()
    out = {"metric": "shared-counter read-modify-write across a GPU offload: lost updates and req/s by guard",
           "unit": "req/s", "handlers": handlers, "counters": 64, "requests": requests, "studies": studies,
           "taxonomy_detect": taxonomy, "taxonomy_bytes": min(sizes),
           "guarded_write_cost_us": round(fault_us, 2),
           "guarded_write_cost_emulated_us": round(fault_emu_us, 2), "store_emulation_selftest": selftest,
           "guarded_write_cost_how": "1 handler, no offload: (detect - unprotected) time per request = one write "
                                     "fault + two mprotect calls, in this CUDA process"}
    if rank == 0:
        print(json.dumps(out), flush=True)
    return 0


def peaks_mode(local):
    """The roofline's denominators, regenerated on this GPU: per-SM issue
    rates (clock64) and host-link bandwidths (CUDA events)."""
    import torch

    from paper_2607_02630_gb300 import aesoffload as A
    from paper_2607_02630_gb300 import build as libbuild

    torch.cuda.set_device(local)
    libbuild.build()
    r = A.measure_peaks()
    pk, pk_kind = peaks()
    f = float(pk.get("sm_max_mhz", 2070.0)) * 1e6
    nsm = r["sms"]
    out = {"metric": "device rates behind the AES-CTR roofline", "rates": r,
           "derived": {"ttable_lookups_per_s_at_max_clock": r["lds32_per_clk_sm"] * nsm * f,
                       "lop3_per_s_at_max_clock": r["lop3_per_clk_sm"] * nsm * f,
                       "sm_max_mhz": f / 1e6, "sm_max_mhz_source": pk_kind},
           "how": "aes_measure_peaks: 2 CTAs x 1024 threads per SM, 8 independent chains a thread, "
                  "clock64 per SM (median over SMs); 256 MiB transfers timed with CUDA events"}
    print(json.dumps(out), flush=True)
    return 0


def served_trace(args, rank):
    """The trace build's step breakdown of one-in-flight served latency
    (paper_2607_02630_gb300.served_trace), in a child process: it loads
    libaesoffload_trace.so, which this process must not have loaded."""
    if rank != 0:
        return 0
    root = os.path.dirname(os.path.abspath(__file__))
    r = subprocess.run([sys.executable, "-m", "paper_2607_02630_gb300.served_trace", "--requests",
                        str(args.served_trace_requests), "--claim-mode", str(args.claim_mode)],
                       capture_output=True, text=True, cwd=root)
    sys.stdout.write(r.stdout)
    sys.stderr.write(r.stderr)
    return r.returncode


# ----------------------------------------------------------------------- our arm

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="only the headline step timing")
    ap.add_argument("--no-e2e", action="store_true", help="skip the pinned-host end-to-end leg")
    ap.add_argument("--requests", type=int, default=4096,
                    help="requests per step (4096 = the benchmark workload; fewer only for profiler captures)")
    ap.add_argument("--oracle-seconds", type=float, default=12.0)
    ap.add_argument("--cpu-study", action="store_true",
                    help="with --impl reference: time the oracle on 1/8/64 MiB buffers, 1 thread and all cores")
    ap.add_argument("--reference-step-seconds", type=float, default=None,
                    help="CPU seconds of oracle work per --impl reference step (default: fit the run in ~150 s)")
    ap.add_argument("--sweep", action="store_true",
                    help="single-buffer sweep instead of the batch step: sizes x key sizes x variants")
    ap.add_argument("--sweep-sizes", default="4096,16384,65536,262144,1048576,4194304,16777216,67108864,268435456")
    ap.add_argument("--sweep-bits", default="128,256")
    ap.add_argument("--sweep-variants", default="ttable,bitslice")
    ap.add_argument("--sweep-reps", type=int, default=20)
    ap.add_argument("--reroute", action="store_true",
                    help="reroute block-size sweep on a single-event-loop server instead of the batch step")
    ap.add_argument("--reroute-sizes", default=",".join(str(4096 << k) for k in range(17)))
    ap.add_argument("--reroute-clients", type=int, default=50)
    ap.add_argument("--reroute-seconds", type=float, default=2.0)
    ap.add_argument("--emulated", action="store_true",
                    help="open-loop study over an emulated offload: blocking vs overlapping server")
    ap.add_argument("--emulated-ns", type=int, default=20_000)
    ap.add_argument("--emulated-rates", default="25000,50000,100000,150000,200000,250000,300000,400000,500000,"
                                                "600000,800000")
    ap.add_argument("--emulated-seconds", type=float, default=0.5)
    ap.add_argument("--conflict", action="store_true",
                    help="conflict-detector study (shared counters across a GPU offload)")
    ap.add_argument("--conflict-bytes", default=f"{1 << 20},{8 << 20}")
    ap.add_argument("--conflict-requests", type=int, default=10000)
    ap.add_argument("--served", action="store_true",
                    help="served-mode studies: open-loop Poisson rates and the large 8 MiB stream")
    ap.add_argument("--served-requests", type=int, default=20000)
    ap.add_argument("--claim-mode", type=int, default=0, choices=[0, 1],
                    help="served studies: 0 = global claim cursor, 1 = per-request claim words")
    ap.add_argument("--served-trace", action="store_true",
                    help="served one-in-flight latency breakdown from the trace build (its own process)")
    ap.add_argument("--served-trace-requests", type=int, default=500)
    ap.add_argument("--batch-shape", default=None,
                    help="variant,threads,tile_blocks,blocks_per_thread: time this batch shape instead of the "
                         "autotuner's pick (profiler captures of the pick)")
    ap.add_argument("--peaks", action="store_true",
                    help="print the roofline's device rates (aes_measure_peaks) as one JSON line and exit")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return reference_arm(args, ws, rank)
    if args.sweep:
        return sweep(args, rank, local)
    if args.reroute:
        return reroute_sweep(args, rank, local)
    if args.emulated:
        return emulated_study(args, rank, local)
    if args.conflict:
        return conflict_study(args, rank, local)
    if args.served:
        return served(args, rank, local)
    if args.served_trace:
        return served_trace(args, rank)
    if args.peaks:
        return peaks_mode(local)

    import torch

    from paper_2607_02630_gb300 import aesoffload as A
    from paper_2607_02630_gb300 import build as libbuild

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    libbuild.build()
    A.lib()
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    sh = int(stream.cuda_stream)

    # ---- workload, resident in HBM
    w = W.batch_varlen(n=args.requests, seed=R.rank_seed(W.SEED_BASE + 3, rank))
    src = torch.from_numpy(w.payload).to(dev)
    dst = torch.empty(w.arena_bytes, dtype=torch.uint8, device=dev)
    ctxs = [A.Context(w.key_of(i).tobytes(), int(w.bits[i])) for i in range(w.n)]
    reqs = [(ctxs[i], w.ivs[i].tobytes(), src.data_ptr() + int(w.offsets[i]),
             dst.data_ptr() + int(w.offsets[i]), int(w.lengths[i])) for i in range(w.n)]
    # the device's rates behind the roofline, then the batch autotuner on
    # these very requests (every candidate shape timed as a graph plan); the
    # plan below uses the shape it picks
    rates = measured_rates(A)
    if not args.no_extras:
        A.autotune()  # the single-buffer shapes per size and key size, for the per-call comparisons
    if args.batch_shape:  # a fixed shape (profiler captures): no tuning
        v, th, tb, nb = (int(x) for x in args.batch_shape.split(","))
        tuned = {"variant": v, "threads": th, "tile_blocks": tb, "ctas": 0, "blocks_per_thread": nb}
        plan = A.BatchPlan(reqs, variant=v, threads=th, tile_blocks=tb, blocks_per_thread=nb)
    else:
        tuned = A.batch_autotune(reqs, sh)
        tuned["candidates_gbs"] = {
            f"v{c['variant']}_t{c['threads']}_tile{c['tile_blocks']}_nb{c['blocks_per_thread']}":
                (round(w.total_bytes / (ms * 1e-3) / 1e9, 1) if ms > 0 else None)
            for c, ms in A.batch_tune_results()}
        plan = A.BatchPlan(reqs)
    step_bytes = plan.nbytes
    torch.cuda.synchronize()

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- headline: K plan launches, events around each on the launch stream
    for _ in range(args.warmup):
        plan.launch(sh)
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for a, b in ev:
            a.record(stream)
            plan.launch(sh)
            b.record(stream)
        t_end.record(stream)
        stream.synchronize()
    barrier()
    elapsed = t_start.elapsed_time(t_end) / 1e3
    per_launch = [a.elapsed_time(b) / 1e3 for a, b in ev]
    elapsed = R.max_over_ranks(elapsed, dist, dev)
    value = R.aggregate_gbs(step_bytes, args.steps, ws, elapsed)
    clocks = clk.summary()

    # ---- roofline of the batch kernel (on-chip bound: shared-memory lookups
    # for the T-tables, logic issue for the bitsliced circuit), from the
    # rates aes_measure_peaks measured on this GPU
    roofline = batch_roofline(torch, dev, w, step_bytes, per_launch, tuned, rates)

    extras = {}
    if not args.no_extras:
        extras = run_extras(A, torch, dev, stream, sh, w, ctxs, reqs, src, dst, step_bytes, args)

    # ---- end to end: payloads in pinned host memory, read/written by the kernel over C2C
    e2e = None if args.no_e2e else run_e2e(A, torch, w, ctxs, args, sh, stream, dist, ws)
    if e2e is not None and rates.get("zero_copy_each_way_gbs"):
        link = rates["zero_copy_each_way_gbs"]
        e2e["link_roof_gbs"] = round(link, 1)
        e2e["frac_of_link_roof"] = round(e2e["value"] / link, 4)
        e2e["link_roof_basis"] = ("aes_measure_peaks: a kernel reading 256 MiB of pinned host memory and writing "
                                  "256 MiB of pinned host memory at once over NVLink-C2C, per direction "
                                  f"(copy engines: {rates['h2d_gbs']:.1f} H2D, {rates['d2h_gbs']:.1f} D2H, "
                                  f"{rates['h2d_d2h_each_way_gbs']:.1f} each way at once)")

    if rank == 0:
        cpu = None
        if ws == 1 and not args.no_extras:
            nthreads = os.cpu_count() or 1
            idx, nbytes = oracle_sample(w, args.oracle_seconds, nthreads)
            secs = run_oracle(w, idx, nthreads)
            cpu = {"value": round(nbytes / secs / 1e9, 6), "unit": UNIT, "cores": nthreads, "cpu": cpu_model(),
                   "kind": "oracle",
                   "sample": f"first {len(idx)} of the 4096 requests ({nbytes / 1e6:.1f} MB), "
                             f"oracle_ctr_mt on {nthreads} threads, {secs:.1f} s"}
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(elapsed / args.steps * 1e3, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic",
            "config": {"workload": workload_name(args.requests),
                       "global_batch": args.requests * ws, "seq_len": None,
                       "parallelism": f"replicas{ws}", "step_bytes": step_bytes,
                       "l2": "no flush: 3.8 GB of inputs per step, far above the 129 MB L2",
                       "launch": "aes_batch_plan_launch (CUDA graph: counter reset + persistent kernel)",
                       "tuned_shape": tuned,
                       "tuner": ("fixed by --batch-shape" if args.batch_shape else
                                 "aes_batch_autotune on these requests before the timed region: 30 shapes "
                                 "(T-table CTAs of 256/512/1024 threads x 1/2/4 blocks per lane x tiles of "
                                 "1024/2048/4096 blocks, and the bitsliced kernel x the 3 tiles), median of 5 "
                                 "graph launches each")},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": args.steps,
            "clocks": clocks,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def batch_roofline(torch, dev, w, step_bytes, per_launch, tuned, rates):
    """The dominant kernel's roofline: achieved payload GB/s per launch
    against the on-chip floor of the variant the tuner picked."""
    pk, pk_kind = peaks()
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max_mhz = float(pk.get("sm_max_mhz", 2070.0))
    launch_s = statistics.mean(per_launch)
    achieved = step_bytes / launch_s / 1e9
    hbm_roof = float(pk.get("hbm_gbs", 6784.5)) / 2.0  # 2 bytes moved per payload byte
    bitsliced = tuned.get("variant") == 2
    measured = "lds32_per_clk_sm" in rates
    if bitsliced:
        work = bitslice_ops(w)
        per_clk = rates["lop3_per_clk_sm"] if measured else 64.0
        what = (f"{work / 1e9:.3f} G logic ops per step (per 32 blocks: 16 S-box circuits of 113 gates per round, "
                f"416 MixColumns xors per full round, 128 key xors per round key) at {per_clk:.1f} lop3 lanes per "
                f"clk per SM")
        kernel = "batch_bitslice_kernel"
    else:
        work = ttable_lookups(w)
        per_clk = rates["lds32_per_clk_sm"] if measured else 32.0
        what = (f"{work / 1e9:.3f} G T-table lookups per step (16*Nr per block, rounds 1-2 counter-cached: 5 per "
                f"block + 27 per 256-block counter group) at {per_clk:.2f} conflict-free 32-bit shared-memory "
                f"loads per clk per SM")
        kernel = "batch_ttable_kernel"
    src = ("measured on this GPU by aes_measure_peaks (clock64 per SM)" if measured
           else f"nominal rate: aes_measure_peaks failed ({rates.get('error')})")
    floor_s = work / (per_clk * nsm * sm_max_mhz * 1e6)
    roof_gbs = step_bytes / floor_s / 1e9
    return {"bound": "alu", "achieved": round(achieved, 2), "peak": round(roof_gbs, 2), "unit": "GB/s",
            "frac": round(achieved / roof_gbs, 4),
            "traffic": captured_traffic(step_bytes) if not bitsliced else None,
            "peak_basis": f"{what} ({src}) x {nsm} SMs x {sm_max_mhz:.0f} MHz ({pk_kind} max clock)",
            "rates": {k: (round(v, 3) if isinstance(v, float) else v) for k, v in rates.items()},
            "hbm_payload_roof_gbs": round(hbm_roof, 1),
            "frac_of_hbm_roof": round(achieved / hbm_roof, 4),
            "kernel": kernel}


def run_extras(A, torch, dev, stream, sh, w, ctxs, reqs, src, dst, step_bytes, args):
    out = {}
    # per-call: the same 4096 requests, one aes_ctr launch each, one stream
    def per_call():
        for r in reqs:
            A.ctr(r[0], r[1], r[2], r[3], r[4], stream=sh)

    per_call()
    stream.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    a.record(stream)
    for _ in range(reps):
        per_call()
    b.record(stream)
    stream.synchronize()
    pc = step_bytes * reps / (a.elapsed_time(b) / 1e3) / 1e9
    # one aes_ctr_batch call (uploads its descriptor table each call) for comparison
    A.batch(reqs, stream=sh)
    stream.synchronize()
    a.record(stream)
    for _ in range(reps):
        A.batch(reqs, stream=sh)
    b.record(stream)
    stream.synchronize()
    one_shot = step_bytes * reps / (a.elapsed_time(b) / 1e3) / 1e9
    # aes_ctr_batch_noalloc over the same requests, in calls of at most 1024
    # (its cap; calls on one stream run one after another, so they may share
    # its static descriptor array)
    def noalloc_step():
        for i in range(0, len(reqs), 1024):
            rc = A.batch_noalloc_status(reqs[i: i + 1024], stream=sh)
            if rc != A.AES_OK:
                raise A.AesError(rc, "aes_ctr_batch_noalloc")

    noalloc_step()
    stream.synchronize()
    a.record(stream)
    for _ in range(reps):
        noalloc_step()
    b.record(stream)
    stream.synchronize()
    na = step_bytes * reps / (a.elapsed_time(b) / 1e3) / 1e9
    out["per_call"] = {"value": round(pc, 3), "unit": UNIT, "launches_per_step": len(reqs),
                       "how": "4096 aes_ctr calls on one stream, tuned shapes"}
    out["batch_noalloc"] = {"value": round(na, 3), "unit": UNIT, "calls_per_step": -(-len(reqs) // 1024),
                            "how": "aes_ctr_batch_noalloc in calls of 1024 requests (descriptor copy + launch "
                                   "each call, no device allocation)"}
    out["batch_one_shot"] = {"value": round(one_shot, 3), "unit": UNIT,
                             "how": "aes_ctr_batch (descriptor upload + launch each call)"}

    # latency of a 1 MiB offload: per-call path with cudaEventQuery polling
    g = W.rng(W.SEED_BASE + 1)
    one = W.single_buffer(1 << 20, 128, seed=W.SEED_BASE + 1)
    s_in = torch.from_numpy(one.payload).to(dev)
    s_out = torch.empty_like(s_in)
    ctx = A.Context(one.key.tobytes(), 128)
    iv = one.iv.tobytes()
    evq = torch.cuda.Event()
    lat = []
    for i in range(50 + 2000):
        t0 = time.perf_counter()
        A.ctr(ctx, iv, s_in, s_out, 1 << 20, stream=sh)
        evq.record(stream)
        while not evq.query():
            pass
        if i >= 50:
            lat.append((time.perf_counter() - t0) * 1e6)
    dev_ms = []
    for i in range(200):
        a.record(stream)
        A.ctr(ctx, iv, s_in, s_out, 1 << 20, stream=sh)
        b.record(stream)
        stream.synchronize()
        dev_ms.append(a.elapsed_time(b))
    out["latency_1mib_per_call_us"] = {"p50": round(float(np.percentile(lat, 50)), 2),
                                       "p99": round(float(np.percentile(lat, 99)), 2),
                                       "device_us_median": round(statistics.median(dev_ms) * 1e3, 2),
                                       "gbs_device": round((1 << 20) / (statistics.median(dev_ms) / 1e3) / 1e9, 2),
                                       "how": "aes_ctr + cudaEventQuery poll, one in flight, 2000 calls"}
    # served path: submit + poll, one in flight
    srv = A.Server(slots=64, max_keys=4, idle_timeout_us=2_000_000)
    try:
        slot = srv.key_register(one.key.tobytes(), 128)
        lat_s = []
        for i in range(50 + 2000):
            t0 = time.perf_counter()
            t = srv.submit(slot, iv, s_in, s_out, 1 << 20)
            while srv.poll(t) == A.AES_PENDING:
                pass
            if i >= 50:
                lat_s.append((time.perf_counter() - t0) * 1e6)
        out["latency_1mib_served_us"] = {"p50": round(float(np.percentile(lat_s, 50)), 2),
                                         "p99": round(float(np.percentile(lat_s, 99)), 2),
                                         "how": "offload_submit + offload_poll, one in flight, 2000 requests"}
    finally:
        srv.close()
    # served throughput: the same 4096 requests through the resident kernel,
    # all offered at once by the native driver's 8 submitter threads (keys
    # from a 64-key set: request i uses key i mod 64)
    srv2 = A.Server(slots=1024, max_keys=64, idle_timeout_us=2_000_000)
    try:
        ks = np.array([srv2.key_register(w.key_of(i).tobytes(), int(w.bits[i])) for i in range(64)])
        dr = np.zeros(len(reqs), dtype=A.drive_dtype())
        dr["key_slot"] = ks[np.arange(len(reqs)) % 64]
        dr["iv"] = w.ivs
        dr["inp"] = [r[2] for r in reqs]
        dr["out"] = [r[3] for r in reqs]
        dr["len"] = [r[4] for r in reqs]
        A.drive_served(srv2, dr, 8)  # warm-up
        lat, res = A.drive_served(srv2, dr, 8)
        out["served_throughput"] = {"value": round(res["bytes"] / res["elapsed_s"] / 1e9, 3), "unit": UNIT,
                                    "errors": res["errors"],
                                    "how": "the 4096 requests offered at once through offload_drive (8 native "
                                           "submitter threads, keys from a 64-key set), first arrival to last "
                                           "completion"}
    finally:
        srv2.close()
    return out


def run_e2e(A, torch, w, ctxs, args, sh, stream, dist, ws):
    """Same metric with payloads in pinned host memory: the kernel reads the
    plaintext from and writes the ciphertext to host memory (NVLink-C2C),
    so each step moves step_bytes host->device and step_bytes device->host."""
    h_in = torch.from_numpy(w.payload).pin_memory()
    h_out = torch.empty(w.arena_bytes, dtype=torch.uint8).pin_memory()
    reqs = [(ctxs[i], w.ivs[i].tobytes(), h_in.data_ptr() + int(w.offsets[i]),
             h_out.data_ptr() + int(w.offsets[i]), int(w.lengths[i])) for i in range(w.n)]
    # Over the host link the kernel waits on NVLink-C2C latency, not on the
    # shared-memory pipe, so the shape tuned for HBM-resident payloads is not
    # the best here: time a few shapes (2 launches each) and keep the fastest.
    best = None
    for v, th, tb, nb in ((1, 512, 2048, 1), (1, 512, 2048, 2), (1, 1024, 2048, 2), (1, 1024, 4096, 4)):
        p = A.BatchPlan(reqs, variant=v, threads=th, tile_blocks=tb, blocks_per_thread=nb)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p.launch(sh)
        a.record(stream)
        p.launch(sh)
        b.record(stream)
        stream.synchronize()
        ms = a.elapsed_time(b)
        if best is None or ms < best[0]:
            if best is not None:
                best[1].close()
            best = (ms, p, {"variant": v, "threads": th, "tile_blocks": tb, "blocks_per_thread": nb})
        else:
            p.close()
    plan, shape = best[1], best[2]
    nbytes = plan.nbytes
    steps = max(3, min(args.steps, 60))
    for _ in range(max(1, min(args.warmup, 3))):
        plan.launch(sh)
    stream.synchronize()
    if dist:
        dist.barrier()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        plan.launch(sh)
    b.record(stream)
    stream.synchronize()
    secs = a.elapsed_time(b) / 1e3
    secs = R.max_over_ranks(secs, dist, torch.device("cuda", torch.cuda.current_device()))
    plan.close()
    return {"value": round(R.aggregate_gbs(nbytes, steps, ws, secs), 3), "unit": UNIT, "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": nbytes, "steps": steps, "shape": shape,
            "how": "aes_batch_plan_launch on pinned host buffers (zero-copy over NVLink-C2C), the fastest of 4 "
                   "batch shapes timed on these buffers"}


if __name__ == "__main__":
    sys.exit(main())
