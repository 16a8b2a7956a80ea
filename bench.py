#!/usr/bin/env python
"""Benchmark of the batched MD5 / SHA-1 / SM3 hot path on B300.

Default workload (the configuration the headline metric is quoted on): a
plain fixed-length batch of 2^22 messages x 55 bytes (one 64-byte block
after padding), uniform random bytes, packed back to back with uint64
offsets and uint32 lengths.  One step hashes every message with each of MD5,
SHA-1 and SM3: by default one launch of the fused kernel (hash_batch_all,
96-byte records), with --separate one launch per algorithm (32-byte slots).
`value` counts input bytes once per algorithm (3 x 230.7 MB per step: the
bytes each algorithm hashed), so it is "byte-hashes per second over the
three algorithms"; the per-algorithm rates of the single-algorithm kernels
are reported beside it.  Inputs (220 MiB + 48 MiB of metadata) are larger
than the 126 MB L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W]
                    [--workload c2|c4|c3|c1] [--impl ours|reference]

Multi-GPU: one process per GPU (torchrun); each rank hashes its own disjoint
shard (the same shape, its own seed) with no collective on the data path;
only a barrier and a max-over-ranks of the timed region use torch.distributed
(weak scaling).  `--impl reference` times the CPU oracle (plain C, RFC 1321 /
FIPS 180-4 / GB/T 32905) on a bounded sample of the same workload; it runs on
rank 0 only.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2407_09333_b300 import workloads  # noqa: E402

METRIC = "hashed GB/s and Mhash/s per alg (plain vs ragged batch); serve p50/p99 latency"
ALG_NAMES = ("md5", "sha1", "sm3", None, "all")   # index 4: the fused kernel

from paper_2407_09333_b300 import shard  # noqa: E402

# Algorithmic 32-bit operations per 64-byte block, one table for the roofline
# and the multi-GPU split (shard.OPS_PER_BLOCK: 324 / 613 / 1412 for MD5 /
# SHA-1 / SM3, counted from the definitions).
OPS_PER_BLOCK = {a: int(shard.OPS_PER_BLOCK[a]) for a in range(3)}
# copy mapping of a launch shape (api.shapes()[i][3])
COPY_MAPPING = {0: "per lane", 1: "cooperative"}


def padded_blocks(lengths: np.ndarray) -> np.ndarray:
    return (lengths.astype(np.uint64) + np.uint64(72)) >> np.uint64(6)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured", "sm_max_mhz": float(d.get("sm_max_mhz", 2032.0))}
    except Exception:
        return {"hbm_gbs": 6400.0, "source": "fallback", "sm_max_mhz": 2032.0}


def alu_peak_tops(sms: int, sm_mhz: float, lanes_per_sm: int = 128) -> float:
    """32-bit integer issue peak: SMs x 4 sub-partitions x 32 lanes x clock
    (one warp instruction per sub-partition per clock, ALU and FMA pipes
    together).  lanes_per_sm=64 gives the ALU pipe alone (LOP3/IADD3/SHF/PRMT
    sustain 64.8 per clock per SM in the microbenchmark)."""
    return sms * lanes_per_sm * sm_mhz * 1e6 / 1e12


# ---------------------------------------------------------------------------
# clocks during the timed region (NVML reads only; no setting is changed)

class ClockSampler:
    """Samples the SM clock and the clock-event reasons while the timed region
    runs: NVML reads from a thread, else `nvidia-smi -lms` in the background.
    Nothing is set; settings are only read."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown",
               0x2: "applications_clocks_setting"}

    def __init__(self, device_index: int, period_s: float = 0.005):
        self.period = period_s
        self.device_index = device_index
        self.samples = []
        self.reasons = 0
        self.max_mhz = None
        self.error = None
        self.source = "nvml"
        self._stop = threading.Event()
        self._thread = None
        self._proc = None
        self._nvml = None
        try:
            import pynvml
            pynvml.nvmlInit()
            self._h = self._handle(pynvml, device_index)
            self.max_mhz = float(pynvml.nvmlDeviceGetMaxClockInfo(self._h, pynvml.NVML_CLOCK_SM))
            self._nvml = pynvml
        except Exception as e:  # fall back to nvidia-smi
            self.error = "nvml: %s" % (e,)
            self.source = "nvidia-smi"

    @staticmethod
    def _handle(nv, device_index):
        """NVML handle of the CUDA device (matched by UUID: NVML numbers all
        GPUs of the machine, CUDA only the visible ones)."""
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(device_index).uuid)
            return nv.nvmlDeviceGetHandleByUUID(uuid if uuid.startswith("GPU-") else "GPU-" + uuid)
        except Exception:
            return nv.nvmlDeviceGetHandleByIndex(device_index)

    def _reasons_now(self):
        nv = self._nvml
        fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(nv, "nvmlDeviceGetCurrentClocksThrottleReasons")
        return fn(self._h)

    def _run(self):
        nv = self._nvml
        while not self._stop.is_set():
            try:
                self.samples.append(float(nv.nvmlDeviceGetClockInfo(self._h, nv.NVML_CLOCK_SM)))
                self.reasons |= int(self._reasons_now())
            except Exception as e:
                self.error = "nvml sample: %s" % (e,)
            time.sleep(self.period)

    def __enter__(self):
        if self._nvml is not None:
            self._thread = threading.Thread(target=self._run, daemon=True)
            self._thread.start()
        else:
            import subprocess
            import tempfile
            self._tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            try:
                self._proc = subprocess.Popen(
                    ["nvidia-smi", "-i", str(self.device_index),
                     "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.active",
                     "--format=csv,noheader,nounits", "-lms", str(max(20, int(self.period * 1e3)))],
                    stdout=self._tmp, stderr=subprocess.DEVNULL)
            except OSError as e:
                self.error = "%s; nvidia-smi: %s" % (self.error, e)
        return self

    def __exit__(self, *exc):
        self._stop.set()
        if self._thread:
            self._thread.join()
        if self._proc is not None:
            self._proc.terminate()
            self._proc.wait()
            self._tmp.seek(0)
            for row in self._tmp.read().splitlines():
                parts = [x.strip() for x in row.split(",")]
                try:
                    self.samples.append(float(parts[0]))
                    self.max_mhz = float(parts[1])
                    self.reasons |= int(parts[2], 16)
                except (ValueError, IndexError):
                    pass

    def summary(self):
        reasons = [name for bit, name in self.REASONS.items() if self.reasons & bit]
        out = {"sm_mhz": float(statistics.median(self.samples)) if self.samples else None,
               "sm_max_mhz": self.max_mhz, "reasons": reasons, "samples": len(self.samples),
               "source": self.source}
        if self.error and not self.samples:
            out["error"] = self.error
        return out


# ---------------------------------------------------------------------------
# distributed plumbing (barrier + max over ranks only)

class Dist:
    def __init__(self, want_gpus: int):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch
            import torch.distributed as dist
            if torch.cuda.is_available():
                torch.cuda.set_device(self.local_rank)  # one GPU per rank from the start
            backend = "nccl" if torch.cuda.is_available() else "gloo"
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group(backend=backend)
            self.pg = dist
        self.want = want_gpus

    def barrier(self):
        if self.pg:
            if self.pg.get_backend() == "nccl":
                import torch
                self.pg.barrier(device_ids=[torch.cuda.current_device()])
            else:
                self.pg.barrier()

    def _reduce(self, value: float, op) -> float:
        import torch
        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([value], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=op)
        return float(t.item())

    def max(self, value: float) -> float:
        """Largest value over ranks (the job's time is its slowest rank's)."""
        return self._reduce(value, self.pg.ReduceOp.MAX) if self.pg else value

    def sum(self, value: float) -> float:
        """Sum over ranks (the job's bytes are every rank's shard)."""
        return self._reduce(value, self.pg.ReduceOp.SUM) if self.pg else value

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def shard_seed(base: int, rank: int) -> int:
    """Each rank hashes its own disjoint synthetic shard."""
    return base + 1000 * rank


def job_rate(dist, local_units: float, local_seconds: float) -> float:
    """Whole-job rate: every rank's units over the slowest rank's time."""
    return dist.sum(local_units) / dist.max(local_seconds)


# ---------------------------------------------------------------------------
# workloads

def make_workload(name: str, rank: int, messages: int = 0):
    if name == "paper":
        # the strings the device generates, laid out in memory (CPU reference arm)
        n = messages or (1 << 22)
        return ("paper: nine-digit decimal strings %d .. %d, MD5 + SHA-1 + SM3" % (0, n - 1),
                workloads.digits9(n), False)
    if name == "c3" and messages:
        return ("ragged mixed-algorithm batch: %d messages, log-uniform lengths in [0, 64 KiB], "
                "1%% at padding boundaries, algorithm per message" % messages,
                workloads.ragged(messages, shard_seed(2, rank)), True)
    if name == "c5":
        # the serving mix as one ragged batch (used by the CPU reference arm)
        reqs = workloads.serve_requests(messages or 64, 1.0, shard_seed(4, rank))
        lengths = np.concatenate([r.lengths for r in reqs])
        algs = np.concatenate([np.full(r.lengths.shape[0], r.alg, np.uint8) for r in reqs])
        offsets = np.zeros(lengths.shape[0], dtype=np.uint64)
        offsets[1:] = np.cumsum(lengths.astype(np.uint64))[:-1]
        packed = workloads.fixed(1, int(lengths.astype(np.int64).sum()), shard_seed(4, rank)).packed
        return ("serving mix as one batch: %d requests, 1-4096 messages each, lengths log-uniform "
                "in [16 B, 1 MiB]" % len(reqs), workloads.Batch(packed, offsets, lengths, algs), True)
    if name == "c1":
        return ("plain fixed-length batch: 4096 messages x 64 B, MD5+SHA-1+SM3 per step",
                workloads.fixed(4096, 64, shard_seed(0, rank)), False)
    if name == "c2":
        return ("plain fixed-length batch: 2^22 messages x 55 B (one block each), "
                "MD5+SHA-1+SM3 per step", workloads.fixed(1 << 22, 55, shard_seed(1, rank)), False)
    if name == "c4":
        return ("long-message batch: 65536 messages x 16 KiB, MD5+SHA-1+SM3 per step",
                workloads.fixed(65536, 16384, shard_seed(3, rank)), False)
    if name == "c3":
        return ("ragged mixed-algorithm batch: 2^20 messages, log-uniform lengths in [0, 64 KiB], "
                "1% at padding boundaries, algorithm per message", workloads.ragged(1 << 20, shard_seed(2, rank)), True)
    raise SystemExit("unknown workload %r" % name)


# ---------------------------------------------------------------------------
# CPU oracle timing (bounded samples)

def oracle_sample(batch, mixed: bool, max_msgs: int):
    n = min(batch.n, max_msgs)
    sub = workloads.Batch(batch.packed, batch.offsets[:n], batch.lengths[:n],
                          batch.algs[:n] if batch.algs is not None else None)
    return sub


def time_oracle(sub, mixed: bool, threads: int):
    import oracle
    t0 = time.perf_counter()
    if mixed:
        oracle.hash_batch(None, sub.packed, sub.offsets, sub.lengths, algs=sub.algs, threads=threads)
        nbytes, nmsgs = sub.total_bytes, sub.n
    else:
        for alg in (0, 1, 2):
            oracle.hash_batch(alg, sub.packed, sub.offsets, sub.lengths, threads=threads)
        nbytes, nmsgs = 3 * sub.total_bytes, 3 * sub.n
    return time.perf_counter() - t0, nbytes, nmsgs


def cpu_baseline(batch, mixed: bool, target_s: float = 10.0, cap_s: float = 30.0):
    import oracle
    threads = oracle.host_threads()
    sub = oracle_sample(batch, mixed, 1 << 18)
    dt, nbytes, nmsgs = time_oracle(sub, mixed, threads)
    passes, tot_t, tot_b, tot_m = 1, dt, nbytes, nmsgs
    while tot_t < target_s and tot_t + dt < cap_s:
        dt, nbytes, nmsgs = time_oracle(sub, mixed, threads)
        passes += 1
        tot_t += dt
        tot_b += nbytes
        tot_m += nmsgs
    return {"value": tot_b / tot_t / 1e9, "unit": "GB/s", "cores": threads, "kind": "oracle",
            "mhash_per_s": tot_m / tot_t / 1e6,
            "sample": "first %d messages of the workload (%s), %d pass(es), %.1f s"
                      % (sub.n, "per-message algorithm" if mixed else "each of MD5, SHA-1, SM3",
                         passes, tot_t)}


def run_reference(args, dist):
    if dist.rank != 0:
        return
    desc, batch, mixed = make_workload(args.workload, 0, args.messages)
    import oracle
    threads = oracle.host_threads()
    sub = oracle_sample(batch, mixed, 1 << 18 if args.workload != "c4" else 1 << 10)
    # keep the whole run within about two minutes: shrink the per-step sample
    # if one step of it would make warm-up plus timed steps take longer
    dt, _, _ = time_oracle(sub, mixed, threads)
    budget_s = 120.0
    runs = args.warmup + args.steps
    if dt * runs > budget_s and sub.n > 64:
        sub = oracle_sample(batch, mixed, max(64, int(sub.n * budget_s / (dt * runs))))
    for _ in range(args.warmup - 1):
        time_oracle(sub, mixed, threads)
    tot_t = tot_b = tot_m = 0
    for _ in range(args.steps):
        dt, nb, nm = time_oracle(sub, mixed, threads)
        tot_t += dt
        tot_b += nb
        tot_m += nm
    value = tot_b / tot_t / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s",
        "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot_t / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": desc, "sample_messages": sub.n},
        "mhash_per_s": tot_m / tot_t / 1e6,
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": threads, "kind": "oracle",
                         "sample": "first %d messages of the workload per step" % sub.n},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the CUDA path

def traffic_for(kernel_key: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel
    sources have not changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(path))
    except Exception:
        return None
    ent = d.get(kernel_key)
    if not ent or ent.get("source_hash") != kernel_source_hash():
        return None
    return ent.get("dram_bytes_per_launch")


# Host-only sources (no device code): changing them does not change a kernel.
HOST_ONLY_SOURCES = ("hb_capi.cu",)


def kernel_source_hash() -> str:
    """Hash of the sources the kernels are compiled from."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2407_09333_b300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".h")) and f not in HOST_ONLY_SOURCES:
            h.update(f.encode())
            h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def run_ours(args, dist):
    """The default run: the headline workload, then (one GPU, default
    workload) short measurements of the long-message and ragged workloads as
    extra keys, each with its own roofline, so that one run reports all three
    measured configurations."""
    import copy
    import torch
    line = measure(args, dist)
    if args.workload == "c2" and dist.world == 1 and not args.no_extras and args.shape is None:
        line["extra_workloads"] = {}
        for name, steps in (("c4", 50), ("c3", 20)):
            torch.cuda.empty_cache()
            sub = copy.copy(args)
            sub.workload, sub.steps, sub.warmup = name, steps, 3
            sub.no_e2e = sub.no_cpu_baseline = True
            sub.messages = 0
            x = measure(sub, dist)
            keep = ("value", "unit", "ms_per_step", "mhash_per_s", "per_alg", "roofline", "clocks",
                    "config", "plain_equal_bytes_gbs", "ragged_vs_plain_equal_bytes", "cost_model",
                    "tuned_shapes", "steps", "warmup", "gpu_launches")
            line["extra_workloads"][name] = {k: x[k] for k in keep if k in x}
    if dist.rank == 0:
        print(json.dumps(line), flush=True)


def clock_window(step, device_index, seconds=1.5):
    """SM clock and throttle reasons while `step` runs back to back for at
    least `seconds` (the counted steps can be too short for the sampler):
    the same launches, outside the timed region."""
    import torch
    with ClockSampler(device_index, period_s=0.01) as clocks:
        t0 = time.perf_counter()
        n = 0
        while time.perf_counter() - t0 < seconds:
            for _ in range(8):
                step()
            n += 8
            torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    out = clocks.summary()
    out.update({"window_s": dt, "window_steps": n,
                "window": "the timed step repeated back to back right after the timed region"})
    return out


def measure(args, dist):
    import torch
    from paper_2407_09333_b300 import api, build

    if torch.cuda.is_available():
        torch.cuda.set_device(dist.local_rank)
    build.build()
    api.lib()
    if args.scaling == "strong":
        # one batch for the whole job; each rank hashes its range, split by
        # estimated work (padded blocks x ops per block)
        from paper_2407_09333_b300 import shard
        desc, full, mixed = make_workload(args.workload, 0, args.messages)
        lo, hi = shard.rank_range(full.lengths, full.algs, alg=None if mixed else 2,
                                  rank=dist.rank, world=dist.world)
        batch = workloads.Batch(full.packed, full.offsets[lo:hi], full.lengths[lo:hi],
                                full.algs[lo:hi] if full.algs is not None else None)
        desc += "; strong scaling: rank %d hashes messages [%d, %d) of %d" % (dist.rank, lo, hi, full.n)
    else:
        desc, batch, mixed = make_workload(args.workload, dist.rank, args.messages)
    packed, off, ln, algs = api.to_device(batch)
    n = batch.n
    out = torch.empty((n, 32), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    nblocks = padded_blocks(batch.lengths)
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sms = props.multi_processor_count

    from paper_2407_09333_b300 import autotune
    if args.relay_blocks is not None:
        api.tune_relay(args.relay_blocks)
    tuned = {}
    mean_len = batch.total_bytes / max(n, 1)
    fused = not mixed and not args.separate
    rec = torch.empty((n, 96), dtype=torch.uint8, device="cuda") if fused else None
    items = fused and args.as_items
    if items:
        # the three-algorithm step as 3n (message, algorithm) items through
        # the ragged kernel: item 3i + a is message i under algorithm a, and
        # its 32-byte slot is slot a of record i
        off3 = off.repeat_interleave(3).contiguous()
        ln3 = ln.repeat_interleave(3).contiguous()
        algs3 = torch.tensor([0, 1, 2], dtype=torch.uint8, device="cuda").repeat(n).contiguous()
        out3 = rec.view(3 * n, 32)
    for a in ([None] if mixed else [0, 1, 2] + ([api.ALL] if fused else [])):
        if items and a == api.ALL:
            if args.shape is not None:
                api.tune_set(api.TUNE_MIXED, args.shape)
                if args.buckets:
                    api.tune_buckets(*[int(x) for x in args.buckets.split(",")])
                tuned["all_as_items"] = {"shape": args.shape, "fixed": True}
                continue
            r = autotune.tune(None, packed, off3, ln3, out3, algs=algs3, mean_len=mean_len)
            tuned["all_as_items"] = {"warps": r["warps"], "stages": r["stages"],
                                     "blocks_per_stage": r.get("blocks_per_stage", 1),
                                     "cooperative": r.get("cooperative", False),
                                     "cached": r["cached"], "warps_per_sm": r.get("warps_per_sm")}
            continue
        if args.shape is not None:
            # fixed launch configuration (reproducible profiler captures)
            api.tune_set(api.TUNE_MIXED if a is None else a, args.shape)
            if a is None and args.buckets:
                api.tune_buckets(*[int(x) for x in args.buckets.split(",")])
            w, st, kb, co = api.shapes()[args.shape]
            tuned["mixed" if a is None else ALG_NAMES[a]] = {"warps": w, "stages": st,
                                                              "blocks_per_stage": kb,
                                                              "copies": COPY_MAPPING[co], "fixed": True}
            continue
        r = autotune.tune(a, packed, off, ln, rec if a == api.ALL else out, algs=algs,
                          mean_len=mean_len)
        tuned["mixed" if a is None else ALG_NAMES[a]] = {"warps": r["warps"], "stages": r["stages"],
                                                          "blocks_per_stage": r.get("blocks_per_stage", 1),
                                                          "copies": COPY_MAPPING[r.get("copy_mapping",
                                                                                       int(r.get("cooperative", 0)))],
                                                          "cached": r["cached"]}
        if "buckets" in r:
            tuned["mixed"]["buckets_per_octave"] = 1 << r["buckets"][0]
            tuned["mixed"]["algorithm_major"] = int(r["buckets"][1])
        if "warps_per_sm" in r:
            tuned["mixed"]["warps_per_sm"] = r["warps_per_sm"] or "occupancy"
        if a is None and "ms" in r:
            # every (shape, warps per SM) the tuner timed, and the bucketings
            tuned["mixed"]["timings_ms"] = r["ms"]
            tuned["mixed"]["bucket_timings_ms"] = r.get("bucket_ms")

    if mixed:
        # the whole ragged sequence (bucketing + persistent kernel) captured
        # once as a CUDA graph and replayed each step
        plan = api.Plan(n)
        plan.capture(algs, packed, off, ln, out)
        launches = [(None, lambda: plan.replay(n))]
        bytes_per_step = batch.total_bytes
        msgs_per_step = n
    elif items:
        launches = [(api.ALL, lambda: api.hash_batch_mixed(algs3, packed, off3, ln3, out=out3))]
        bytes_per_step = 3 * batch.total_bytes
        msgs_per_step = 3 * n
    elif fused:
        # every message with all three algorithms in one pass (hash_batch_all)
        launches = [(api.ALL, lambda: api.hash_batch_all(packed, off, ln, out=rec))]
        bytes_per_step = 3 * batch.total_bytes
        msgs_per_step = 3 * n
    else:
        launches = [(a, (lambda a=a: api.hash_batch(a, packed, off, ln, out=out))) for a in (0, 1, 2)]
        bytes_per_step = 3 * batch.total_bytes
        msgs_per_step = 3 * n

    for _ in range(args.warmup):
        for _, fn in launches:
            fn()
    torch.cuda.synchronize()

    nl = len(launches)
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(nl)] for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clocks:
        t_start.record(stream)
        for k in range(args.steps):
            for j, (_, fn) in enumerate(launches):
                ev[k][j][0].record(stream)
                fn()
                ev[k][j][1].record(stream)
        t_end.record(stream)
        torch.cuda.synchronize()
    dist.barrier()
    ms_local = t_start.elapsed_time(t_end)
    ms = dist.max(ms_local)
    job_bytes = dist.sum(float(bytes_per_step) * args.steps)
    job_msgs = dist.sum(float(msgs_per_step) * args.steps)
    status = api.device_status()
    if status:
        raise SystemExit("device status reported error bits %#x" % status)

    per_launch_ms = [statistics.median([ev[k][j][0].elapsed_time(ev[k][j][1]) for k in range(args.steps)])
                     for j in range(nl)]
    value = job_bytes / (ms * 1e-3) / 1e9
    peaks = load_peaks()
    # clocks: the sampler also ran during the counted steps, which can be too
    # short for it; a window of the same steps repeated for a second gives
    # the clock record (time x clock lets runs at different clocks compare)
    timed_clk = clocks.summary()

    def one_step():
        for _, fn in launches:
            fn()
    clk = clock_window(one_step, torch.cuda.current_device())
    clk["during_timed_steps"] = {"samples": timed_clk["samples"], "sm_mhz": timed_clk["sm_mhz"],
                                 "reasons": timed_clk["reasons"]}
    if clk["sm_mhz"]:
        clk["ms_per_step_x_sm_mhz"] = ms / args.steps * clk["sm_mhz"]
    sm_mhz = clk["sm_mhz"] or peaks["sm_max_mhz"]

    def launch_figures(a, t):
        """GB/s, Mhash/s and roofline fractions of one launch of `a`."""
        copies = 3 if a == api.ALL else 1
        if a == api.ALL:
            ops = float(nblocks.sum()) * sum(OPS_PER_BLOCK.values())
        elif a is not None:
            ops = float(nblocks.sum()) * OPS_PER_BLOCK[a]
        else:
            ops = float(sum(float(nblocks[batch.algs == x].sum()) * OPS_PER_BLOCK[x] for x in (0, 1, 2)))
        hbm = batch.total_bytes + 12 * n + (1 * n if mixed else 0) + 32 * copies * n
        return {
            "GB/s": copies * batch.total_bytes / t / 1e9, "Mhash/s": copies * n / t / 1e6, "ms": t * 1e3,
            "alu_Tops": ops / t / 1e12,
            "alu_frac_at_clock": ops / t / 1e12 / alu_peak_tops(sms, sm_mhz),
            "hbm_frac": hbm / t / 1e9 / peaks["hbm_gbs"],
        }, ops, hbm

    per_alg = {}
    hbm_of = {}
    for j, (a, _) in enumerate(launches):
        name = ALG_NAMES[a] if a is not None else "mixed"
        per_alg[name], _, hbm_of[name] = launch_figures(a, per_launch_ms[j] * 1e-3)
    per_alg_separate = None
    if fused:
        # the three single-algorithm kernels, for the per-algorithm figures
        # (timed like a step of the --separate mode: back to back on the
        # stream, an event pair around each launch)
        per_alg_separate = {}
        sep = [(a, (lambda a=a: api.hash_batch(a, packed, off, ln, out=out))) for a in (0, 1, 2)]
        for _, fn in sep:
            fn()
        torch.cuda.synchronize()
        reps = 20
        sev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in sep] for _ in range(reps)]
        for k in range(reps):
            for j, (_, fn) in enumerate(sep):
                sev[k][j][0].record(stream)
                fn()
                sev[k][j][1].record(stream)
        torch.cuda.synchronize()
        for j, (a, _) in enumerate(sep):
            t = statistics.median([sev[k][j][0].elapsed_time(sev[k][j][1]) for k in range(reps)])
            per_alg_separate[ALG_NAMES[a]] = launch_figures(a, t * 1e-3)[0]
    dom = max(range(nl), key=lambda j: per_launch_ms[j])
    dom_alg = launches[dom][0]
    dom_name = ALG_NAMES[dom_alg] if dom_alg is not None else "mixed"
    t_dom = per_launch_ms[dom] * 1e-3
    dom_ops = per_alg[dom_name]["alu_Tops"] * 1e12 * t_dom
    hbm_bytes_per_launch = hbm_of[dom_name]
    peak_alu = alu_peak_tops(sms, peaks["sm_max_mhz"])
    relay = dom_name == "all" and not items and api.all_uses_relay(n)
    kernel_key = "%s:%s" % (args.workload, "items" if items else dom_name + ("_relay" if relay else ""))
    roofline = {
        "bound": "alu", "kernel": "hb_%s_kernel<%s>" % ("mixed" if mixed or items else
                                                      "relay" if relay else "plain",
                                                      "3n items" if items else dom_name),
        "achieved": dom_ops / t_dom / 1e12, "peak": peak_alu, "unit": "Tops/s",
        "frac": dom_ops / t_dom / 1e12 / peak_alu,
        "peak_source": "derived: %d SMs x 4 sub-partitions x 32 lanes x %.0f MHz max SM clock "
                       "(INT32 issue peak, ALU and FMA pipes together)" % (sms, peaks["sm_max_mhz"]),
        "frac_at_measured_clock": dom_ops / t_dom / 1e12 / alu_peak_tops(sms, sm_mhz),
        "frac_of_alu_pipe": dom_ops / t_dom / 1e12 / alu_peak_tops(sms, peaks["sm_max_mhz"], 64),
        "algorithmic_ops_per_launch": dom_ops,
        "hbm_achieved_gbs": hbm_bytes_per_launch / t_dom / 1e9,
        "hbm_peak_gbs": peaks["hbm_gbs"], "hbm_peak_source": peaks["source"],
        "hbm_frac": hbm_bytes_per_launch / t_dom / 1e9 / peaks["hbm_gbs"],
        "traffic": traffic_for(kernel_key),
    }

    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": dist.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": args.scaling, "vs_baseline": None, "dtype": "u32",
        "data": "synthetic: uniform random bytes (numpy PCG64), shard seed per rank",
        "config": {"workload": desc, "messages_per_gpu": n, "bytes_per_gpu": batch.total_bytes,
                   "value_counts": ("message bytes hashed, once per message" if mixed else
                                    "byte-hashes over three algorithms: each message's bytes once "
                                    "per algorithm (3 x %d bytes per step%s); per-algorithm rates "
                                    "of the single-algorithm kernels are in per_alg_separate_kernels"
                                    % (batch.total_bytes, ", one fused launch reading them once"
                                       if fused else ", three launches")),
                   "l2": "no flush: inputs larger than the 126 MB L2",
                   "parallelism": "dp%d: disjoint message shards, no collective on the data path" % dist.world},
        "mhash_per_s": job_msgs / (ms * 1e-3) / 1e6,
        "per_alg": per_alg,
        "per_alg_separate_kernels": per_alg_separate,
        "tuned_shapes": tuned,
        "roofline": roofline,
        # plain: one fused kernel (or one per algorithm with --separate);
        # ragged graph: count-setter, group histogram, scan, scatter and the
        # persistent hashing kernel
        "gpu_launches": args.steps * nl * (5 if mixed else 4 if items else 1),
        "clocks": clk,
    }

    if mixed:
        # the ragged launch against the plain kernels at equal bytes
        pg, pl = plain_equal_bytes_gbs(api, torch, batch.lengths, batch.algs, packed)
        line["plain_equal_bytes_gbs"] = pg
        line["plain_mean_length"] = pl
        line["ragged_vs_plain_equal_bytes"] = per_alg["mixed"]["GB/s"] / pg
        line["cost_model"] = cost_model_report(api, torch, batch, packed, per_alg["mixed"]["ms"])
    if not args.no_e2e:
        line["e2e"] = e2e_measure(args, batch, mixed, api, torch, dist)
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(batch, mixed)
    return line


def e2e_measure(args, batch, mixed, api, torch, dist):
    """Same metric through hash_batch_host with pinned host buffers: the
    host->device copy of the step's inputs and the device->host copy of its
    digests are inside the timed region.  Whole job: every rank's bytes over
    the slowest rank's time."""
    n = batch.n
    packed_h = torch.from_numpy(np.ascontiguousarray(batch.packed)).pin_memory()
    off_h = torch.from_numpy(batch.offsets.view(np.int64)).pin_memory()
    len_h = torch.from_numpy(batch.lengths.view(np.int32)).pin_memory()
    algs_h = torch.from_numpy(batch.algs).pin_memory() if mixed else None
    fused = not mixed and not args.separate
    calls = [None] if mixed else [api.ALL] if fused else [0, 1, 2]
    # digests come back packed (16 / 20 / 32 bytes, 68 for all three) unless
    # the batch is mixed (variable sizes) or --e2e-slots asks for the slots
    pack = not mixed and not args.e2e_slots
    outs = {a: torch.empty((n, api.host_digest_bytes(a, pack)), dtype=torch.uint8).pin_memory()
            for a in calls}

    def step():
        for a in calls:
            api.hash_batch_host(a, packed_h, off_h, len_h, outs[a], algs=algs_h, packed_digests=pack)

    if args.host_limit_mib:
        api.set_host_memory_limit(args.host_limit_mib << 20)
        try:
            step()
        except api.HashBatchError as e:
            api.set_host_memory_limit(0)
            return {"value": None, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                    "device_memory_limit_bytes": args.host_limit_mib << 20,
                    "error": "%s (windows need messages in memory order)" % e}

    steps = max(1, min(args.steps, args.e2e_steps))
    for _ in range(max(1, min(args.warmup, 3))):
        step()
    torch.cuda.synchronize()
    dist.barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    dist.barrier()
    per_call_in = batch.packed.nbytes + 12 * n + (n if mixed else 0)
    if args.host_limit_mib:
        api.set_host_memory_limit(0)
    hashed = (3 if fused else len(calls)) * batch.total_bytes
    return {"value": job_rate(dist, hashed * steps, dt) / 1e9, "unit": "GB/s",
            "device_memory_limit_bytes": args.host_limit_mib << 20,
            "h2d_bytes_per_step": len(calls) * per_call_in,
            "d2h_bytes_per_step": sum(o.numel() for o in outs.values()), "steps": steps,
            "api": "hash_batch_host%s (pinned host buffers)" % ("_packed" if pack else ""),
            "digests": ("packed: digest bytes only" if pack else
                        "32-byte slots" + (" (96-byte records)" if fused else ""))}


def plain_equal_bytes_gbs(api, torch, lengths, algs, pool, reps=3, max_msgs=1 << 18):
    """Rate of the plain (fixed-length) kernels at equal bytes: per algorithm
    a batch of messages of the set's mean length, timed with its best launch
    shape; the set's bytes of each algorithm at that algorithm's rate.  The
    batch holds the algorithm's bytes of the set or max_msgs messages,
    whichever is fewer (enough to fill the GPU: the rate no longer depends on
    the batch size), read from `pool` (device random bytes) at spread
    16-byte aligned offsets.  Returns (GB/s, mean length)."""
    L = max(1, int(round(float(lengths.astype(np.float64).mean()))))
    span = max(1, (pool.numel() - L) // 16)
    t_total = 0.0
    b_total = 0
    for a in (0, 1, 2):
        nbytes = int(lengths[algs == a].astype(np.int64).sum())
        if nbytes == 0:
            continue
        n = max(1, min(nbytes // L, max_msgs))
        i = torch.arange(n, dtype=torch.int64, device=pool.device)
        o = ((i * 2654435761) % span) * 16
        l = torch.full((n,), L, dtype=torch.int32, device=pool.device)
        out = torch.empty((n, 32), dtype=torch.uint8, device=pool.device)
        best = float("inf")
        for sh in range(len(api.shapes())):
            fn = lambda: api.hash_batch(a, pool, o, l, out=out, shape=sh)
            fn()
            torch.cuda.synchronize()
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(); fn(); e1.record(); e1.synchronize()
                best = min(best, e0.elapsed_time(e1))
        rate = n * L / (best * 1e-3)               # bytes per second
        t_total += nbytes / rate
        b_total += nbytes
        del o, l, out
    return b_total / t_total / 1e9, L


def _timed_s(torch, fn, reps=3):
    """Best of `reps` CUDA-event timings of fn() after one untimed call."""
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(); fn(); e1.record(); e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best * 1e-3


def fit_launch_model(api, torch, pool, shape=-1, lengths=(1024, 16384), launch_bytes=1 << 30,
                     reps=3):
    """Eq. 2's linear form (per-algorithm rate per op, per-message term,
    launch cost T0) for the persistent ragged kernel in launch shape `shape`,
    fitted on launches that its throughput bounds: per algorithm, messages
    of one fixed length (every chain equally long, so no chain outlasts the
    rest) read from `pool` at 16-byte aligned offsets, at two lengths (which
    separates the per-message term) and two batch sizes (which separates
    T0) -- twelve launches."""
    from paper_2407_09333_b300 import costmodel
    samples = []
    span = max(1, (pool.numel() - max(lengths)) // 16)
    for a in (0, 1, 2):
        for L in lengths:
            n_full = max(1024, launch_bytes // L)
            for n in (n_full, n_full // 2):
                i = torch.arange(n, dtype=torch.int64, device=pool.device)
                o = ((i * 2654435761) % span) * 16
                l = torch.full((n,), L, dtype=torch.int32, device=pool.device)
                g = torch.full((n,), a, dtype=torch.uint8, device=pool.device)
                out = torch.empty((n, 32), dtype=torch.uint8, device=pool.device)
                t = _timed_s(torch, lambda: api.hash_batch_mixed(g, pool, o, l, out=out, shape=shape),
                             reps)
                samples.append((costmodel.work_by_alg(np.full(n, L), alg=a),
                                costmodel.msgs_by_alg(n, alg=a), t))
                del i, o, l, g, out
    return costmodel.fit(samples)


def cost_model_report(api, torch, batch, pool, measured_ms):
    """The ragged kernel's cost model (fit_launch_model, in the launch shape
    the batch was hashed with) predicting the measured ragged launch from its
    lengths and algorithms alone.  The batch also has a tail the model does
    not describe: its longest messages are serial chains that start first and
    end last, on a GPU that the rest of the work has left by then."""
    m = fit_launch_model(api, torch, pool)
    pred = m.predict_batch(batch.lengths, algs=batch.algs) * 1e3
    return {"form": "T = sum over algorithms of (rate x padded blocks x ops per block + per-message "
                    "x messages) + T0",
            "fitted_on": "12 launches of the ragged kernel (tuned shape): each algorithm, messages of "
                         "1 KiB and of 16 KiB, 1 GiB and 0.5 GiB per launch",
            "rate_ps_per_op": [r * 1e12 for r in m.rate],
            "per_message_ns": [x * 1e9 for x in m.per_msg], "overhead_us": m.overhead * 1e6,
            "r2": m.r2, "predicted_ms": pred, "measured_ms": measured_ms,
            "measured_over_predicted": measured_ms / pred}


def run_serve(args, dist):
    """Serving sweep: Poisson request streams at fractions of the ragged
    path's measured throughput, served under a device-memory budget."""
    # one hardware queue per serving slot, so a long batch does not hold up
    # the batches behind it (must be set before CUDA starts)
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    import torch
    from paper_2407_09333_b300 import api, build, serve

    if torch.cuda.is_available():
        torch.cuda.set_device(dist.local_rank)
    build.build()
    # reference throughput: the ragged path on the 2^20-message ragged batch
    rb = workloads.ragged(1 << 20, shard_seed(2, dist.rank))
    rp, ro, rl, ra = api.to_device(rb)
    rout = torch.empty((rb.n, 32), dtype=torch.uint8, device="cuda")
    for _ in range(3):
        api.hash_batch_mixed(ra, rp, ro, rl, out=rout)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(5):
        api.hash_batch_mixed(ra, rp, ro, rl, out=rout)
    e1.record(); e1.synchronize()
    ref_gbs = 5 * rb.total_bytes / (e0.elapsed_time(e1) * 1e-3) / 1e9
    del rp, ro, rl, ra, rout, rb
    torch.cuda.empty_cache()

    pool_bytes = args.pool_mib << 20
    pool_host = workloads.fixed(1, pool_bytes, shard_seed(4, dist.rank)).packed
    pool = torch.from_numpy(np.ascontiguousarray(pool_host)).cuda()
    in_place = not args.staged

    def make_server(place):
        return serve.Server(pool, budget=args.budget_gib << 30, rounds=args.rounds,
                            segment_bytes=(3 * args.segment_kib << 10, 2 * args.segment_kib << 10,
                                           args.segment_kib << 10), shape=args.serve_shape,
                            warps_per_sm=args.serve_warps, in_place=place)

    def serve_point(srv, load, seed, adm=None, count=None):
        rate = load * ref_gbs * 1e9 / mean_req
        reqs = serve.make_requests(count or args.requests, rate, seed, pool_bytes, align=args.align)
        r0, s0 = srv.rounds_launched, srv.segments
        srv.run(reqs, admission=adm)
        st = serve.latency_stats(reqs)
        st.update({"offered_load": load, "offered_gbs": rate * mean_req / 1e9,
                   "requests": len(reqs), "rounds": srv.rounds_launched - r0,
                   "segments": srv.segments - s0})
        if adm is not None:
            st["prediction"] = serve.prediction_stats(reqs)
        return st, reqs

    probe = serve.make_requests(args.requests, 1.0, shard_seed(4, dist.rank), pool_bytes)
    mean_req = float(np.mean([r.nbytes for r in probe]))
    all_lengths = np.concatenate([r.lengths for r in probe])
    all_algs = np.concatenate([np.full(r.lengths.shape[0], r.alg, np.uint8) for r in probe])
    points = []
    srv = make_server(in_place)
    # Eq. 2's linear form for the served work: throughput and per-message
    # terms from ragged launches of the rounds' pieces, then the serial-chain
    # term and the fixed latency calibrated on a shorter run at half load;
    # every load point then predicts each request's completion at admission
    from paper_2407_09333_b300 import costmodel
    model, cal, drain, shed_point = None, [], 1.0, None
    if not args.no_admission:
        model = fit_launch_model(api, torch, pool, shape=args.serve_shape)
        _, cal = serve_point(srv, 0.5, shard_seed(4, dist.rank) + 991, serve.Admission(model),
                             count=min(args.requests, 4000))
        model = costmodel.fit_chain(model, [(r.alg, int(r.lengths.max()), r.done - r.arrival)
                                            for r in cal if r.done >= 0])
        # the served path's rate against the model's: a burst of requests
        burst = serve.make_requests(min(args.requests, 3000), 1e9, shard_seed(4, dist.rank) + 993,
                                    pool_bytes, align=args.align)
        for r in burst:
            r.arrival = 0.0
        srv.run(burst)
        drain = serve.calibrate_drain(model, burst)
    cap_s = args.cap_ms * 1e-3 if args.cap_ms > 0 else None
    adm = ((lambda **kw: serve.Admission(model, drain=drain, cap_s=cap_s, **kw)) if model
           else (lambda **kw: None))
    # the serving loop polls the device from the host; a slow clock sampler
    # (nvidia-smi takes driver locks on every poll) keeps out of its way
    with ClockSampler(torch.cuda.current_device(), period_s=0.2) as clocks:
        for k, load in enumerate(args.loads):
            points.append(serve_point(srv, load, shard_seed(4, dist.rank) + 17 * k, adm())[0])
        if model is not None:
            # admission control at the top load: a request whose predicted
            # completion lies more than --slo-ms after its arrival is shed there
            shed_point = serve_point(srv, max(args.loads),
                                     shard_seed(4, dist.rank) + 17 * len(args.loads),
                                     adm(slo_s=args.slo_ms * 1e-3))[0]
            shed_point["slo_ms"] = args.slo_ms
            shed_point["cap_ms"] = args.cap_ms
            shed_point["shed_fraction"] = shed_point.get("rejected", 0) / max(shed_point["requests"], 1)
    budget_used = {"ring_and_rounds": serve.device_bytes(srv.book.capacity, srv.book.req_capacity,
                                                         len(srv.slots), srv.max_msgs),
                   "staging": 0 if srv.in_place else srv.staging_per_round * len(srv.slots)}
    srv.close()
    del srv
    # the other mode at the highest offered load, for comparison
    other_point = None
    if not args.no_other_mode:
        other = make_server(not in_place)
        other_point = serve_point(other, max(args.loads),
                                  shard_seed(4, dist.rank) + 17 * len(args.loads))[0]
        other.close()
        del other
    torch.cuda.empty_cache()
    host_ingress = None
    if args.host_requests > 0:
        # host ingress: the clients' bytes in pinned host memory; each round's
        # copy step brings its segments over the bus, so the device holds
        # segments only.  Loads are fractions of the measured host-to-device
        # copy rate, which bounds this mode.
        host_pool = torch.from_numpy(np.ascontiguousarray(pool_host)).pin_memory()
        probe_dev = torch.empty(1 << 30, dtype=torch.uint8, device="cuda")
        bus_s = _timed_s(torch, lambda: probe_dev.copy_(host_pool[:1 << 30], non_blocking=True))
        bus_gbs = (1 << 30) / bus_s / 1e9
        del probe_dev
        hsrv = serve.Server(host_pool, budget=args.budget_gib << 30, rounds=args.rounds,
                            segment_bytes=(3 * args.segment_kib << 10, 2 * args.segment_kib << 10,
                                           args.segment_kib << 10), shape=args.serve_shape,
                            warps_per_sm=args.serve_warps, in_place=False)
        hpoints = []
        for k, load in enumerate(args.host_loads):
            rate = load * bus_gbs * 1e9 / mean_req
            reqs = serve.make_requests(args.host_requests, rate, shard_seed(4, dist.rank) + 331 * (k + 1),
                                       pool_bytes, align=args.align)
            hsrv.run(reqs)
            st = serve.latency_stats(reqs)
            st.update({"offered_load_of_bus": load, "offered_gbs": rate * mean_req / 1e9,
                       "requests": len(reqs)})
            hpoints.append(st)
        hsrv.close()
        del hsrv, host_pool
        torch.cuda.empty_cache()
        host_ingress = {"bus_h2d_gbs": bus_gbs, "points": hpoints,
                        "mode": "pinned host pool, segments copied over the bus by each round "
                                "(staging copy), %d GiB device budget" % args.budget_gib}
    plain_gbs, plain_L = plain_equal_bytes_gbs(api, torch, all_lengths, all_algs, pool)
    top = max(points, key=lambda p: p["offered_load"])
    # sustained rate at the highest offered load: bytes of every request over
    # the whole span from the first arrival to the last completion (every
    # rank's servers); the 10th-90th percentile window is reported beside it
    job_gbs = dist.sum(top["gbs"])
    line = {
        "metric": METRIC, "value": job_gbs, "unit": "GB/s", "n_gpus": dist.world,
        "steps": len(points), "warmup": 3, "ms_per_step": None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic: Poisson arrivals; per request 1-4096 messages (log-uniform count), "
                "lengths log-uniform in [16 B, 1 MiB], random algorithm; bytes from a %d MiB "
                "random pool (numpy PCG64)" % args.pool_mib,
        "config": {"workload": "serving: continuous batching under a %d GiB device budget, "
                               "%d streaming rounds (%s), %d KiB SM3 segments, %d requests per load point"
                               % (args.budget_gib, args.rounds,
                                  "in place" if in_place else "staging copy",
                                  args.segment_kib, args.requests),
                   "reference_ragged_gbs": ref_gbs, "mean_request_bytes": mean_req,
                   "parallelism": "dp%d: independent servers, no collective" % dist.world},
        "serve": points,
        "served_vs_plain_equal_bytes": top["gbs"] / plain_gbs,
        "served_vs_plain_definition": "whole span: all bytes of the top load point from its first "
                                      "arrival to its last completion, over the plain kernels' rate "
                                      "at equal bytes",
        "steady_vs_plain_equal_bytes": top["steady_gbs"] / plain_gbs,
        "cost_model": None if model is None else {
            "rate_ps_per_op": [r * 1e12 for r in model.rate],
            "per_message_ns": [x * 1e9 for x in model.per_msg],
            "overhead_us": model.overhead * 1e6, "r2": model.r2,
            "chain_mops_per_s": [c / 1e6 for c in model.chain],
            "latency_t0_ms": model.latency_t0 * 1e3, "served_over_model_rate": drain,
            "fitted_on": "12 fixed-length launches of the ragged kernel in the rounds' shape "
                         "(throughput terms), a %d-request run at half load (chain terms) and a "
                         "burst of %d requests (served rate)" % (len(cal), min(args.requests, 3000))},
        "admission_control": shed_point,
        "host_ingress": host_ingress,
        "device_budget_bytes": budget_used,
        "other_mode": None if other_point is None else dict(
            other_point, mode="staging copy" if in_place else "in place",
            steady_vs_plain_equal_bytes=other_point["steady_gbs"] / plain_gbs),
        "plain_equal_bytes_gbs": plain_gbs, "plain_mean_length": plain_L,
        "p50_ms_at_top_load": top["p50_ms"], "p99_ms_at_top_load": top["p99_ms"],
        "clocks": clocks.summary(),
    }
    if dist.rank == 0:
        print(json.dumps(line), flush=True)


def run_paper(args, dist):
    """The paper's workload (Sec. V-A.2) generated on the device: every
    9-character decimal string "000000000" .. "999999999" hashed with each of
    MD5, SHA-1 and SM3 per step, the 10^9 strings split evenly across ranks."""
    import torch
    from paper_2407_09333_b300 import api, build

    if torch.cuda.is_available():
        torch.cuda.set_device(dist.local_rank)
    build.build()
    # --messages hashes the first strings only (a small case for profiling)
    total = min(args.messages, api.DIGITS_COUNT) if args.messages else api.DIGITS_COUNT
    per = (total + dist.world - 1) // dist.world
    first = dist.rank * per
    count = max(0, min(per, total - first))
    out = torch.empty((max(count, 1), 32), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    launches = [(a, (lambda a=a: api.hash_digits(a, first, count, out=out))) for a in (0, 1, 2)]
    for _ in range(args.warmup):
        for _, fn in launches:
            fn()
    torch.cuda.synchronize()
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in launches] for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clocks:
        t0.record(stream)
        for k in range(args.steps):
            for j, (_, fn) in enumerate(launches):
                ev[k][j][0].record(stream)
                fn()
                ev[k][j][1].record(stream)
        t1.record(stream)
        torch.cuda.synchronize()
    dist.barrier()
    ms = dist.max(t0.elapsed_time(t1))
    job_msgs = dist.sum(float(3 * count * args.steps))
    peaks = load_peaks()
    clk = clocks.summary()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    peak = alu_peak_tops(sms, peaks["sm_max_mhz"])
    per_alg = {}
    for j, (a, _) in enumerate(launches):
        t = statistics.median([ev[k][j][0].elapsed_time(ev[k][j][1]) for k in range(args.steps)]) * 1e-3
        ops = float(count) * OPS_PER_BLOCK[a]
        per_alg[ALG_NAMES[a]] = {"Mhash/s": count / t / 1e6, "GB/s": 9 * count / t / 1e9, "ms": t * 1e3,
                                 "s_for_1e9": t * api.DIGITS_COUNT / max(count, 1), "alu_Tops": ops / t / 1e12,
                                 "alu_frac": ops / t / 1e12 / peak}
    dom = max(per_alg, key=lambda k: per_alg[k]["ms"])
    line = {
        "metric": METRIC, "value": job_msgs * 9 / (ms * 1e-3) / 1e9, "unit": "GB/s",
        "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "u32",
        "data": "generated on the device: the 10^9 nine-character decimal strings (no input bytes)",
        "config": {"workload": ("paper: all 10^9 nine-digit decimal strings" if total == api.DIGITS_COUNT
                                else "paper: the first %d nine-digit decimal strings" % total)
                               + ", MD5 + SHA-1 + SM3 per step",
                   "messages_per_gpu": count, "l2": "no inputs; 32 GB of digest slots per launch"},
        "mhash_per_s": job_msgs / (ms * 1e-3) / 1e6,
        "per_alg": per_alg,
        "roofline": {"bound": "alu", "kernel": "hb_digits_kernel<%s>" % dom,
                     "achieved": per_alg[dom]["alu_Tops"], "peak": peak, "unit": "Tops/s",
                     "frac": per_alg[dom]["alu_frac"],
                     "peak_source": "derived: %d SMs x 4 sub-partitions x 32 lanes x %.0f MHz max SM clock"
                                    % (sms, peaks["sm_max_mhz"]),
                     "traffic": None},
        "e2e": None, "e2e_note": "no input bytes: the strings are generated on the device",
        "gpu_launches": 3 * args.steps,
        "clocks": clk,
    }
    if dist.rank == 0:
        print(json.dumps(line), flush=True)


def run_int_peak(args, dist):
    """K5: sustained 32-bit operations per clock per SM for each op class."""
    import torch
    from paper_2407_09333_b300 import api, build

    build.build()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    names = ["LOP3", "IADD3", "SHF", "PRMT", "LOP3/IADD3/SHF", "IMAD", "LOP3/IMAD", "IADD3/IMAD",
             "SHF/IMAD", "LOP3/FFMA", "IMAD-add", "LOP3/IMAD-add", "LOP3/SHF/IADD3/IMAD-add",
             "IMAD.HI", "LOP3/IMAD.HI", "LOP3/rotation-as-IMAD-pair", "rotation-as-IMAD.WIDE+IMAD",
             "LOP3/rotation-as-IMAD.WIDE+IMAD", "SHF/rotation-as-IMAD.WIDE+IMAD"]
    threads, iters = 512, 4000
    blocks = sms * 4
    res = {}
    for op, name in enumerate(names):
        api.int_peak(op, blocks, threads, 200)
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        cyc = api.int_peak(op, blocks, threads, iters)
        e.record()
        e.synchronize()
        ms = s.elapsed_time(e)
        ops = blocks * threads * iters * api.int_peak_ops_per_iter()
        cmax = int(cyc.max().item())
        res[name] = {"ops_per_clk_per_sm": ops / cmax / sms, "tops": ops / ms / 1e9,
                     "clock_mhz": cmax / ms / 1e3}
    print(json.dumps({"int_peak": res, "sms": sms, "blocks": blocks, "threads": threads,
                      "iters": iters, "ops_per_iter": api.int_peak_ops_per_iter()}), flush=True)


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--workload", default="c2", choices=["c1", "c2", "c3", "c4", "c5", "paper"])
    p.add_argument("--requests", type=int, default=20000, help="requests per load point (c5)")
    p.add_argument("--loads", type=float, nargs="+", default=[0.1, 0.3, 0.5, 0.7, 0.9, 1.1],
                   help="offered loads as fractions of the ragged path's throughput (c5)")
    p.add_argument("--budget-gib", type=int, default=8, help="device-memory budget (c5)")
    p.add_argument("--rounds", type=int, default=2, help="streaming rounds in flight (c5)")
    p.add_argument("--segment-kib", type=int, default=32,
                   help="SM3 segment of long messages; SHA-1 2x, MD5 3x (c5)")
    p.add_argument("--serve-shape", type=int, default=11, help="launch shape of the rounds (c5)")
    p.add_argument("--serve-warps", type=int, default=8, help="resident warps per SM per round (c5)")
    p.add_argument("--staged", action="store_true",
                   help="serve through the staging copy instead of hashing segments where the "
                        "client's bytes are (c5)")
    p.add_argument("--pool-mib", type=int, default=2048, help="random-byte pool for requests (c5)")
    p.add_argument("--align", type=int, default=16,
                   help="messages start at multiples of this many bytes of the pool (c5; 1 = any)")
    p.add_argument("--slo-ms", type=float, default=100.0,
                   help="latency target of the admission-control point (c5)")
    p.add_argument("--cap-ms", type=float, default=0.0,
                   help="c5: hold requests on the host while the predicted in-flight work exceeds "
                        "this many ms (0 = admit while the ring has room)")
    p.add_argument("--no-other-mode", action="store_true",
                   help="c5: skip the comparison point in the other serving mode")
    p.add_argument("--no-admission", action="store_true",
                   help="c5: skip the cost model, its calibration and the admission-control point")
    p.add_argument("--host-requests", type=int, default=2000,
                   help="requests per load point of the host-ingress sweep (c5; 0 = skip)")
    p.add_argument("--host-loads", type=float, nargs="+", default=[0.5, 0.9],
                   help="host-ingress loads as fractions of the measured bus copy rate (c5)")
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--e2e-steps", type=int, default=10)
    p.add_argument("--e2e-slots", action="store_true",
                   help="e2e copies back 32-byte slots instead of packed digests")
    p.add_argument("--shape", type=int, default=None,
                   help="fixed launch shape index instead of the autotuner's choice")
    p.add_argument("--relay-blocks", type=int, default=None,
                   help="segment blocks of the fused kernel's relay form for batches of few "
                        "long messages (0 = grid-stride kernel only; default: the library's)")
    p.add_argument("--buckets", default="",
                   help="fixed ragged bucketing 'sub_log2,alg_major' (with --shape)")
    p.add_argument("--messages", type=int, default=0,
                   help="message count of the ragged workload (default 2^20) or of the paper "
                        "workload's strings (default all 10^9); smaller for profiling")
    p.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                   help="weak: every rank hashes its own batch; strong: the ranks split one batch "
                        "by estimated work")
    p.add_argument("--host-limit-mib", type=int, default=0,
                   help="device memory the e2e host path may use (0 = whole batch on the device)")
    p.add_argument("--separate", action="store_true",
                   help="plain workloads: one kernel per algorithm instead of the fused kernel")
    p.add_argument("--as-items", action="store_true",
                   help="plain workloads: the three-algorithm step as (message, algorithm) items "
                        "through the ragged kernel instead of the fused kernel")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="default run: skip the short long-message and ragged measurements")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--int-peak", action="store_true",
                   help="run the integer-issue microbenchmark instead of the hashing step")
    args = p.parse_args(argv)
    if args.warmup < 3:
        raise SystemExit("--warmup must be at least 3")
    dist = Dist(args.gpus)
    try:
        if args.int_peak:
            run_int_peak(args, dist)
        elif args.workload == "c5" and args.impl == "ours":
            run_serve(args, dist)
        elif args.workload == "paper" and args.impl == "ours":
            run_paper(args, dist)
        elif args.impl == "reference":
            run_reference(args, dist)
        else:
            run_ours(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
