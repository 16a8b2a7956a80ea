"""Autotuner for the launch shape of the hashing kernels.

A shape is (warps per block, stages in flight per warp, 64-byte blocks per
stage, cooperative copies): the threads per block, how far ahead each warp
stages its messages (stages x blocks per stage x 32 lanes x 64 bytes, plus
alignment slack) and whether a warp copies message by message (cooperative)
or lane by lane.  For a given algorithm and a representative batch, every
shape is timed with CUDA events on the caller's stream, the three fastest
are timed again in turns (median of several launches), and the winner is
installed in the library (hash_tune_set); the ragged path also tunes its
bucketing and its resident warps per SM.  Results are cached in JSON keyed by device name,
SM count, algorithm (or "mixed") and a length class (floor(log2(mean
message length + 1))), so a later process with the same device and workload
shape reuses them without timing.
"""
from __future__ import annotations

import json
import math
import os

from . import api

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "hashbatch", "tune.json")


def cache_path() -> str:
    return os.environ.get("HB_TUNE_CACHE", DEFAULT_CACHE)


def length_class(mean_len: float) -> int:
    return int(math.floor(math.log2(max(mean_len, 0.0) + 1.0)))


def cache_key(device_name: str, sms: int, alg, mean_len: float) -> str:
    name = "mixed" if alg is None else "all" if alg == api.ALL else api.ALG_NAMES[alg]
    return "%s|%d|%s|L%d" % (device_name, sms, name, length_class(mean_len))


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str | None = None):
    path = path or cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp.%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time_ms(torch, fn, reps: int) -> float:
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record()
        fn()
        e.record()
        e.synchronize()
        best = min(best, s.elapsed_time(e))
    return best


def _final_round(torch, timings: dict, make, reps: int, finalists: int = 3, keep=None,
                 margin: float = 0.01):
    """The best of the first pass's `finalists` fastest candidates, timed
    again in turns (so that a drift of the clock hits all of them alike),
    by the median of several launches: one lucky launch in the first pass
    does not decide.  `keep` (the setting in force, when it was timed) always
    takes part and stays unless another candidate's median is more than
    `margin` below its own: candidates within a launch's noise of each other
    do not displace a setting chosen on longer measurements."""
    cands = sorted(timings, key=timings.get)[:finalists]
    if keep is not None and keep in timings and keep not in cands:
        cands.append(keep)
    if len(cands) == 1:
        return cands[0]
    samples = {k: [] for k in cands}
    for _ in range(max(5, 2 * reps)):
        for k in cands:
            samples[k].append(_time_ms(torch, make(k), 1))
    med = {k: sorted(samples[k])[len(samples[k]) // 2] for k in cands}
    best = min(cands, key=med.get)
    if keep in med and med[best] > med[keep] * (1.0 - margin):
        return keep
    return best


def tune(alg, packed, offsets, lengths, out, algs=None, mean_len: float | None = None,
         reps: int = 3, use_cache: bool = True, path: str | None = None) -> dict:
    """Pick and install the fastest shape for `alg` (None = the mixed path,
    api.ALL = the fused three-algorithm kernel; `out` then holds 96-byte
    records).

    Returns {"shape": index, "warps": w, "stages": s, "ms": {index: ms},
    "cached": bool}.
    """
    import torch

    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    if mean_len is None:
        mean_len = float(lengths.double().mean().item()) if lengths.numel() else 0.0
    key = cache_key(props.name, props.multi_processor_count, alg, mean_len)
    tune_alg = api.TUNE_MIXED if alg is None else alg
    shapes = api.shapes()
    cache = load_cache(path) if use_cache else {}
    if key in cache and 0 <= cache[key]["shape"] < len(shapes):
        api.tune_set(tune_alg, cache[key]["shape"])
        if alg is None and "buckets" in cache[key]:
            api.tune_buckets(*cache[key]["buckets"])
        if alg is None and "warps_per_sm" in cache[key]:
            api.tune_mixed_warps(cache[key]["warps_per_sm"])
        return dict(cache[key], cached=True)

    def run(idx):
        if alg is None:
            return lambda: api.hash_batch_mixed(algs, packed, offsets, lengths, out=out, shape=idx)
        if alg == api.ALL:
            return lambda: api.hash_batch_all(packed, offsets, lengths, out=out, shape=idx)
        return lambda: api.hash_batch(alg, packed, offsets, lengths, out=out, shape=idx)

    result = {"key": key}
    keep_shape = api.tune_get(tune_alg)  # the shape in force (the library's default at first)
    if alg is None:
        # Ragged path: bucket resolution and ordering first (default shape),
        # then the launch shape with the chosen bucketing.
        api.tune_mixed_warps(api.DEFAULT_MIXED_WARPS)
        btimes = {}
        for sub in (4, 5, 6):
            for major in (0, 1, 2):
                api.tune_buckets(sub, major)
                btimes[(sub, major)] = _time_ms(torch, run(keep_shape), reps)

        def with_buckets(k):
            api.tune_buckets(*k)
            return run(keep_shape)

        bbest = _final_round(torch, btimes, with_buckets, reps, keep=api.DEFAULT_BUCKETS)
        api.tune_buckets(*bbest)
        result["buckets"] = list(bbest)
        result["bucket_ms"] = {"%d,%d" % k: v for k, v in btimes.items()}
    timings = {}
    if alg is None:
        # launch shape x resident warps per SM (the persistent kernel's grid)
        for idx in range(len(shapes)):
            for wps in (8, 12, 16, 0):
                if wps and wps % shapes[idx][0]:
                    continue
                api.tune_mixed_warps(wps)
                timings[(idx, wps)] = _time_ms(torch, run(idx), reps)
        def with_warps(k):
            api.tune_mixed_warps(k[1])
            return run(k[0])

        (best, best_wps) = _final_round(torch, timings, with_warps, reps,
                                        keep=(keep_shape, api.DEFAULT_MIXED_WARPS))
        api.tune_mixed_warps(best_wps)
        result["warps_per_sm"] = best_wps
        ms = {"%d,%d" % k: v for k, v in timings.items()}
    else:
        for idx in range(len(shapes)):
            timings[idx] = _time_ms(torch, run(idx), reps)
        best = _final_round(torch, timings, run, reps, keep=keep_shape)
        ms = {str(k): v for k, v in timings.items()}
    api.tune_set(tune_alg, best)
    result.update({"shape": best, "warps": shapes[best][0], "stages": shapes[best][1],
                   "blocks_per_stage": shapes[best][2], "cooperative": shapes[best][3] == 1,
                   "copy_mapping": int(shapes[best][3]),
                   "ms": ms})
    if use_cache:
        cache = load_cache(path)
        cache[key] = result
        try:
            save_cache(cache, path)
        except OSError:
            pass
    return dict(result, cached=False)
