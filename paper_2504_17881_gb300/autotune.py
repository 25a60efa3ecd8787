"""Autotuner of the batched launch: CTAs per lane, largest tile bits, single-CTA size.

The best lane size and tile size depend on the mix of run sizes: many small
runs favour short lanes (more runs in flight, fewer idle members), a few
large runs favour long lanes (each state's tiles spread over more SMs, fewer
states competing for L2).  The tuner times whole batch launches on the device
(CUDA events on the batch's stream, after one untimed launch) in three
stages -- lane size, then tile bits at the best lane size, then the largest
n run by one CTA alone (no lane barriers; longer single runs) -- and caches
the winner per device and batch signature in a JSON file.

Timing runs the real batch, so a tuning call costs a few launches of it per
candidate plus the host schedule of each candidate (about a second for 512
runs).
"""
from __future__ import annotations

import hashlib
import json
import os

from . import PS_C64, Batch

LANE_SIZES = (8, 16, 32, 64)
TILE_BITS = {PS_C64: (13, 12, 11, 10), 1: (12, 11, 10)}
SINGLE_BITS = (None, 15, 16, 17)  # None: the library default (one above the resident size)


def cache_file() -> str:
    base = os.environ.get("PS_TUNE_CACHE")
    if base:
        return base
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_2504_17881_gb300", "batch_tuning.json")


def signature(runs, ps_dtype: int, device_name: str) -> str:
    """Device, dtype and the work histogram of the batch: per n, the number
    of runs and the rotations (rounded to 2 significant digits)."""
    hist: dict[int, list] = {}
    for r in runs:
        h = hist.setdefault(int(r["n"]), [0, 0])
        h[0] += 1
        h[1] += len(r["x"])
    key = [device_name, ps_dtype] + [(n, c, float(f"{rot:.2g}")) for n, (c, rot) in sorted(hist.items())]
    return hashlib.sha256(json.dumps(key).encode()).hexdigest()[:24]


def _load():
    try:
        with open(cache_file()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(db):
    path = cache_file()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(db, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_batch(b: Batch, reps: int = 2) -> float:
    """Milliseconds of one launch: best of `reps` after one untimed launch."""
    import torch
    b.launch()
    b.wait()
    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(b.stream)
        b.launch()
        e1.record(b.stream)
        b.wait()
        best = min(best, e0.elapsed_time(e1))
    return best


def tune_batch(runs, dtype=None, reps: int = 2, use_cache: bool = True, lane_sizes=LANE_SIZES, tile_bits=None,
               log=None) -> dict:
    """Best {lane_size, tile_bits} for these runs (dicts as for Batch; their
    `state` tensors, if given, are reused by every candidate).  Returns the
    configuration plus the timings of every candidate."""
    import torch
    from . import _ps_dtype
    dtype = torch.complex64 if dtype is None else dtype
    psd = _ps_dtype(dtype)
    dev = runs[0]["psi0"].device if runs and runs[0].get("psi0") is not None else torch.device("cuda")
    sig = signature(runs, psd, torch.cuda.get_device_name(dev))
    db = _load() if use_cache else {}
    if use_cache and sig in db:
        return dict(db[sig], cached=True)
    # one set of output states for every candidate
    runs = [dict(r) for r in runs]
    for r in runs:
        if r.get("state") is None:
            r["state"] = torch.zeros(1 << int(r["n"]), dtype=dtype, device=dev)
    timings = {}

    def measure(cfg):
        key = json.dumps(cfg, sort_keys=True)
        if key not in timings:
            b = Batch(runs, dtype=dtype, cfg=cfg)
            timings[key] = time_batch(b, reps)
            b.close()
            if log:
                log(f"batch autotune {cfg}: {timings[key]:.3f} ms")
        return timings[key]

    best_lane = min(lane_sizes, key=lambda s: measure({"lane_size": s}))
    tbs = tile_bits or TILE_BITS[psd]
    best_tb = min(tbs, key=lambda t: measure({"lane_size": best_lane, "tile_bits": t}))

    def with_single(sb):
        cfg = {"lane_size": best_lane, "tile_bits": best_tb}
        if sb is not None:
            cfg["single_bits"] = sb
        return cfg

    best_sb = min(SINGLE_BITS, key=lambda sb: measure(with_single(sb)))
    best = with_single(best_sb)
    result = dict(best, ms=measure(best), timings_ms=timings, signature=sig)
    if use_cache:
        db = _load()
        db[sig] = result
        _store(db)
    return dict(result, cached=False)
