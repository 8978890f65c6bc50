"""Autotuner for the flight launch: block size, staged rate-table size and
particle sort period, chosen by timing short runs of the actual workload on
the device and cached per (GPU, workload shape) in a JSON file.

The cache lives at $EMC_AUTOTUNE_CACHE or ~/.cache/paper_1707_09073_gb300/
autotune.json.  Timings use CUDA events on a dedicated stream.
"""
from __future__ import annotations

import itertools
import json
import os
import time

from . import emc as _emc

DEFAULT_SPACE = {
    "block_size": (128, 256),
    "table_smem_kb": (16, 32, 64),
    "sort_period": (0, 10, 20, 40),
}


def cache_path() -> str:
    p = os.environ.get("EMC_AUTOTUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_1707_09073_gb300", "autotune.json")


def signature(cfgs: list[dict], precision: int) -> str:
    c0 = cfgs[0]
    n = sum(int(c["n_particles"]) for c in cfgs)
    cells = c0["nx"] * c0["ny"] * c0["nz"] if c0["geometry"] == 1 else 1
    # particle counts bucketed to a factor of two: tuning transfers within a bucket
    return "geom%d_ens%d_n2^%d_cells%d_prec%d" % (c0["geometry"], len(cfgs), max(n, 1).bit_length(), cells, precision)


def _device_name() -> str:
    import torch
    return torch.cuda.get_device_name()


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(d: dict):
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def time_candidate(cfgs: list[dict], params: dict, precision: int, chunks: int, warmup: int,
                   steps_per_chunk: int) -> float:
    """Seconds per chunk of `steps_per_chunk` steps for one parameter set."""
    import torch
    stream = torch.cuda.Stream()
    cand = [dict(c, **params) for c in cfgs]
    with torch.cuda.stream(stream):
        ctx = _emc.Context(cand, precision=precision, stream=stream.cuda_stream)
        try:
            for _ in range(warmup):
                ctx.emc_step(steps_per_chunk)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(chunks):
                ctx.emc_step(steps_per_chunk)
            b.record(stream)
            b.synchronize()
            return a.elapsed_time(b) * 1e-3 / chunks
        finally:
            ctx.close()


def tune(cfgs: list[dict], precision: int = _emc.FP32, space: dict | None = None, chunks: int = 30,
         warmup: int = 5, force: bool = False, verbose: bool = False) -> dict:
    """Return the best {block_size, table_smem_kb, sort_period} for this
    workload, from the cache when present."""
    space = space or DEFAULT_SPACE
    key = _device_name() + "|" + signature(cfgs, precision)
    cache = _load()
    if not force and key in cache:
        return dict(cache[key]["params"])
    c0 = cfgs[0]
    spc = c0["steps_per_poisson"] if c0["geometry"] == 1 else (c0.get("steps_per_launch") or 50)
    results = []
    names = list(space)
    t0 = time.time()
    for combo in itertools.product(*(space[k] for k in names)):
        params = dict(zip(names, combo))
        try:
            t = time_candidate(cfgs, params, precision, chunks, warmup, spc)
        except _emc.EmcError:
            continue
        results.append((t, params))
        if verbose:
            print("autotune", params, "%.3f ms/chunk" % (t * 1e3))
    results.sort(key=lambda r: r[0])
    best_t, best = results[0]
    cache[key] = {"params": best, "seconds_per_chunk": best_t, "tried": len(results),
                  "tuning_seconds": time.time() - t0}
    _store(cache)
    return dict(best)
