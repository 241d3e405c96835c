"""Autotuner of the batched step's form and launch shape.

For a list of cases it times sph_batch_step over a few steps for every
(threads per block, resident blocks per SM) pair that the occupancy of the
persistent kernel allows, and for the phased form (one launch per phase),
on a scratch copy of the packed state, and keeps the fastest.  Results are cached as JSON keyed by GPU name, dimension,
precision and the power-of-two bucket of the packed particle count; the
cache lives in $SPH_TUNE_CACHE or ~/.cache/paper_1710_08259_gb300/tune.json.
"""
from __future__ import annotations

import json
import math
import os
from typing import Optional

from . import sph as S

BLOCKS = (64, 128, 256)


def cache_path() -> str:
    p = os.environ.get("SPH_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_1710_08259_gb300", "tune.json")


def _load():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(d):
    p = cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        tmp = p + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, p)
    except OSError:
        pass


def key_for(cases, precision) -> str:
    import torch
    n = sum(c.n for c in cases)
    name = torch.cuda.get_device_name()
    return f"{name}|d{cases[0].dim}|{'f32' if precision == S.SPH_PREC_F32 else 'f64'}|n2^{int(math.log2(max(n, 1)))}"


def time_config(cases, precision, block, bps, steps=3, form=S.SPH_BATCH_PERSISTENT) -> float:
    """ms per step of one form and launch shape (the state is a scratch copy)."""
    import torch
    t = S.SphTune()
    t.block, t.blocks_per_sm, t.spin_limit, t.form = block, bps, 0, form
    b = S.Batch(cases, precision, tune=t)
    try:
        b.step(steps)  # graph capture for this step count + warm-up
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        b.step(steps)
        e1.record()
        e1.synchronize()
        if b.status() != 0:
            return math.inf
        return e0.elapsed_time(e1) / steps
    finally:
        b.close()


def autotune(cases, precision=S.SPH_PREC_F32, steps=3, use_cache=True, verbose=False) -> dict:
    """Best {form, block, blocks_per_sm, ms_per_step} for these cases (cached)."""
    key = key_for(cases, precision)
    cache = _load() if use_cache else {}
    if use_cache and key in cache:
        return cache[key]
    results = []
    for blk in BLOCKS:
        probe = S.SphTune()
        probe.block, probe.blocks_per_sm, probe.spin_limit = blk, 0, 0
        b = S.Batch(cases[:1], precision, tune=probe)
        info = b.info()
        b.close()
        import torch
        nsm = torch.cuda.get_device_properties(0).multi_processor_count
        occ = max(1, info["grid"] // nsm)
        for bps in sorted({1, max(1, occ // 2), occ}):
            ms = time_config(cases, precision, blk, bps, steps)
            results.append({"form": "persistent", "block": blk, "blocks_per_sm": bps, "ms_per_step": ms})
            if verbose:
                print(results[-1])
    ms = time_config(cases, precision, 128, 0, steps, form=S.SPH_BATCH_PHASED)
    results.append({"form": "phased", "block": 128, "blocks_per_sm": 0, "ms_per_step": ms})
    if verbose:
        print(results[-1])
    best = min(results, key=lambda r: r["ms_per_step"])
    best = dict(best)
    best["tried"] = results
    if use_cache:
        cache[key] = best
        _store(cache)
    return best


def tune_struct(best: Optional[dict]) -> Optional[S.SphTune]:
    if not best:
        return None
    t = S.SphTune()
    t.block, t.blocks_per_sm, t.spin_limit = int(best["block"]), int(best["blocks_per_sm"]), 0
    t.form = S.SPH_BATCH_PHASED if best.get("form") == "phased" else S.SPH_BATCH_PERSISTENT
    return t
