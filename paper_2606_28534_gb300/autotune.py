"""Autotuner of an ensemble's launch configuration (pic_batch_tuning), cached in JSON per
(GPU, ensemble shape).

The configuration does not change any result (every simulation of a batch computes the same state
whatever the shape of the step kernel, the CTA counts or the use of graphs), only the time a step
takes.  The tuner times candidates on the batch itself, over whole cycles of 2 * sort_interval
steps (so that each trial holds the same share of sort steps as a long run, and a graph replay),
with CUDA events on the batch's stream:

1. every compiled shape of the particle-step kernel, with as many CTAs per SM as fit;
2. for the fastest shape, fewer CTAs per SM;
3. for the fastest so far, launching the steps one by one instead of replaying a CUDA graph.

It then sets the winner and returns the batch to its initial state (pic_batch_reset), since the
trials advanced it.  The cache key holds the GPU's name and SM count, the compiled shapes, the
number of runs and log2 buckets of the total particle count and of the mean particles per run; a
hit sets the cached configuration without any trial.
"""
from __future__ import annotations

import json
import math
import os

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "paper_2606_28534_gb300", "tuning.json")


def shape_key(params_list, device_name: str, sms: int, variants) -> str:
    n = len(params_list)
    total = sum(int(p["ncells"]) * (int(p["ppc"][0]) + int(p["ppc"][1])) for p in params_list)
    per_run = total / max(1, n)
    return (f"{device_name}|sms={sms}|shapes={','.join(variants)}|runs={n}"
            f"|particles=2^{round(math.log2(max(1, total)))}|per_run=2^{round(math.log2(max(1.0, per_run)))}")


def load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(path: str, cache: dict) -> None:
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _valid_entry(e, nvariants: int) -> bool:
    try:
        t = e["tuning"]
        return 0 <= int(t["variant"]) < nvariants and int(t["ctas_per_sm"]) >= 0 and \
            isinstance(t["use_graph"], bool) and isinstance(e["ms_per_step"], (int, float))
    except (KeyError, TypeError, ValueError):
        return False


def cuda_timer(batch, steps: int) -> float:
    """Milliseconds of ``steps`` steps between two CUDA events on the batch's stream."""
    import torch

    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(batch.stream)
    batch.step(steps)
    b.record(batch.stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def _device():
    import torch

    d = torch.cuda.current_device()
    return torch.cuda.get_device_name(d), torch.cuda.get_device_properties(d).multi_processor_count


def tune(batch, *, cache_path: str | None = None, force: bool = False, timer=None, device=None,
         variants=None, max_ctas: int = 8) -> dict:
    """Pick and set the fastest launch configuration of ``batch`` (a ``pic.Batch`` or anything with
    its ``params``, ``set_tuning``, ``step``, ``sync`` and ``reset``).  Returns
    ``{"tuning": ..., "ms_per_step": ..., "cached": bool, "trials": [...], "key": ...}``."""
    from . import pic

    cache_path = cache_path or os.environ.get("PIC_TUNING_CACHE") or DEFAULT_CACHE
    timer = timer or cuda_timer
    name, sms = device if device is not None else _device()
    variants = list(variants) if variants is not None else pic.batch_variants()
    key = shape_key(batch.params, name, sms, variants)
    cache = load_cache(cache_path)
    if not force and _valid_entry(cache.get(key), len(variants)):
        e = cache[key]
        batch.set_tuning(**e["tuning"])
        return {"tuning": dict(e["tuning"]), "ms_per_step": e["ms_per_step"], "cached": True, "trials": [],
                "key": key}

    cycle = 2 * int(batch.params[0]["sort_interval"])
    trials = []

    def trial(t: dict):
        try:
            batch.set_tuning(**t)
        except pic.PicError as err:
            if err.status == 1:  # not a valid configuration on this GPU (e.g. too many CTAs)
                return None
            raise
        batch.step(cycle)  # warm-up: first touch, graph capture
        batch.sync()
        ms = timer(batch, cycle) / cycle
        batch.sync()
        trials.append({"tuning": dict(t), "ms_per_step": ms})
        return ms

    base = {"variant": 0, "ctas_per_sm": 0, "use_graph": True}
    best, best_ms = None, math.inf
    for v in range(len(variants)):
        t = dict(base, variant=v)
        ms = trial(t)
        if ms is not None and ms < best_ms:
            best, best_ms = t, ms
    if best is None:
        raise RuntimeError("no launch configuration of the batch could be timed")
    for c in range(1, max_ctas + 1):
        t = dict(best, ctas_per_sm=c)
        ms = trial(t)
        if ms is not None and ms < best_ms:
            best, best_ms = t, ms
    t = dict(best, use_graph=False)
    ms = trial(t)
    if ms is not None and ms < best_ms:
        best, best_ms = t, ms
    batch.set_tuning(**best)
    batch.reset()  # the trials advanced the batch
    cache[key] = {"tuning": best, "ms_per_step": best_ms, "variant_name": variants[best["variant"]]}
    save_cache(cache_path, cache)
    return {"tuning": dict(best), "ms_per_step": best_ms, "cached": False, "trials": trials, "key": key}
