"""Autotuner for the batched bucket peel's launch shape.

Sweeps hpeel_batch_tuning (threads per block, blocks per SM, shared memory per
block) on a caller-given batched workload, times each candidate with CUDA
events, and caches the fastest per device (name, SM count, driver) and
workload class (number of buckets and median bucket size, rounded to powers
of two) in a JSON file beside the built library.  The tuning only changes
the schedule, never the results.
"""
from __future__ import annotations

import json
import math
import os
import threading

from . import _build_dir

CACHE = os.path.join(_build_dir(), "autotune.json")
_lock = threading.Lock()

CANDIDATES = [
    {"threads": t, "ctas_per_sm": c}
    for t in (128, 256, 512)
    for c in (1, 2, 3, 4, 6, 8)
    if t * c <= 2048
]


def _device_key(torch):
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    try:
        drv = torch.cuda.driver_version() if hasattr(torch.cuda, "driver_version") else ""
    except Exception:  # pragma: no cover - older torch
        drv = ""
    return f"{p.name}|sm{p.major}{p.minor}|{p.multi_processor_count}|{drv}"


def workload_key(B: int, median_keys: int, gamma_milli: int, with_g: bool) -> str:
    b2 = 1 << max(0, int(round(math.log2(max(B, 1)))))
    m2 = 1 << max(0, int(round(math.log2(max(median_keys, 1)))))
    return f"B{b2}|med{m2}|g{gamma_milli}|G{int(with_g)}"


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(data):
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def tune(keys, bucket_off, gamma_milli: int = 1230, with_g: bool = False, reps: int = 3,
         candidates=None, force: bool = False):
    """Best tuning dict for this workload on the current device (cached)."""
    import numpy as np
    import torch

    from . import batched_workspace_size, peel_batched

    B = bucket_off.shape[0] - 1
    sizes = (bucket_off[1:] - bucket_off[:-1]).cpu().numpy()
    key = _device_key(torch) + "||" + workload_key(B, int(np.median(sizes)) if B else 0,
                                                   gamma_milli, with_g)
    with _lock:
        cache = _load()
        if not force and key in cache:
            return cache[key]["tuning"]
    results = []
    for cand in candidates or CANDIDATES:
        need = batched_workspace_size(B, gamma_milli, cand)
        if need == 0:
            continue
        ws = torch.empty(need, dtype=torch.uint8, device=keys.device)
        out = peel_batched(keys, bucket_off, gamma_milli, with_g=with_g, tuning=cand, workspace=ws)
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            peel_batched(keys, bucket_off, gamma_milli, with_g=with_g, tuning=cand,
                         workspace=ws, out=out)
            b.record()
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        results.append((best, cand))
        del ws
    results.sort(key=lambda x: x[0])
    best_ms, best = results[0]
    with _lock:
        cache = _load()
        cache[key] = {"tuning": best, "ms": best_ms,
                      "sweep": [{"tuning": c, "ms": t} for t, c in results]}
        _store(cache)
    return best
