"""Autotuning cache for libmertens.

``autotune(ns)`` runs the native ``mertens_autotune`` coordinate search for a
workload and stores the winning parameters in a JSON cache keyed by
(GPU name, floor(log10 max n), batch size); ``apply(ns)`` looks the key up and
installs the cached parameters with ``mertens_set_tuning``.  Parameters only
change speed, never results.
"""
from __future__ import annotations

import json
import math
import os

from . import _lib as L

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "libmertens", "tuning.json")


def _gpu_name() -> str:
    try:
        import torch

        return torch.cuda.get_device_name(torch.cuda.current_device())
    except Exception:  # noqa: BLE001 - no torch or no device: a generic key
        return "unknown-gpu"


def key(ns) -> str:
    ns = [int(v) for v in ns]
    return f"{_gpu_name()}|1e{int(math.log10(max(ns)))}|N{len(ns)}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def autotune(ns, runs: int = 1, cache_path: str = DEFAULT_CACHE) -> dict:
    """Searches, caches and returns {"tuning": ..., "ms": ...} for ns."""
    best, ms = L.mertens_autotune(ns, runs)
    cache = _load(cache_path)
    cache[key(ns)] = {"tuning": best, "ms": ms}
    os.makedirs(os.path.dirname(cache_path), exist_ok=True)
    tmp = cache_path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, cache_path)
    return cache[key(ns)]


def apply(ns, cache_path: str = DEFAULT_CACHE) -> dict | None:
    """Installs the cached tuning for ns if there is one; returns it."""
    hit = _load(cache_path).get(key(ns))
    if hit:
        L.mertens_set_tuning(**hit["tuning"])
        return hit["tuning"]
    return None
