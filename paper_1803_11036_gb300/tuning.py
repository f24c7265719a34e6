"""A file cache of launch configurations picked by ``Context.autotune``.

The library's autotuner (``ssd_autotune``) times one field of the launch
configuration at a time on the caller's own slot; the result depends on the
GPU, the parameter set, the number of routers and the size of a slot, and on
nothing else. This module keys the chosen configuration by exactly those, so a
deployment tunes once per (GPU, parameters, routers, slot-size class) and later
contexts take the stored configuration without timing anything. The cache is a
JSON object {key: {field: value}}; a missing or unreadable file is an empty
cache. No stored value can change a result: every field only spreads the same
work differently.
"""
from __future__ import annotations

import json
import math
import os
import tempfile

from ._abi import TUNING_FIELDS, Params

_PARAM_FIELDS = ("log2_eta", "q", "r", "delta", "k", "theta", "flags")


def size_class(pairs_per_slot: int) -> int:
    """Slots whose total pair count rounds to the same power of two share a configuration."""
    return 0 if pairs_per_slot <= 0 else int(round(math.log2(pairs_per_slot)))


def cache_key(device_name: str, params: Params, n_routers: int, pairs_per_slot: int) -> str:
    p = "-".join(f"{f}{int(getattr(params, f))}" for f in _PARAM_FIELDS)
    return f"{device_name.strip()}|{p}|n{int(n_routers)}|s{size_class(pairs_per_slot)}"


def load(path: str) -> dict:
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return {}
    if not isinstance(data, dict):
        return {}
    out = {}
    for k, v in data.items():
        if isinstance(v, dict) and set(v) == set(TUNING_FIELDS) and all(isinstance(x, int) for x in v.values()):
            out[k] = v
    return out


def store(path: str, key: str, tuning: dict) -> None:
    """Add or replace one entry (written to a temporary file, then renamed over the cache)."""
    if set(tuning) != set(TUNING_FIELDS):
        raise ValueError(f"a tuning has the fields {TUNING_FIELDS}")
    data = load(path)
    data[key] = {f: int(tuning[f]) for f in TUNING_FIELDS}
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=d, prefix=".tuning-", suffix=".json")
    with os.fdopen(fd, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tuned(ctx, routers, pairs_list, global_sketch=None, path: str | None = None, reps: int = 3) -> dict:
    """The context's configuration for this slot shape: from the cache at `path` when it holds
    one, else picked by ctx.autotune (same preconditions: no slot run yet) and stored there."""
    import torch
    n_pairs = sum(int(t.numel()) // 2 for t in pairs_list)
    key = cache_key(torch.cuda.get_device_name(ctx.device), ctx.params, len(routers), n_pairs)
    if path is not None:
        hit = load(path).get(key)
        if hit is not None:
            ctx.tuning = hit
            return dict(hit)
    t = ctx.autotune(routers, pairs_list, global_sketch, reps=reps)
    if path is not None:
        store(path, key, t)
    return t
