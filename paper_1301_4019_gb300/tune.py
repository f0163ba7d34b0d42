"""Autotuned launch shapes of the batched Metropolis path, cached on disk.

`rs_tune_batched` times every (threads per CTA, particles per thread) shape of the batched
Metropolis kernel and of the batched Permute on the caller's own batch and keeps the fastest in
the handle. Tuning costs a few hundred calls, so `autotune_batched` stores the choice in a JSON
file keyed by GPU model, dtype and the batch's size class (log2 of the particle and filter
counts) and re-applies it with `rs_set_batched_launch` when the same kind of batch comes again.
The shapes change only the speed: every ancestor is the same for any shape.
"""
from __future__ import annotations

import json
import math
import os

import torch


def default_cache_path() -> str:
    """$RS_TUNE_CACHE, else ~/.cache/paper_1301_4019_gb300/batched_launch.json."""
    env = os.environ.get("RS_TUNE_CACHE")
    if env:
        return env
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_1301_4019_gb300",
                        "batched_launch.json")


def cache_key(gpu: str, dtype: torch.dtype, particles: int, filters: int) -> str:
    """One entry per GPU model, dtype and size class (particles and filters rounded to the
    nearest power of two)."""
    dt = {torch.float32: "f32", torch.float64: "f64"}[dtype]
    n = round(math.log2(max(1, particles)))
    f = round(math.log2(max(1, filters)))
    return f"{gpu}|metropolis|{dt}|N2^{n}|F2^{f}"


def load_cache(path: str) -> dict:
    try:
        with open(path) as fh:
            data = json.load(fh)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(path: str, cache: dict) -> None:
    """Writes the whole cache atomically (temporary file, then rename)."""
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def autotune_batched(h, logw: torch.Tensor, offsets: torch.Tensor, B: int = 0,
                     B_per_filter: torch.Tensor | None = None, reps: int = 3,
                     cache_path: str | None = None, gpu: str | None = None,
                     _tune=None, _set=None) -> dict:
    """Applies the cached shapes for this kind of batch, or tunes them (rs_tune_batched) and
    caches the result. Returns {"metropolis": (block, ipt), "permute": (block, ipt),
    "cached": bool, "key": str}. `_tune` / `_set` replace the library calls (tests)."""
    import paper_1301_4019_gb300 as rs
    tune = _tune or rs.rs_tune_batched
    setter = _set or rs.rs_set_batched_launch
    if gpu is None:
        gpu = torch.cuda.get_device_name(logw.device)
    path = cache_path or default_cache_path()
    key = cache_key(gpu, logw.dtype, logw.numel(), offsets.numel() - 1)
    cache = load_cache(path)
    kernel = (rs.BATCHED_METROPOLIS_F64 if logw.dtype == torch.float64
              else rs.BATCHED_METROPOLIS_F32)
    entry = cache.get(key)
    if entry is not None:
        try:
            m, p = tuple(entry["metropolis"]), tuple(entry["permute"])
            setter(h, kernel, *m)
            setter(h, rs.BATCHED_PERMUTE, *p)
            return {"metropolis": m, "permute": p, "cached": True, "key": key}
        except (KeyError, TypeError, ValueError, rs.RsError):
            pass  # a stale or damaged entry: tune again
    shapes = tune(h, logw, offsets, B=B, B_per_filter=B_per_filter, reps=reps)
    m, p = tuple(shapes["metropolis"]), tuple(shapes["permute"])
    cache[key] = {"metropolis": list(m), "permute": list(p)}
    save_cache(path, cache)
    return {"metropolis": m, "permute": p, "cached": False, "key": key}
