"""Autotuner for the core kernel's variant, cached per (GPU, dtype, size class).

The library times each variant on a representative frame (lacos_autotune)
and keeps the fastest.  The choice is stored in a JSON cache keyed by the
GPU name, the frame dtype and a size class, so later contexts apply it with
lacos_set_core_variant without re-timing.  The cache path is
$LACOS_AUTOTUNE_CACHE, else ~/.cache/lacos_gb300/autotune.json.
"""
from __future__ import annotations

import json
import os


def cache_path() -> str:
    return os.environ.get("LACOS_AUTOTUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "lacos_gb300", "autotune.json")


def size_class(ny: int, nx: int) -> str:
    npx = ny * nx
    if npx < (1 << 20):
        return "lt1Mpx"
    if npx < (16 << 20):
        return "1to16Mpx"
    return "ge16Mpx"


def key(gpu_name: str, dtype: str, ny: int, nx: int) -> str:
    return f"{gpu_name}|{dtype}|{size_class(ny, nx)}"


def load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def store(entries: dict) -> None:
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(entries, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(ctx, frame, params, mask, clean, reps: int = 2, use_cache: bool = True):
    """Apply the cached variant for this frame's class, or time the variants and cache
    the winner.  Returns (variant, per-variant ms or None when taken from the cache)."""
    import torch
    name = torch.cuda.get_device_name(frame.device)
    dt = "u16" if frame.dtype == torch.uint16 else "f32"
    k = key(name, dt, *frame.shape)
    entries = load() if use_cache else {}
    if k in entries:
        ctx.set_core_variant(int(entries[k]["variant"]))
        return int(entries[k]["variant"]), None
    best, ms = ctx.autotune(frame, params, mask, clean, reps)
    entries = load()
    entries[k] = {"variant": best, "ms": ms}
    store(entries)
    return best, ms
