"""Tile-size autotuner for the wavelet level kernels.

For a plan (N, L) it times a few warm iterations with each allowed tile edge
(MF_OPT_WAV_TILE = 64 or 32; the arithmetic is identical for both) using the
library's per-kernel CUDA-event timing, keeps the faster one, and caches the
choice in a JSON file keyed by (GPU name, N, L, precision).  The plan's ADMM
state is saved before and restored after the trials.
"""

from __future__ import annotations

import json
import os

from . import MF_OPT_WAV_TILE, Plan

TILES = (64, 32)
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "mf_gb300_autotune.json")


def _key(N, L, precision):
    import torch

    return f"{torch.cuda.get_device_name()}|N={N}|L={L}|prec={precision}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune(plan: Plan, y, iters: int = 3, cache: str | None = DEFAULT_CACHE, **params) -> dict:
    """Sets the fastest wavelet tile on `plan` and returns {"wav_tile": t, "ms": {t: ms}}."""
    precision = params.get("precision", 0)
    key = _key(plan.N, plan.L, precision)
    db = _load(cache) if cache else {}
    if key in db:
        plan.set_option(MF_OPT_WAV_TILE, int(db[key]["wav_tile"]))
        return db[key]
    state = plan.get_state().clone()
    params = dict(params)
    params.pop("warm_start", None)
    plan.iterate(y, 1, **params)  # a valid state to iterate from
    times = {}
    for t in TILES:
        plan.set_option(MF_OPT_WAV_TILE, t)
        plan.iterate(y, 1, warm_start=1, **params)
        plan.set_timing(True)
        plan.iterate(y, iters, warm_start=1, **params)
        tm = plan.timing()
        plan.set_timing(False)
        times[t] = sum(tm[k][0] for k in ("wav_level1", "wav_levelj")) / iters
    best = min(times, key=times.get)
    plan.set_option(MF_OPT_WAV_TILE, best)
    plan.set_state(state)
    rec = {"wav_tile": best, "ms": {str(k): v for k, v in times.items()}}
    if cache:
        db = _load(cache)
        db[key] = rec
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        tmp = cache + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(db, f, indent=1)
        os.replace(tmp, cache)
    return rec
