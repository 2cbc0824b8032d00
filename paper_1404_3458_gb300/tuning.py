"""A JSON cache of autotuned transform plans (lch_autotune / lch_tune_set).

Plans depend on the GPU model and the library build, so the cache records
both and ignores entries made under another key.  Keys are "field/h/S".
"""
from __future__ import annotations

import json
import os

from . import lch


def _device_key() -> str:
    import torch

    lib = lch.LIB_PATH
    stamp = int(os.path.getmtime(lib)) if os.path.exists(lib) else 0
    return f"{torch.cuda.get_device_name()}|sm_{''.join(map(str, torch.cuda.get_device_capability()))}|{stamp}"


def _key(field: int, h: int, S: int) -> str:
    return f"{field}/{h}/{S}"


def load(path: str) -> dict:
    """The cache's plans for this device and build ({} when absent)."""
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return {}
    if data.get("device") != _device_key():
        return {}
    return dict(data.get("plans", {}))


def save(path: str, plans: dict):
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump({"device": _device_key(), "plans": plans}, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(ctx: "lch.Context", shapes, path: str | None = None, stream=None) -> dict:
    """Install a plan on `ctx` for every (field, h, shard_bytes) in `shapes`:
    from the cache at `path` when it has one, else by lch_autotune (and the
    cache is updated).  Returns the plans by key."""
    plans = load(path) if path else {}
    changed = False
    out = {}
    for field, h, S in shapes:
        if h < 2:
            continue
        k = _key(field, h, S)
        plan = plans.get(k)
        if plan is None:
            plan = ctx.autotune(field, h, S, stream=stream)
            plans[k] = plan
            changed = True
        else:
            ctx.tune_set(field, h, S, plan)
        out[k] = plan
    if path and changed:
        save(path, plans)
    return out
