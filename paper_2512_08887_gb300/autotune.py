"""Autotuned plans: the stage-1 launch shapes (Stockham radix, transforms per CTA) chosen by timing
on the GPU (fbst_autotune) and cached in a JSON file keyed by problem size.

The cache path is the argument, else $FBST_AUTOTUNE_CACHE, else fbst_autotune.json in the system
temporary directory. A cached entry is applied with fbst_set_shapes; a miss runs the tuner once.
"""
from __future__ import annotations

import json
import os
import tempfile

from ._native import Plan


def cache_path(path: str | None = None) -> str:
    return path or os.environ.get("FBST_AUTOTUNE_CACHE") or os.path.join(tempfile.gettempdir(), "fbst_autotune.json")


def _key(plan: Plan, nblk: int) -> str:
    i, g = plan.info, plan.geom
    nu = ":nonuniform" if getattr(plan, "nonuniform", False) else ""
    return f"k{g.kind}:m{g.mx}x{g.my}:b{g.bx}x{g.by}:N{i.N}:L{i.L}:Pt{i.P_time}:Ps{i.P_space_x}:nb{nblk}{nu}"


def tune(plan: Plan, nblk: int, path: str | None = None, stream=None) -> tuple:
    """Apply the cached shapes for this plan and block count, or run the tuner and cache them."""
    p = cache_path(path)
    cache = {}
    if os.path.exists(p):
        try:
            with open(p) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    key = _key(plan, nblk)
    if key in cache:
        plan.set_shapes(*cache[key])
        return tuple(cache[key])
    shapes = plan.autotune(nblk, stream)
    cache[key] = list(shapes)
    tmp = p + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, p)
    return shapes
