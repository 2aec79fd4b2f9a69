"""JSON cache of autotuned ensemble tilings.

The key is the ensemble's signature: GPU name, precision and the sorted
member shapes.  The cache lives in $GRMHD_TUNING_CACHE, else
~/.cache/grmhd_gb300/ensemble_tiling.json.
"""
from __future__ import annotations

import json
import os

from . import grmhd as G


def cache_path() -> str:
    p = os.environ.get("GRMHD_TUNING_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "grmhd_gb300", "ensemble_tiling.json")


def signature(members, gpu_name: str) -> str:
    shapes = sorted(tuple(m.shape) for m in members)
    prec = "mixed" if members[0].grid.precision == G.MIXED else "fp64"
    return f"{gpu_name}|{prec}|" + ";".join("x".join(map(str, s)) for s in shapes)


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune_or_load(ens: G.Ensemble, gpu_name: str, trial_steps: int = 2) -> tuple[dict, bool]:
    """Apply the cached tiling of this ensemble if there is one, else run the
    autotuner and store its choice.  Returns (tiling, came_from_cache)."""
    key = signature(ens.members, gpu_name)
    db = _load()
    if key in db:
        t = db[key]
        G.ensemble_set_tiling(ens, t["items_flux"], t["items_update"], t["blocks_per_sm_flux"],
                              t["blocks_per_sm_update"], t.get("solo_log2", 0))
        return t, True
    t, _ = G.ensemble_autotune(ens, trial_steps)
    db[key] = t
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(db, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass
    return t, False
