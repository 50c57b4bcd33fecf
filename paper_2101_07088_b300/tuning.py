"""Cache of autotuned launch shapes (dpslab_plan_autotune), keyed by grid,
precision and device name, in a JSON file: a plan for a grid tuned before
takes the stored knobs instead of tuning again."""
import json
import os

from . import dpslab


def key(plan, device_name):
    d = plan.derived
    return f"{d['nx']}x{d['ny']}x{d['nz']}:p{int(plan.params.precision)}:{device_name}"


def load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tuned(plan, pos, q, path, reps=5):
    """Apply the cached knobs for this plan's grid, or autotune on (pos, q)
    and store them. Returns (knobs, whether they came from the cache)."""
    import torch
    name = torch.cuda.get_device_name()
    cache = load(path)
    k = key(plan, name)
    if k in cache:
        try:
            plan.set_tuning(cache[k])
            return cache[k], True
        except dpslab.DpslabError:
            pass
    knobs = plan.autotune(pos, q, reps)
    cache[k] = knobs
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return knobs, False
