"""Autotuner of the tensor-core launches.

Tree / chain plans (tmc_plan_set_tuning): the tcgen05 tile is fixed by the M = 128
instruction shape and the S-chunk width by tensor memory, so the knobs are those of the
persistent edge launches:
  schedule       the order in which the CTAs take the edge tiles of a level (0, 1, 2)
  prologue_lead  chunks before the end of a forward item at which the next item's prologue
                 enters the ring and the MMA order (1, 2, 3)
  grid           CTAs per persistent launch (one per SM, or three quarters of that)
Loopy plans (tmc_loopy_plan_set_tile): the N tile of the message products (128 or 256).
The tuner times the plan's own step on the caller's inputs under every combination (CUDA
events, after warm-up), keeps the fastest, and caches the choice in a JSON file keyed by GPU
name, driver version and a digest of the problem's shape, so a later process with the same
shapes skips the timing.  No knob changes the arithmetic of a tile: every choice gives the same
log P_TMC bit for bit (tree plans) or up to the order of FP32 sums within a tile (loopy).
"""
from __future__ import annotations

import hashlib
import itertools
import json
import os

import numpy as np

SCHEDULES = (0, 1, 2)
PROLOGUE_LEADS = (1, 2, 3)
KEY_VERSION = "v2"  # the knob set; entries written by another knob set are not reused
DEFAULT_CACHE = os.environ.get("TMC_AUTOTUNE_CACHE",
                               os.path.join(os.path.expanduser("~"), ".cache", "tmc_gb300_autotune.json"))
GRADS = ("dq_mean", "dq_logstd", "dW", "dbias", "dC")


def problem_key(p, precision: str) -> str:
    h = hashlib.sha1()
    for a in (p.n, p.parent, p.K, p.d, p.obs):
        h.update(np.ascontiguousarray(a, dtype=np.int32).tobytes())
    for a in (p.Kn, p.dn):
        if a is not None:
            h.update(np.ascontiguousarray(a, dtype=np.int32).tobytes())
    h.update(("%d|%s|%d" % (int(p.shared), precision, int(p.q_A is not None))).encode())
    return h.hexdigest()[:16]


def device_key() -> str:
    import torch
    name = torch.cuda.get_device_name()
    drv = torch.cuda.get_device_properties(0).major, torch.cuda.get_device_properties(0).minor
    try:
        import subprocess
        drv = subprocess.run(["nvidia-smi", "--query-gpu=driver_version", "--format=csv,noheader"],
                             capture_output=True, text=True, timeout=10).stdout.strip().splitlines()[0]
    except Exception:
        pass
    return "%s|%s" % (name, drv)


def _events_ms(fn, reps=5, warm=2):
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _load(cache_path):
    if cache_path and os.path.exists(cache_path):
        try:
            return json.load(open(cache_path))
        except (OSError, ValueError):
            pass
    return {}


def _store(cache_path, cache):
    if not cache_path:
        return
    os.makedirs(os.path.dirname(cache_path) or ".", exist_ok=True)
    tmp = cache_path + ".%d.tmp" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, cache_path)


def grid_choices() -> tuple:
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    return (0, (3 * sms) // 4)


def apply(plan, choice: dict):
    for k in ("schedule", "prologue_lead", "grid"):
        plan.set_tuning(k, choice[k])


def autotune(plan, p, t, cache_path: str | None = DEFAULT_CACHE, force: bool = False) -> dict:
    """Chooses the persistent-launch knobs of ``plan`` (problem ``p``, device inputs ``t``)
    by timing one forward + parameter-gradient step per combination."""
    import torch
    key = "%s|%s|%s" % (KEY_VERSION, device_key(), problem_key(p, plan.precision))
    cache = _load(cache_path)
    if not force and key in cache:
        apply(plan, cache[key])
        return dict(cache[key], cached=True)
    out = torch.empty(p.B, dtype=torch.float64, device=t["eps"].device)
    src = {"dq_mean": "q_mean", "dq_logstd": "q_logstd", "dW": "W", "dbias": "bias", "dC": "C"}
    g = {k: torch.empty_like(t[src[k]]) for k in GRADS}

    def step():
        plan.forward(t, out=out)
        plan.backward(t, out=g, want=GRADS)

    times = {}
    for s, lead, grid in itertools.product(SCHEDULES, PROLOGUE_LEADS, grid_choices()):
        apply(plan, {"schedule": s, "prologue_lead": lead, "grid": grid})
        times["%d/%d/%d" % (s, lead, grid)] = _events_ms(step)
    best = min(times, key=times.get)
    s, lead, grid = (int(v) for v in best.split("/"))
    res = {"schedule": s, "prologue_lead": lead, "grid": grid, "ms": times,
           "spread": max(times.values()) / min(times.values()) - 1.0}
    apply(plan, res)
    cache[key] = res
    _store(cache_path, cache)
    return dict(res, cached=False)


def autotune_loopy(plan, p, t, cache_path: str | None = DEFAULT_CACHE, force: bool = False) -> dict:
    """Chooses the N tile of a loopy plan's message products by timing its forward."""
    import torch
    key = "%s|%s|loopy|%d|%d|%d|%d|%d" % (KEY_VERSION, device_key(), p.B, p.K, p.d, p.obs, int(p.shared))
    cache = _load(cache_path)
    if not force and key in cache:
        plan.set_tile(cache[key]["n_tile"])
        return dict(cache[key], cached=True)
    out = torch.empty(p.B, dtype=torch.float64, device=t["eps"].device)
    times = {}
    for n_tile in ((128, 256) if p.K > 128 else (128,)):
        plan.set_tile(n_tile)
        times[str(n_tile)] = _events_ms(lambda: plan.forward(t, out=out))
    best = int(min(times, key=times.get))
    plan.set_tile(best)
    res = {"n_tile": best, "ms": times, "spread": max(times.values()) / min(times.values()) - 1.0}
    cache[key] = res
    _store(cache_path, cache)
    return dict(res, cached=False)
