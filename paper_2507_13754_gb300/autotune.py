"""Column-pass tile-shape autotuning with a JSON cache.

``tune(plan)`` asks the library to time every compiled column-pass variant for
the plan's padded size on the plan's own buffers (tbs_autotune) and keeps the
fastest; results are cached per (GPU, kernel sources, M, n_rhs) so later
plans reuse the choice with tbs_set_col_variant instead of timing again, and
a rebuilt library with changed kernels times afresh.
"""
from __future__ import annotations

import json
import os
import threading

from . import build, tbs

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "tbs_gb300_autotune.json")
_lock = threading.Lock()


def _gpu_name():
    try:
        import torch
        return torch.cuda.get_device_name()
    except Exception:
        return "unknown"


def _key(plan):
    return "%s|src=%s|M=%d|nrhs=%d" % (_gpu_name(), build.source_hash(), plan.m, plan.n_rhs)


def tune(plan, cache_path: str | None = DEFAULT_CACHE, reps: int = 5, force: bool = False):
    """Select the column-pass variant of `plan`; returns (variant, times or None)."""
    nv = tbs.tbs_col_variants(plan.handle)
    if nv <= 1:
        return 0, None
    key = _key(plan)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except Exception:
            cache = {}
    if not force and key in cache and 0 <= int(cache[key]["variant"]) < nv:
        tbs.tbs_set_col_variant(plan.handle, int(cache[key]["variant"]))
        return int(cache[key]["variant"]), None
    import torch
    best, times = tbs.tbs_autotune(plan.handle, reps, torch.cuda.current_stream().cuda_stream)
    if cache_path:
        with _lock:
            os.makedirs(os.path.dirname(cache_path), exist_ok=True)
            cache[key] = {"variant": best, "ms": times}
            tmp = cache_path + ".%d.tmp" % os.getpid()
            json.dump(cache, open(tmp, "w"), indent=1)
            os.replace(tmp, cache_path)
    return best, times
