"""Autotuning of the two passes' kernel shapes, with a JSON cache.

``tune(plan)`` asks the library to time every compiled column-pass variant
(tile width, columns per thread, pipelined or lockstep staging) on the plan's
own buffers (tbs_autotune) and every steady-state row-pass variant
(persistent or one block per row; tbs_autotune_rows), and keeps the fastest
of each.  Results are cached per (GPU, kernel sources, M, n_rhs, grid kind)
so later plans reuse the choice with tbs_set_col_variant and
tbs_set_row_variant instead of timing again, and a rebuilt library with
changed kernels times afresh.
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
    # the row shapes available depend on N as well as M (odd N has no
    # persistent row pass), so their count is part of the key
    return "%s|src=%s|M=%d|nrhs=%d|%s|row_shapes=%d" % (_gpu_name(), build.source_hash(), plan.m, plan.n_rhs,
                                                        "periodic" if plan.periodic else "padded",
                                                        tbs.tbs_row_variants(plan.handle))


def tune(plan, cache_path: str | None = DEFAULT_CACHE, reps: int = 5, force: bool = False):
    """Select the column- and row-pass variants of `plan`.

    Returns ((column variant, row variant), times or None): times is
    {"col": [ms per variant], "row": [ms per variant]} when they were timed,
    None when the cache supplied the choice."""
    ncv = tbs.tbs_col_variants(plan.handle)
    nrv = tbs.tbs_row_variants(plan.handle)
    if ncv <= 1 and nrv <= 1:
        return (0, 0), None
    key = _key(plan)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except Exception:
            cache = {}
    hit = cache.get(key) if not force else None
    if hit and 0 <= int(hit.get("col", -1)) < ncv and 0 <= int(hit.get("row", -1)) < nrv:
        tbs.tbs_set_col_variant(plan.handle, int(hit["col"]))
        tbs.tbs_set_row_variant(plan.handle, int(hit["row"]))
        return (int(hit["col"]), int(hit["row"])), None
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    cbest, ctimes = tbs.tbs_autotune(plan.handle, reps, stream) if ncv > 1 else (0, None)
    rbest, rtimes = tbs.tbs_autotune_rows(plan.handle, reps, stream) if nrv > 1 else (0, None)
    times = {"col": ctimes, "row": rtimes}
    if cache_path:
        with _lock:
            os.makedirs(os.path.dirname(cache_path), exist_ok=True)
            cache[key] = {"col": cbest, "row": rbest, "ms": times}
            tmp = cache_path + ".%d.tmp" % os.getpid()
            json.dump(cache, open(tmp, "w"), indent=1)
            os.replace(tmp, cache_path)
    return (cbest, rbest), times
