"""Work-unit autotuner for the matrix-profile kernel.

The diagonal kernel splits each band of 512 diagonals into work units of a
given number of rows.  Larger units start fewer anchors, smaller
units balance the last wave better; the best height depends on the GPU, the
subsequence length and the size and shape of the stream layout.  `tune` times
mp_selfjoin at a few candidate heights with the library's own CUDA-event
kernel timing and stores the fastest per layout bucket in a JSON cache;
`rows_for` returns the cached choice (0, the library's automatic rule, when a
layout was never tuned).
"""
from __future__ import annotations

import functools
import json
import math
import os
import threading
from typing import Callable, Sequence

import numpy as np

CANDIDATES = (0, 2048, 3072, 4096, 6144)
_lock = threading.Lock()
_mem: dict = {}
_loaded_from: str | None = None


def cache_path() -> str:
    p = os.environ.get("TSK_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "tsketch", "tile_rows.json")


def layout_key(stream_len: Sequence[int], m: int, excl: int, device_name: str, sm_count: int) -> str:
    """Bucket a layout: total cells and stream count to half/whole powers of two."""
    e = np.asarray(stream_len, dtype=np.float64) - m + 1 - excl
    e = e[e > 0]
    cells = float(np.sum(e * (e + 1) / 2.0))
    cb = round(2.0 * math.log2(max(cells, 1.0))) / 2.0
    sb = round(math.log2(max(len(stream_len), 1)))
    return f"{device_name}|sm{sm_count}|m{m}|e{excl}|c{cb:g}|s{sb}"


def _load() -> dict:
    global _loaded_from
    path = cache_path()
    if _loaded_from != path:
        _mem.clear()
        try:
            with open(path) as f:
                _mem.update(json.load(f))
        except (OSError, ValueError):
            pass
        _loaded_from = path
    return _mem


def _save() -> None:
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(_mem, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


@functools.lru_cache(maxsize=None)
def _device_props(index: int):
    import torch
    props = torch.cuda.get_device_properties(index)
    return props.name, props.multi_processor_count


def _device():
    import torch
    return _device_props(torch.cuda.current_device())


def rows_for(stream_len: Sequence[int], m: int, excl: int, device_name: str | None = None,
             sm_count: int | None = None) -> int:
    """Cached rows per work unit for this layout bucket (0 when untuned)."""
    if device_name is None or sm_count is None:
        device_name, sm_count = _device()
    with _lock:
        return int(_load().get(layout_key(stream_len, m, excl, device_name, sm_count), 0))


def select(timings: dict) -> int:
    """The candidate with the smallest time (ties: the smaller height, 0 first)."""
    return min(timings, key=lambda r: (timings[r], r))


def record(stream_len: Sequence[int], m: int, excl: int, rows: int, device_name: str, sm_count: int) -> None:
    with _lock:
        _load()[layout_key(stream_len, m, excl, device_name, sm_count)] = int(rows)
        _save()


def tune(X, stream_len: Sequence[int], m: int, excl: int, candidates=CANDIDATES, reps: int = 2,
         timer: Callable[[int], float] | None = None) -> int:
    """Time each candidate height and cache the fastest; returns it.

    `timer(rows) -> milliseconds` defaults to running mp_selfjoin on X with that
    height and reading the kernel's device time.
    """
    device_name, sm_count = _device() if timer is None else ("cpu", 0)
    if timer is None:
        from . import api

        def timer(rows: int) -> float:
            api.mp_selfjoin(X, stream_len, m, excl, tile_rows=rows)  # warm the layout
            api.sync()
            api.profile_enable(True)
            api.profile_read("mp_diag")
            for _ in range(reps):
                api.mp_selfjoin(X, stream_len, m, excl, tile_rows=rows)
            api.sync()
            ms, launches = api.profile_read("mp_diag")
            api.profile_enable(False)
            return ms / max(launches, 1)

    timings = {int(r): float(timer(int(r))) for r in candidates}
    best = select(timings)
    record(stream_len, m, excl, best, device_name, sm_count)
    return best
