"""Cache of autotuned settings per (graph class, GPU).

``tuned(handle, graph, sample)`` applies cached settings when this GPU has
already tuned a graph of the same class, and otherwise runs dawn_autotune
(short timed trials in the library) and stores the result.  The graph class
is (n, m, symmetric, log2 of the largest out-degree): graphs drawn by the same
generator at the same size share settings.  The cache is a small JSON file.
"""
from __future__ import annotations

import json
import os
from pathlib import Path

import numpy as np

from . import dawn

DEFAULT_CACHE = Path(os.environ.get("DAWN_TUNING_CACHE", Path.home() / ".cache" / "dawn_b300" / "tuning.json"))


def graph_class(n: int, m: int, symmetric: bool, max_degree: int) -> str:
    return f"n{n}_m{m}_{'sym' if symmetric else 'dir'}_d{int(np.log2(max(1, max_degree)))}"


def gpu_name() -> str:
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.get_device_name(0)
    except ImportError:
        pass
    return "unknown"


def _load(path: Path) -> dict:
    try:
        return json.loads(path.read_text())
    except (OSError, ValueError):
        return {}


def tuned(handle: int, row_ptr, col_idx, symmetric: bool, sample, cache: Path | None = None) -> dict:
    """Settings for `handle`: from the cache when present, else measured and cached."""
    cache = Path(cache) if cache else DEFAULT_CACHE
    n = int(row_ptr.shape[0] - 1)
    m = int(col_idx.shape[0])
    deg = np.diff(np.asarray(row_ptr))
    key = f"{gpu_name()}|{graph_class(n, m, symmetric, int(deg.max()) if n else 0)}"
    data = _load(cache)
    if key in data:
        dawn.dawn_set_tuning(handle, data[key])
        return dict(data[key], cached=True)
    t = dawn.dawn_autotune(handle, np.ascontiguousarray(sample, dtype=np.int32))
    data[key] = t
    try:
        cache.parent.mkdir(parents=True, exist_ok=True)
        tmp = cache.with_suffix(".tmp")
        tmp.write_text(json.dumps(data, indent=1, sort_keys=True))
        tmp.replace(cache)
    except OSError:
        pass  # read-only home: the settings still apply to this handle
    return dict(t, cached=False)
