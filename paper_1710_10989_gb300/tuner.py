"""Driver of the batched path's autotuner (bbc_batch_tune): runs the library's
timing loop once per GPU model and reservation, caches the choice (product family
and product shapes per size bucket, persistent grid) in a JSON file and restores
it on later runs.

    from paper_1710_10989_gb300 import api, tuner
    h = api.Handle(0)
    h.batch_reserve(256, api.PREC_OZAKI)
    mask, ctas = tuner.tuned(h, 256)
"""
from __future__ import annotations

import json
import os

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_CACHE = os.path.join(HERE, "_build", "batch_tuning.json")


def _gpu_key(device: int) -> str:
    import torch
    p = torch.cuda.get_device_properties(device)
    return f"{p.name}|sm{p.major}{p.minor}|{p.multi_processor_count}SM"


def cache_key(gpu: str, max_n: int, tol: float) -> str:
    return f"{gpu}|max_n={int(max_n)}|tol={float(tol)!r}"


def load(path: str) -> dict:
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def save(path: str, data: dict) -> None:
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tuned(h, max_n: int, tol: float = 0.0, path: str = DEFAULT_CACHE, force: bool = False,
          gpu: str | None = None) -> tuple[int, int]:
    """(split_mask, ctas) for this handle's GPU: from the cache, else measured by
    bbc_batch_tune and cached. Installs the choice, shapes included, in the handle
    either way (a cache entry without shapes restores the default shapes)."""
    key = cache_key(gpu if gpu is not None else _gpu_key(h.device), max_n, tol)
    data = load(path)
    hit = data.get(key)
    if hit and not force:
        h.batch_set_tuning(int(hit["split_mask"]), int(hit["ctas"]))
        h.batch_set_shapes(hit.get("shapes"))
        return int(hit["split_mask"]), int(hit["ctas"])
    mask, ctas = h.batch_tune(max_n, tol)
    data[key] = {"split_mask": mask, "ctas": ctas, "shapes": list(h.batch_get_shapes())}
    save(path, data)
    return mask, ctas
