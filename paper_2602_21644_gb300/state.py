"""Dump and restore of the tracking/mapping state for reproducible reruns:
Gaussian records (with their MP words), labels, poses, the pose optimiser's
Adam state, the learned network's blob, master weights and moments, and the
seeds that made the synthetic inputs. Plain .npz; tensors are copied to the
host on save and returned as numpy arrays on load."""
from __future__ import annotations

import json

import numpy as np

FORMAT = "dags-state-1"


def save_state(path: str, seeds: dict | None = None, **arrays) -> None:
    """save_state("run.npz", seeds={"scene": 0}, gauss=..., poses=..., adam=...)"""
    out = {}
    for k, v in arrays.items():
        if v is None:
            continue
        if hasattr(v, "detach"):                     # a torch tensor (any device)
            v = v.detach().cpu().numpy()
        out[k] = np.ascontiguousarray(v)
    meta = {"format": FORMAT, "seeds": seeds or {}, "dtypes": {k: str(v.dtype) for k, v in out.items()}}
    np.savez(path, __meta__=np.frombuffer(json.dumps(meta).encode(), np.uint8), **out)


def load_state(path: str):
    """(arrays dict, seeds dict) of a save_state file."""
    with np.load(path) as z:
        meta = json.loads(bytes(z["__meta__"]).decode())
        if meta.get("format") != FORMAT:
            raise ValueError(f"{path}: not a {FORMAT} file")
        arrays = {k: z[k] for k in z.files if k != "__meta__"}
    return arrays, meta.get("seeds", {})
