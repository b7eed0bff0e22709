"""Hierarchy files: save and load the node arrays (the layouts of h3dgs_hierarchy).

A file is a NumPy .npz archive with a format version, the node count and SH degree, and the ten
arrays (mean [N,3], scale [N,3], rot [N,4], opacity [N], sh [N,48], box_min [N,3], box_max [N,3] as
little-endian fp32; parent, child_start, child_count [N] as little-endian int32).  Loading checks
the version, the shapes and the topology invariants the library relies on (parent < child,
children contiguous and pointing back at their parent).
"""
from __future__ import annotations

import numpy as np

FORMAT_VERSION = 1
FLOAT_KEYS = ("mean", "scale", "rot", "opacity", "sh", "box_min", "box_max")
INT_KEYS = ("parent", "child_start", "child_count")
WIDTH = {"mean": 3, "scale": 3, "rot": 4, "opacity": 0, "sh": 48, "box_min": 3, "box_max": 3}


def _host(a):
    return a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)


def save_hierarchy(path: str, hier) -> None:
    """hier: any object with the ten arrays as attributes (numpy arrays or torch tensors)."""
    arrs = {k: np.ascontiguousarray(_host(getattr(hier, k)), "<f4") for k in FLOAT_KEYS}
    arrs.update({k: np.ascontiguousarray(_host(getattr(hier, k)), "<i4") for k in INT_KEYS})
    n = arrs["mean"].shape[0]
    np.savez(path, version=np.int64(FORMAT_VERSION), n_nodes=np.int64(n), sh_degree=np.int64(3), **arrs)


def load_hierarchy(path: str) -> dict:
    """Returns the ten arrays (numpy) after checking the format and the topology."""
    with np.load(path) as f:
        if int(f["version"]) != FORMAT_VERSION:
            raise ValueError(f"unsupported hierarchy file version {int(f['version'])}")
        n = int(f["n_nodes"])
        out = {k: f[k].astype(np.float32) for k in FLOAT_KEYS}
        out.update({k: f[k].astype(np.int32) for k in INT_KEYS})
    for k in FLOAT_KEYS:
        want = (n,) if WIDTH[k] == 0 else (n, WIDTH[k])
        if out[k].shape != want:
            raise ValueError(f"{k}: shape {out[k].shape}, expected {want}")
    for k in INT_KEYS:
        if out[k].shape != (n,):
            raise ValueError(f"{k}: shape {out[k].shape}, expected ({n},)")
    par, cs, cc = out["parent"], out["child_start"], out["child_count"]
    if n < 1 or par[0] != -1 or np.any(par[1:] < 0) or np.any(par[1:] >= np.arange(1, n)):
        raise ValueError("parents must precede their children and the root must be node 0")
    inner = np.nonzero(cc > 0)[0]
    kids = np.repeat(cs[inner], cc[inner]) + np.concatenate([np.arange(c) for c in cc[inner]]) if len(inner) else []
    if len(inner) and (np.any(kids >= n) or np.any(par[kids] != np.repeat(inner, cc[inner]))):
        raise ValueError("child ranges must point at nodes whose parent is the range's owner")
    if int(cc.sum()) != n - 1:
        raise ValueError("every node but the root must be exactly one node's child")
    return out
