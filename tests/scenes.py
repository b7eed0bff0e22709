"""Small hand-made scenes and cached seeded scenes shared by the tests (inputs only)."""
from __future__ import annotations

import functools

import numpy as np

from paper_2406_12080_b300 import synth


def leaves_from(mean, scale, rot, opacity, sh=None) -> synth.Leaves:
    mean = np.atleast_2d(np.asarray(mean, np.float32))
    n = mean.shape[0]
    sh = np.zeros((n, 48), np.float32) if sh is None else np.asarray(sh, np.float32).reshape(n, 48)
    return synth.Leaves(np.ascontiguousarray(mean), np.ascontiguousarray(np.atleast_2d(scale), np.float32),
                        np.ascontiguousarray(np.atleast_2d(rot), np.float32),
                        np.ascontiguousarray(np.atleast_1d(opacity), np.float32), np.ascontiguousarray(sh))


def axis_camera(width, height, f, cx=None, cy=None, tau=6.0, pos=(0.0, 0.0, 0.0)) -> synth.Camera:
    """Camera at `pos` looking down +z (world axes = camera axes)."""
    R = np.eye(3, dtype=np.float32)
    T = -np.asarray(pos, np.float32)
    return synth.Camera(R, T, float(f), float(f), float(width / 2 if cx is None else cx),
                        float(height / 2 if cy is None else cy), int(width), int(height), float(tau))


def small_random_scene(n_leaves=64, seed=7, res=(48, 40), cube=1.0, dist=3.0, tau=6.0,
                       log_scale=-2.5):
    """A few dozen leaves in a small cube in front of a small camera (for brute force / FD)."""
    rng = np.random.default_rng(seed)
    mean = rng.uniform(-cube, cube, size=(n_leaves, 3))
    mean[:, 2] += dist
    scale = np.exp(rng.normal(log_scale, 0.4, size=(n_leaves, 3)))
    q = rng.normal(size=(n_leaves, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    op = 1 / (1 + np.exp(-rng.normal(0.5, 1.0, n_leaves)))
    sh = rng.normal(0, 0.3, size=(n_leaves, 48))
    lv = leaves_from(mean, scale, q, op, sh)
    w, h = res
    cam = axis_camera(w, h, f=0.9 * w, tau=tau)
    return lv, cam


@functools.lru_cache(maxsize=None)
def tiny():
    import oracle
    sc = synth.tiny_scene()
    return sc, oracle.build_tree(sc.leaves)


@functools.lru_cache(maxsize=None)
def corridor(n_leaves=1_000_000):
    import oracle
    sc = synth.corridor_scene(n_leaves=n_leaves)
    return sc, oracle.build_tree(sc.leaves)


def _city_chunk(a):
    seed, c, grid, per = a
    return c, synth.city_chunk_leaves(seed, c % grid, c // grid, per)


def city_device(ctx, grid=20, per=125_000, seed=2):
    """The chunked city (grid x grid chunks of `per` leaves) as device leaf tensors, generated on the
    host cores chunk by chunk (spawned workers: the parent already holds a CUDA context)."""
    import multiprocessing as mp
    import os
    import torch
    K = grid * grid
    L = K * per
    f = lambda *shape: torch.empty(shape, dtype=torch.float32, device="cuda")
    leaves = {"mean": f(L, 3), "scale": f(L, 3), "rot": f(L, 4), "opacity": f(L), "sh": f(L, 48)}
    with mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1))) as pool:
        for c, lv in pool.imap(_city_chunk, [(seed, c, grid, per) for c in range(K)], chunksize=4):
            for k in leaves:
                leaves[k][c * per:(c + 1) * per].copy_(torch.from_numpy(getattr(lv, k)))
    return leaves, np.arange(K + 1, dtype=np.int64) * per


@functools.lru_cache(maxsize=None)
def two_corridors(n_leaves=1_000_000):
    """Two copies of the corridor hierarchy under a new root (the second one shifted along x by the
    street's length; 4M nodes at the default size, a scan of several waves).  Ids:
    0 the new root, 1 and 2 the copies' roots, then the rest of the first copy, then of the second."""
    import oracle
    _, h = corridor(n_leaves)
    n = h.n
    shift = np.zeros(3, np.float32)
    shift[0] = float(h.box_max[0][0] - h.box_min[0][0]) * 1.05
    ida = np.concatenate([[1], np.arange(3, n + 2)])            # new id of the first copy's node i
    idb = np.concatenate([[2], np.arange(n + 2, 2 * n + 1)])    # and of the second copy's

    def cat(a, b_shift=None):
        b = a if b_shift is None else a + b_shift
        return np.ascontiguousarray(np.concatenate([a[:1], a[:1], b[:1], a[1:], b[1:]]))

    def topo(idm, arr_par, arr_cs):
        par = np.where(arr_par >= 0, idm[np.maximum(arr_par, 0)], 0).astype(np.int32)
        cs = np.where(h.child_count > 0, idm[np.minimum(arr_cs, n - 1)], 0).astype(np.int32)
        return par, cs

    pa, ca = topo(ida, h.parent, h.child_start)
    pb, cb = topo(idb, h.parent, h.child_start)
    parent = np.concatenate([[-1], pa[:1], pb[:1], pa[1:], pb[1:]]).astype(np.int32)
    child_start = np.concatenate([[1], ca[:1], cb[:1], ca[1:], cb[1:]]).astype(np.int32)
    child_count = np.concatenate([[2], h.child_count[:1], h.child_count[:1], h.child_count[1:],
                                  h.child_count[1:]]).astype(np.int32)
    bmin = cat(h.box_min, shift)
    bmax = cat(h.box_max, shift)
    bmin[0] = np.minimum(h.box_min[0], h.box_min[0] + shift)
    bmax[0] = np.maximum(h.box_max[0], h.box_max[0] + shift)
    return oracle.Hierarchy(cat(h.mean, shift), cat(h.scale), cat(h.rot), cat(h.opacity), cat(h.sh), bmin, bmax,
                            parent, child_start, child_count)


def random_case(seed):
    """A seeded random scene (50, 500 or 4096 leaves in a 10 m cube) and camera: inside the cube
    looking anywhere, or outside looking at it; random ragged resolution, field of view and tau."""
    rng = np.random.default_rng([seed, 91])
    n_leaves = int(rng.choice([50, 500, 4096]))
    sc = synth.tiny_scene(seed=200 + seed, n_leaves=n_leaves)
    import oracle
    h = oracle.build_tree(sc.leaves)
    inside = bool(rng.integers(2))
    pos = rng.uniform(2.0, 8.0, 3) if inside else np.array([5.0, 5.0, 5.0]) + rng.normal(size=3) * 12.0
    fwd = rng.normal(size=3) if inside else np.array([5.0, 5.0, 5.0]) - pos
    up = np.cross(fwd, rng.normal(size=3))
    w, hgt = int(rng.integers(150, 330)), int(rng.integers(100, 260))
    tau = float(np.exp(rng.uniform(np.log(0.5), np.log(50.0))))
    return h, synth.look_camera(pos, fwd, up, w, hgt, float(rng.uniform(40, 90)), tau)
