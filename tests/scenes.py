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
