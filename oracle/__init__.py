"""TEST INFRASTRUCTURE ONLY: Python wrapper around the CPU oracle (h3dgs_oracle.cpp).

The oracle is a plain CPU restatement of the paper's method (fp64 values, fp32 decisions; see
the header of h3dgs_oracle.cpp).  Only tests, the smoke check and the benchmark's CPU-baseline
leg may import this package; the product library never does.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "h3dgs_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

NSH = 48
NATTR = 59
NINTERP = 62
NVAL = 13


def build(force: bool = False) -> str:
    """Compile the oracle with IEEE semantics (no fast-math, no contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", _LIB + ".tmp", _SRC]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class OrCamera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("T", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("znear", C.c_float), ("tau", C.c_float)]


class OrHier32(C.Structure):
    _fields_ = [("n", C.c_int64)] + [(k, C.POINTER(C.c_float)) for k in
                                     ("mean", "scale", "rot", "opacity", "sh", "box_min", "box_max")] + \
               [(k, C.POINTER(C.c_int32)) for k in ("parent", "child_start", "child_count")]


class OrHier64(C.Structure):
    _fields_ = [(k, C.POINTER(C.c_double)) for k in ("mean", "scale", "rot", "opacity", "sh")]


class OrOpts(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("lowpass", C.c_float),
                ("aa_compensate", C.c_int32), ("interpolate", C.c_int32), ("alpha_clamp", C.c_float),
                ("alpha_floor", C.c_float), ("t_min", C.c_float), ("bg", C.c_float * 3)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.or_build_tree.restype = C.c_int64
        _lib.or_select_cut.restype = C.c_int64
        _lib.or_select_cut_descent.restype = C.c_int64
        _lib.or_compact.restype = C.c_int64
        _lib.or_tile_lists.restype = C.c_int64
        _lib.or_weighted_image_sum.restype = C.c_double
        _lib.or_rotation_angle.restype = C.c_double
        _lib.or_num_threads.restype = C.c_int32
        _lib.or_ellipsoid_area.restype = C.c_double
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------------- data

@dataclass
class Hierarchy:
    """Node arrays (fp32, the stored format), BFS order, children contiguous."""
    mean: np.ndarray
    scale: np.ndarray
    rot: np.ndarray
    opacity: np.ndarray
    sh: np.ndarray
    box_min: np.ndarray
    box_max: np.ndarray
    parent: np.ndarray
    child_start: np.ndarray
    child_count: np.ndarray

    @property
    def n(self):
        return int(self.mean.shape[0])

    def c32(self):
        h = OrHier32()
        h.n = self.n
        for k in ("mean", "scale", "rot", "opacity", "sh", "box_min", "box_max"):
            setattr(h, k, _p(getattr(self, k), C.c_float))
        for k in ("parent", "child_start", "child_count"):
            setattr(h, k, _p(getattr(self, k), C.c_int32))
        h._keep = self
        return h


@dataclass
class Attrs64:
    """Value-track attributes in double (perturbed by the finite-difference checks)."""
    mean: np.ndarray
    scale: np.ndarray
    rot: np.ndarray
    opacity: np.ndarray
    sh: np.ndarray

    @staticmethod
    def of(h: Hierarchy) -> "Attrs64":
        return Attrs64(*[_f64(getattr(h, k)) for k in ("mean", "scale", "rot", "opacity", "sh")])

    def c64(self):
        a = OrHier64()
        for k in ("mean", "scale", "rot", "opacity", "sh"):
            setattr(a, k, _p(getattr(self, k), C.c_double))
        a._keep = self
        return a


@dataclass
class Opts:
    tile_w: int = 16
    tile_h: int = 16
    lowpass: float = 0.3
    aa_compensate: int = 1
    interpolate: int = 1
    alpha_clamp: float = 0.99
    alpha_floor: float = float(np.float32(1.0) / np.float32(255.0))
    t_min: float = 1e-4
    bg: tuple = (0.0, 0.0, 0.0)

    def c(self):
        o = OrOpts()
        for k in ("tile_w", "tile_h", "lowpass", "aa_compensate", "interpolate", "alpha_clamp",
                  "alpha_floor", "t_min"):
            setattr(o, k, getattr(self, k))
        o.bg = (C.c_float * 3)(*self.bg)
        return o


def camera(cam) -> OrCamera:
    c = OrCamera()
    c.R = (C.c_float * 9)(*np.asarray(cam.R, np.float32).reshape(-1).tolist())
    c.T = (C.c_float * 3)(*np.asarray(cam.T, np.float32).tolist())
    c.fx, c.fy, c.cx, c.cy = cam.fx, cam.fy, cam.cx, cam.cy
    c.width, c.height, c.znear, c.tau = cam.width, cam.height, cam.znear, cam.tau
    return c


def tiles(cam, opts: Opts):
    return (cam.width + opts.tile_w - 1) // opts.tile_w, (cam.height + opts.tile_h - 1) // opts.tile_h


# --------------------------------------------------------------------------------- builder

def build_tree(leaves) -> Hierarchy:
    L = leaves.n
    N = 2 * L - 1
    out = Hierarchy(np.empty((N, 3), np.float32), np.empty((N, 3), np.float32),
                    np.empty((N, 4), np.float32), np.empty(N, np.float32),
                    np.empty((N, NSH), np.float32), np.empty((N, 3), np.float32),
                    np.empty((N, 3), np.float32), np.empty(N, np.int32), np.empty(N, np.int32),
                    np.empty(N, np.int32))
    args = [_f32(leaves.mean), _f32(leaves.scale), _f32(leaves.rot), _f32(leaves.opacity),
            _f32(leaves.sh)]
    n = lib().or_build_tree(C.c_int64(L), *[_p(a, C.c_float) for a in args],
                            *[_p(getattr(out, k), C.c_float) for k in
                              ("mean", "scale", "rot", "opacity", "sh", "box_min", "box_max")],
                            *[_p(getattr(out, k), C.c_int32) for k in
                              ("parent", "child_start", "child_count")])
    assert n == N, (n, N)
    return out


def _rows64(h: Hierarchy, v: int) -> np.ndarray:
    """Node v's attribute row (mean 3, scale 3, rot 4, opacity 1, sh 48) in double."""
    return np.concatenate([h.mean[v], h.scale[v], h.rot[v], [h.opacity[v]], h.sh[v]]).astype(np.float64)


def consolidate(chunks: list) -> Hierarchy:
    """Chunk hierarchies joined under a global root (Sec. 6.3, chunk consolidation), step by step as
    the reading states it: every chunk keeps the hierarchy built from its own leaves; a top tree is
    built over the chunk roots with the rules of the chunk trees -- a group's box is the union of its
    members' boxes (a chunk root's box is its leaf-union box), it is split at the median of the members'
    means projected on the longest box axis (ties to the lower axis; members ordered by (projected mean,
    chunk index); the left child takes the first floor(n/2)), interior nodes merge their two children
    (Eq. merge) and are orientation-matched top-down, the chunk roots keeping their own frames.  Node
    order: the top tree breadth-first (its leaves are the chunk roots), then each chunk's nodes except
    its root in the chunk's breadth-first order."""
    K = len(chunks)
    root_mean = np.stack([c.mean[0] for c in chunks]).astype(np.float32)
    root_lo = np.stack([c.box_min[0] for c in chunks]).astype(np.float32)
    root_hi = np.stack([c.box_max[0] for c in chunks]).astype(np.float32)
    perm = list(range(K))
    tnodes = [[0, K, -1, 0, -1]]          # lo, hi, first child, child count, parent
    cur = 0
    while cur < len(tnodes):
        lo, hi = tnodes[cur][0], tnodes[cur][1]
        if hi - lo >= 2:
            mem = perm[lo:hi]
            bmin, bmax = root_lo[mem].min(axis=0), root_hi[mem].max(axis=0)
            ext = bmax.astype(np.float64) - bmin.astype(np.float64)
            axis = int(np.argmax(ext))           # the first maximum: ties to the lower axis
            perm[lo:hi] = sorted(mem, key=lambda c: (root_mean[c, axis], c))
            mid = lo + (hi - lo) // 2
            tnodes[cur][2], tnodes[cur][3] = len(tnodes), 2
            tnodes.append([lo, mid, -1, 0, cur])
            tnodes.append([mid, hi, -1, 0, cur])
        cur += 1
    n_top = len(tnodes)
    chunk_of = {v: perm[t[0]] for v, t in enumerate(tnodes) if t[3] == 0}   # top leaf -> chunk
    # bottom-up merge of the top tree's interior nodes (double rows), then boxes
    rows = [None] * n_top
    lo_b = np.zeros((n_top, 3), np.float32)
    hi_b = np.zeros((n_top, 3), np.float32)
    for v in range(n_top - 1, -1, -1):
        t = tnodes[v]
        if t[3] == 0:
            c = chunk_of[v]
            rows[v] = _rows64(chunks[c], 0)
            lo_b[v], hi_b[v] = chunks[c].box_min[0], chunks[c].box_max[0]
        else:
            kids = [t[2], t[2] + 1]
            rows[v] = merge_rows(np.stack([rows[k] for k in kids]))
            lo_b[v] = np.minimum(lo_b[kids[0]], lo_b[kids[1]])
            hi_b[v] = np.maximum(hi_b[kids[0]], hi_b[kids[1]])
    # top-down orientation matching inside the top tree (chunk roots keep their frames)
    for v in range(n_top):
        t = tnodes[v]
        for k in range(t[2], t[2] + t[3]):
            if tnodes[k][3] > 0:
                rows[k] = match_orientation(rows[v], rows[k])
    sizes = [c.n - 1 for c in chunks]
    bases = n_top + np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    N = n_top + int(np.sum(sizes))
    out = Hierarchy(np.empty((N, 3), np.float32), np.empty((N, 3), np.float32), np.empty((N, 4), np.float32),
                    np.empty(N, np.float32), np.empty((N, NSH), np.float32), np.empty((N, 3), np.float32),
                    np.empty((N, 3), np.float32), np.empty(N, np.int32), np.empty(N, np.int32),
                    np.empty(N, np.int32))
    top_of_chunk = {c: v for v, c in chunk_of.items()}
    for v in range(n_top):
        t = tnodes[v]
        if t[3] == 0:   # a chunk root: its own (fp32) row, box and children
            c = chunk_of[v]
            h = chunks[c]
            for k in ("mean", "scale", "rot", "opacity", "sh", "box_min", "box_max"):
                getattr(out, k)[v] = getattr(h, k)[0]
            out.child_count[v] = h.child_count[0]
            out.child_start[v] = bases[c] + h.child_start[0] - 1 if h.child_count[0] > 0 else -1
        else:
            r = rows[v]
            out.mean[v], out.scale[v], out.rot[v] = r[0:3], r[3:6], r[6:10]
            out.opacity[v], out.sh[v] = r[10], r[11:59]
            out.box_min[v], out.box_max[v] = lo_b[v], hi_b[v]
            out.child_count[v], out.child_start[v] = t[3], t[2]
        out.parent[v] = t[4]
    for c, h in enumerate(chunks):
        g = slice(int(bases[c]), int(bases[c]) + h.n - 1)
        for k in ("mean", "scale", "rot", "opacity", "sh", "box_min", "box_max"):
            getattr(out, k)[g] = getattr(h, k)[1:]
        par = h.parent[1:].astype(np.int64)
        out.parent[g] = np.where(par == 0, top_of_chunk[c], bases[c] + par - 1)
        cs = h.child_start[1:].astype(np.int64)
        out.child_start[g] = np.where(h.child_count[1:] > 0, bases[c] + cs - 1, -1)
        out.child_count[g] = h.child_count[1:]
    return out


def merge_rows(rows: np.ndarray) -> np.ndarray:
    rows = _f64(rows)
    out = np.empty(NATTR, np.float64)
    lib().or_merge(C.c_int32(rows.shape[0]), _p(rows, C.c_double), _p(out, C.c_double))
    return out


def match_orientation(parent_row: np.ndarray, child_row: np.ndarray) -> np.ndarray:
    p = _f64(parent_row).copy()
    c = _f64(child_row).copy()
    lib().or_match_orientation(_p(p, C.c_double), _p(c, C.c_double))
    return c


def rotation_angle(qa, qb) -> float:
    a, b = _f64(qa), _f64(qb)
    return lib().or_rotation_angle(_p(a, C.c_double), _p(b, C.c_double))


# --------------------------------------------------------------------------------- cut

def granularity(cam, h: Hierarchy) -> np.ndarray:
    eps = np.empty(h.n, np.float32)
    lib().or_granularity(C.byref(camera(cam)), C.byref(h.c32()), _p(eps, C.c_float))
    return eps


def select_cut(cam, h: Hierarchy, interpolate: int = 1):
    ids = np.empty(h.n, np.int32)
    t = np.empty(h.n, np.float32)
    m = lib().or_select_cut(C.byref(camera(cam)), C.byref(h.c32()), C.c_int32(interpolate),
                            _p(ids, C.c_int32), _p(t, C.c_float), C.c_int64(h.n))
    return ids[:m].copy(), t[:m].copy()


def select_cut_descent(cam, h: Hierarchy):
    ids = np.empty(h.n, np.int32)
    m = lib().or_select_cut_descent(C.byref(camera(cam)), C.byref(h.c32()), _p(ids, C.c_int32),
                                    C.c_int64(h.n))
    return ids[:m].copy()


def compact(cams, h: Hierarchy, tau_min: float, tau_max: float):
    """Compacted hierarchy (Sec. 5.2) over the training cameras `cams`.

    Returns (Hierarchy, old_of_new): the kept nodes renumbered breadth-first with their attribute
    rows and boxes unchanged, and the old index of every new node."""
    N = h.n
    oc = (OrCamera * max(len(cams), 1))(*[camera(c) for c in cams])
    old = np.empty(N, np.int32)
    par, cs, cc = np.empty(N, np.int32), np.empty(N, np.int32), np.empty(N, np.int32)
    m = lib().or_compact(oc, C.c_int32(len(cams)), C.byref(h.c32()), C.c_float(tau_min), C.c_float(tau_max),
                         _p(old, C.c_int32), _p(par, C.c_int32), _p(cs, C.c_int32), _p(cc, C.c_int32))
    if m < 0:
        raise ValueError("compact: tau_min must be > 0 and tau_max finite")
    o = old[:m].copy()
    g = lambda a: np.ascontiguousarray(a[o])
    out = Hierarchy(g(h.mean), g(h.scale), g(h.rot), g(h.opacity), g(h.sh), g(h.box_min), g(h.box_max),
                    par[:m].copy(), cs[:m].copy(), cc[:m].copy())
    return out, o


def stream_trace(cams, h: Hierarchy, update_every: int = 2, cleanup_every: int = 100, max_age: int = 100,
                 interpolate: int = 1):
    """Node residency of streamed rendering along a camera path (Sec. 6.3: the cut is updated every
    few frames by transferring the nodes it needs from CPU RAM to the GPU; a cleanup runs every 100
    frames).  Frame f = 0, 1, ...:
      * if f % update_every == 0: the cut of cams[f]; the needed nodes are its nodes and the parents
        of its entries with t != 0; the ones not resident are transferred; all needed are stamped f;
      * the frame renders that cut;
      * if (f + 1) % cleanup_every == 0: every resident node with f - stamp > max_age is evicted.
    Returns (transfers per update, resident count after each cleanup, resident count at the end)."""
    resident = np.zeros(h.n, bool)
    stamp = np.full(h.n, -1, np.int64)
    transfers, after_cleanup = [], []
    for f, cam in enumerate(cams):
        if f % update_every == 0:
            ids, t = select_cut(cam, h, interpolate)
            par = h.parent[ids]
            need = np.zeros(h.n, bool)
            need[ids] = True
            need[par[(t != 0) & (par >= 0)]] = True
            transfers.append(int(np.sum(need & ~resident)))
            resident |= need
            stamp[need] = f
        if (f + 1) % cleanup_every == 0:
            resident &= ~(f - stamp > max_age)
            after_cleanup.append(int(resident.sum()))
    return transfers, after_cleanup, int(resident.sum())


# --------------------------------------------------------------------------------- render

def interpolate(h: Hierarchy, ids, t, a64: Attrs64 | None = None):
    a64 = a64 or Attrs64.of(h)
    M = len(ids)
    o32 = np.empty((NINTERP, M), np.float32)
    o64 = np.empty((NINTERP, M), np.float64)
    ids, t = np.ascontiguousarray(ids, np.int32), _f32(t)
    lib().or_interpolate(C.byref(h.c32()), C.byref(a64.c64()), C.c_int64(M), _p(ids, C.c_int32),
                         _p(t, C.c_float), _p(o32, C.c_float), _p(o64, C.c_double))
    return o32, o64


@dataclass
class Frame:
    ids: np.ndarray
    t: np.ndarray
    rec32: np.ndarray      # [M, 10] u v ca cb cc on op t K depth (fp32 decision track)
    rect: np.ndarray       # [M, 4]  x0 x1 y0 y1, -1 if culled
    val64: np.ndarray      # [M, 13] u v A B C on op t K r g b z (fp64 value track)
    ranges: np.ndarray | None = None   # [tiles, 2]
    lists: np.ndarray | None = None    # [P] splat indices (cut positions)
    image: np.ndarray | None = None    # [3, H, W] fp64
    T_final: np.ndarray | None = None
    n_contrib: np.ndarray | None = None
    ambiguous: np.ndarray | None = None
    depth: np.ndarray | None = None    # [H, W] expected depth sum(T alpha z), fp64


def preprocess(cam, h: Hierarchy, ids, t, opts: Opts, a64: Attrs64 | None = None) -> Frame:
    a64 = a64 or Attrs64.of(h)
    M = len(ids)
    ids, t = np.ascontiguousarray(ids, np.int32), _f32(t)
    rec = np.empty((M, 10), np.float32)
    rect = np.empty((M, 4), np.int32)
    val = np.empty((M, NVAL), np.float64)
    lib().or_preprocess(C.byref(camera(cam)), C.byref(opts.c()), C.byref(h.c32()),
                        C.byref(a64.c64()), C.c_int64(M), _p(ids, C.c_int32), _p(t, C.c_float),
                        _p(rec, C.c_float), _p(rect, C.c_int32), _p(val, C.c_double))
    return Frame(ids, t, rec, rect, val)


def tile_lists(cam, fr: Frame, opts: Opts):
    TX, TY = tiles(cam, opts)
    ranges = np.empty((TX * TY, 2), np.int32)
    M = len(fr.ids)
    cap = max(1, int(np.sum(np.where(fr.rect[:, 0] >= 0,
                                     (fr.rect[:, 1] - fr.rect[:, 0] + 1) * (fr.rect[:, 3] - fr.rect[:, 2] + 1),
                                     0))))
    lists = np.empty(cap, np.int32)
    P = lib().or_tile_lists(C.byref(camera(cam)), C.byref(opts.c()), C.c_int64(M), _p(fr.rec32, C.c_float),
                            _p(fr.rect, C.c_int32), _p(ranges, C.c_int32), _p(lists, C.c_int32),
                            C.c_int64(cap))
    assert P <= cap
    fr.ranges, fr.lists = ranges, lists[:P].copy()
    return fr


def blend(cam, fr: Frame, opts: Opts, exposure=None):
    """Image (exposure = the camera's 3x4 affine, row-major, applied when given), expected depth,
    final transmittance, contributor counts and the ambiguity flags."""
    H, W = cam.height, cam.width
    img = np.empty((3, H, W), np.float64)
    dep = np.empty((H, W), np.float64)
    Tf = np.empty((H, W), np.float64)
    nc = np.empty((H, W), np.int32)
    amb = np.empty((H, W), np.uint8)
    lists = fr.lists if len(fr.lists) else np.zeros(1, np.int32)
    E = None if exposure is None else np.ascontiguousarray(exposure, np.float32).reshape(12)
    lib().or_blend(C.byref(camera(cam)), C.byref(opts.c()), _p(fr.rec32, C.c_float), _p(fr.val64, C.c_double),
                   _p(fr.ranges, C.c_int32), _p(lists, C.c_int32), None if E is None else _p(E, C.c_float),
                   _p(img, C.c_double), _p(dep, C.c_double), _p(Tf, C.c_double), _p(nc, C.c_int32),
                   _p(amb, C.c_uint8))
    fr.image, fr.depth, fr.T_final, fr.n_contrib, fr.ambiguous = img, dep, Tf, nc, amb.astype(bool)
    return fr


def blend_bruteforce(cam, fr: Frame, opts: Opts) -> np.ndarray:
    img = np.empty((3, cam.height, cam.width), np.float64)
    lib().or_blend_bruteforce(C.byref(camera(cam)), C.byref(opts.c()), C.c_int64(len(fr.ids)),
                              _p(fr.rec32, C.c_float), _p(fr.rect, C.c_int32), _p(fr.val64, C.c_double),
                              _p(img, C.c_double))
    return img


def render(cam, h: Hierarchy, opts: Opts | None = None, a64: Attrs64 | None = None,
           cut=None, exposure=None) -> Frame:
    """Cut -> interpolate/project -> tile lists -> blend, all on the CPU."""
    opts = opts or Opts()
    # t is a property of the cut (camera + hierarchy); interpolate = 0 only zeroes it when rendering
    ids, t = cut if cut is not None else select_cut(cam, h, 1)
    fr = preprocess(cam, h, ids, t, opts, a64)
    tile_lists(cam, fr, opts)
    return blend(cam, fr, opts, exposure)


def backward(cam, h: Hierarchy, fr: Frame, dL_dimage: np.ndarray, opts: Opts,
             a64: Attrs64 | None = None, freeze_leaves: int = 0, dL_ddepth=None, exposure=None) -> np.ndarray:
    """Gradient [N, 59] of sum(dL_dimage * image) + sum(dL_ddepth * depth) w.r.t. node attributes
    (fp64); the image carries the exposure when given."""
    a64 = a64 or Attrs64.of(h)
    g = np.empty((h.n, NATTR), np.float64)
    dl = _f64(dL_dimage)
    dd = None if dL_ddepth is None else _f64(dL_ddepth)
    E = None if exposure is None else np.ascontiguousarray(exposure, np.float32).reshape(12)
    lists = fr.lists if len(fr.lists) else np.zeros(1, np.int32)
    lib().or_backward(C.byref(camera(cam)), C.byref(opts.c()), C.byref(h.c32()), C.byref(a64.c64()),
                      C.c_int64(len(fr.ids)), _p(fr.ids, C.c_int32), _p(fr.t, C.c_float),
                      _p(fr.rec32, C.c_float), _p(fr.rect, C.c_int32), _p(fr.val64, C.c_double),
                      _p(fr.ranges, C.c_int32), _p(lists, C.c_int32), _p(dl, C.c_double),
                      None if dd is None else _p(dd, C.c_double), None if E is None else _p(E, C.c_float),
                      C.c_int32(freeze_leaves), _p(g, C.c_double))
    return g


def weighted_image_sum(cam, h: Hierarchy, fr: Frame, w: np.ndarray, opts: Opts, a64: Attrs64,
                       w_depth=None, exposure=None) -> float:
    """sum(w * image) + sum(w_depth * depth) of the fp64 track with the decisions of `fr` held fixed."""
    M = len(fr.ids)
    val = np.empty((M, NVAL), np.float64)
    rec = np.empty((M, 10), np.float32)
    rect = np.empty((M, 4), np.int32)
    lib().or_preprocess(C.byref(camera(cam)), C.byref(opts.c()), C.byref(h.c32()), C.byref(a64.c64()),
                        C.c_int64(M), _p(fr.ids, C.c_int32), _p(fr.t, C.c_float), _p(rec, C.c_float),
                        _p(rect, C.c_int32), _p(val, C.c_double))
    w = _f64(w)
    wd = None if w_depth is None else _f64(w_depth)
    E = None if exposure is None else np.ascontiguousarray(exposure, np.float32).reshape(12)
    lists = fr.lists if len(fr.lists) else np.zeros(1, np.int32)
    return lib().or_weighted_image_sum(C.byref(camera(cam)), C.byref(opts.c()), _p(fr.rec32, C.c_float),
                                       _p(val, C.c_double), _p(fr.ranges, C.c_int32), _p(lists, C.c_int32),
                                       None if E is None else _p(E, C.c_float), _p(w, C.c_double),
                                       None if wd is None else _p(wd, C.c_double))


def pair_alpha(fr: Frame, splat, px, py, opts: Opts):
    """alpha of splat `splat[i]` of frame `fr` at pixel position (px[i], py[i]) in both tracks:
    (fp32 decision track, fp64 value track)."""
    s = np.ascontiguousarray(splat, np.int32)
    x, y = _f64(px), _f64(py)
    a32 = np.empty(len(s), np.float32)
    a64 = np.empty(len(s), np.float64)
    lib().or_pair_alpha(_p(fr.rec32, C.c_float), _p(fr.val64, C.c_double), C.c_int64(len(s)), _p(s, C.c_int32),
                        _p(x, C.c_double), _p(y, C.c_double), C.c_float(opts.alpha_clamp), _p(a32, C.c_float),
                        _p(a64, C.c_double))
    return a32, a64


def ellipsoid_area(s) -> float:
    a = _f64(s)
    return lib().or_ellipsoid_area(_p(a, C.c_double))


def sh_basis(d) -> np.ndarray:
    out = np.empty(16, np.float64)
    lib().or_sh_basis(C.c_double(d[0]), C.c_double(d[1]), C.c_double(d[2]), _p(out, C.c_double))
    return out


def num_threads() -> int:
    return int(lib().or_num_threads())
