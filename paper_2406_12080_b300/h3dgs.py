"""Thin Python binding of libh3dgs (include/h3dgs.h): argument marshalling only.

Every function named h3dgs_* forwards to the C entry point of the same name.  Buffers are torch
CUDA tensors (device memory) and the context's stream is a torch stream; all arithmetic runs in
the library's CUDA kernels.  If the library is missing this module raises instead of falling
back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os
import re
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# the library to load: H3DGS_LIB names another build (e.g. the bounds-checked libh3dgs_check.so)
LIB_PATH = os.environ.get("H3DGS_LIB") or os.path.join(_PKG, "libh3dgs.so")
HEADER_PATH = os.path.join(os.path.dirname(_PKG), "include", "h3dgs.h")

H3DGS_OK = 0
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "CAPACITY", 5: "TIMEOUT", 6: "STATE",
                7: "NO_DEVICE"}
NINTERP = 62


class H3dgsError(RuntimeError):
    def __init__(self, status: int, msg: str, total: int | None = None):
        super().__init__(f"h3dgs {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status
        self.total = total      # the untruncated size, for CAPACITY errors that report one


class h3dgs_camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("T", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("znear", C.c_float), ("tau", C.c_float)]


class h3dgs_hierarchy(C.Structure):
    _fields_ = [("n_nodes", C.c_int64)] + [(k, C.c_void_p) for k in (
        "mean", "scale", "rot", "opacity", "sh", "box_min", "box_max", "parent", "child_start", "child_count")]


class h3dgs_node_arrays(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in (
        "mean", "scale", "rot", "opacity", "sh", "box_min", "box_max", "parent", "child_start", "child_count")]


class h3dgs_grads(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("mean", "scale", "rot", "opacity", "sh")]


class h3dgs_render_opts(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("lowpass", C.c_float),
                ("alpha_clamp", C.c_float), ("alpha_floor", C.c_float), ("t_min", C.c_float),
                ("aa_compensate", C.c_int32), ("interpolate", C.c_int32), ("bg", C.c_float * 3),
                ("blend_chunk", C.c_int32)]


class h3dgs_stats(C.Structure):
    _fields_ = [("n_cut", C.c_int64), ("n_visible", C.c_int64), ("n_pairs", C.c_int64),
                ("n_tiles", C.c_int64), ("n_pixels", C.c_int64), ("device_flags", C.c_uint32),
                ("n_evals", C.c_int64), ("n_evals_tpass", C.c_int64), ("n_items", C.c_int64),
                ("n_evals_interp", C.c_int64), ("n_contrib", C.c_int64),
                ("n_contrib_interp", C.c_int64), ("n_cut_visited", C.c_int64)]


STAGES = ["cut", "preprocess", "depth_sort", "duplicate", "tile_sort", "ranges", "blend", "backward_blend",
          "backward_splat", "blend_queue"]


_lib = None


def lib():
    """Load libh3dgs.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} missing: build it with `python -m paper_2406_12080_b300.build`")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        sig = {
            "h3dgs_create": (i32, [C.POINTER(vp), i32, vp]),
            "h3dgs_destroy": (i32, [vp]),
            "h3dgs_last_error": (C.c_char_p, [vp]),
            "h3dgs_default_opts": (None, [C.POINTER(h3dgs_render_opts)]),
            "h3dgs_reserve": (i32, [vp, i64, i64]),
            "h3dgs_upload_hierarchy": (i32, [vp, C.POINTER(h3dgs_hierarchy)]),
            "h3dgs_upload_hierarchy_streamed": (i32, [vp, C.POINTER(h3dgs_hierarchy), i64]),
            "h3dgs_stream_update": (i32, [vp, i32, vp, vp, vp, i32, C.POINTER(i64)]),
            "h3dgs_stream_cleanup": (i32, [vp, i32, i32, C.POINTER(i64)]),
            "h3dgs_build_hierarchy": (i32, [vp, i64, vp, vp, vp, vp, vp, C.POINTER(h3dgs_node_arrays)]),
            "h3dgs_build_hierarchy_chunked": (i32, [vp, i32, C.POINTER(C.c_int64), vp, vp, vp, vp, vp,
                                                    C.POINTER(h3dgs_node_arrays)]),
            "h3dgs_compact_hierarchy": (i32, [vp, C.POINTER(h3dgs_camera), i32, C.c_float, C.c_float,
                                              C.POINTER(h3dgs_node_arrays), i64, vp, C.POINTER(i64)]),
            "h3dgs_select_cut": (i32, [vp, C.POINTER(h3dgs_camera), i32, vp, vp, vp, i64, C.POINTER(i64)]),
            "h3dgs_interpolate": (i32, [vp, C.POINTER(h3dgs_camera), i32, vp, vp, vp, i32, vp, i64]),
            "h3dgs_select_cut_noalloc": (i32, [C.POINTER(h3dgs_hierarchy), C.POINTER(h3dgs_camera), vp, vp, vp, i64,
                                               C.POINTER(i64), vp]),
            "h3dgs_render": (i32, [vp, C.POINTER(h3dgs_camera), i32, vp, vp, vp, C.POINTER(h3dgs_render_opts), vp, i32]),
            "h3dgs_render_backward": (i32, [vp, vp, C.POINTER(h3dgs_grads), i32]),
            "h3dgs_render_ex": (i32, [vp, C.POINTER(h3dgs_camera), i32, vp, vp, vp, C.POINTER(h3dgs_render_opts), vp,
                                      vp, vp, i32]),
            "h3dgs_render_backward_ex": (i32, [vp, vp, vp, C.POINTER(h3dgs_grads), i32]),
            "h3dgs_get_stats": (i32, [vp, C.POINTER(h3dgs_stats)]),
            "h3dgs_measure_peaks": (i32, [vp, C.POINTER(C.c_float), C.POINTER(C.c_float)]),
            "h3dgs_set_profiling": (i32, [vp, i32]),
            "h3dgs_debug_wait_timeout": (i32, [vp, i32]),
            "h3dgs_get_stage_times": (i32, [vp, vp]),
            "h3dgs_debug_tile_lists": (i32, [vp, i32, vp, vp, i64, C.POINTER(i64)]),
            "h3dgs_debug_splats": (i32, [vp, vp, vp, vp, i64]),
            "h3dgs_debug_pixel_state": (i32, [vp, vp, vp, i64]),
            "h3dgs_build_flags": (i32, []),
            "h3dgs_set_cut_mode": (i32, [vp, i32]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def header_symbols() -> list[str]:
    """Entry points declared in include/h3dgs.h."""
    txt = open(HEADER_PATH).read()
    pat = r"^(?:const\s+)?(?:h3dgs_status|void|char|int32_t|int64_t)\s*\**\s*(h3dgs_\w+)\s*\("
    return sorted(set(re.findall(pat, txt, re.M)))


# ----------------------------------------------------------------------------- marshalling

def _ptr(t) -> int | None:
    return None if t is None else int(t.data_ptr())


def camera_struct(cam) -> h3dgs_camera:
    c = h3dgs_camera()
    c.R = (C.c_float * 9)(*np.asarray(cam.R, np.float32).reshape(-1).tolist())
    c.T = (C.c_float * 3)(*np.asarray(cam.T, np.float32).reshape(-1).tolist())
    c.fx, c.fy, c.cx, c.cy = cam.fx, cam.fy, cam.cx, cam.cy
    c.width, c.height, c.znear, c.tau = cam.width, cam.height, cam.znear, cam.tau
    return c


def camera_array(cams):
    arr = (h3dgs_camera * len(cams))()
    for i, c in enumerate(cams):
        arr[i] = camera_struct(c)
    return arr


def default_opts(**kw) -> h3dgs_render_opts:
    o = h3dgs_render_opts()
    lib().h3dgs_default_opts(C.byref(o))
    for k, v in kw.items():
        if k == "bg":
            o.bg = (C.c_float * 3)(*v)
        else:
            setattr(o, k, v)
    return o


# ----------------------------------------------------------------------------- C entry points

def h3dgs_last_error(ctx) -> str:
    """The context's last error message ("" if none)."""
    return lib().h3dgs_last_error(ctx).decode() if ctx else ""


def h3dgs_set_cut_mode(ctx, mode: int):
    """0 (default) and 1: the scan of every node's record; 2: the root-down traversal."""
    _check(ctx, lib().h3dgs_set_cut_mode(ctx, mode))


def h3dgs_build_flags() -> int:
    """H3DGS_BUILD_CHECKED (1) for the bounds-checked debug build, else 0."""
    return int(lib().h3dgs_build_flags())


def _check(ctx, status):
    if status != H3DGS_OK:
        msg = lib().h3dgs_last_error(ctx).decode() if ctx else ""
        raise H3dgsError(status, msg)


def h3dgs_create(device: int = 0, stream: int | None = None):
    out = C.c_void_p()
    st = lib().h3dgs_create(C.byref(out), device, stream)
    if st != H3DGS_OK:
        raise H3dgsError(st, "h3dgs_create failed")
    return out


def h3dgs_destroy(ctx):
    _check(None, lib().h3dgs_destroy(ctx))


def h3dgs_reserve(ctx, max_splats: int, max_pairs: int):
    _check(ctx, lib().h3dgs_reserve(ctx, max_splats, max_pairs))


def h3dgs_upload_hierarchy(ctx, hier: "DeviceHierarchy"):
    h = h3dgs_hierarchy()
    h.n_nodes = hier.n
    for k in ("mean", "scale", "rot", "opacity", "sh", "box_min", "box_max", "parent", "child_start",
              "child_count"):
        setattr(h, k, _ptr(getattr(hier, k)))
    _check(ctx, lib().h3dgs_upload_hierarchy(ctx, C.byref(h)))


def h3dgs_build_hierarchy(ctx, leaves: dict, out: "DeviceHierarchy"):
    """leaves: dict of device tensors mean [L,3], scale [L,3], rot [L,4], opacity [L], sh [L,48]."""
    a = h3dgs_node_arrays()
    for k in ("mean", "scale", "rot", "opacity", "sh", "box_min", "box_max", "parent", "child_start",
              "child_count"):
        setattr(a, k, _ptr(getattr(out, k)))
    L = int(leaves["mean"].shape[0])
    _check(ctx, lib().h3dgs_build_hierarchy(ctx, L, *[_ptr(leaves[k]) for k in ("mean", "scale", "rot", "opacity", "sh")],
                                            C.byref(a)))


def h3dgs_compact_hierarchy(ctx, cams, tau_min: float, tau_max: float, out: "DeviceHierarchy", old_index=None) -> int:
    """Compacts the resident hierarchy into `out` (capacity = out.n); returns the kept node count."""
    a = h3dgs_node_arrays()
    for k in ("mean", "scale", "rot", "opacity", "sh", "box_min", "box_max", "parent", "child_start",
              "child_count"):
        setattr(a, k, _ptr(getattr(out, k)))
    n = C.c_int64(0)
    _check(ctx, lib().h3dgs_compact_hierarchy(ctx, camera_array(cams), len(cams), tau_min, tau_max, C.byref(a),
                                              out.n, _ptr(old_index), C.byref(n)))
    return n.value


def h3dgs_upload_hierarchy_streamed(ctx, hier: "DeviceHierarchy", cache_nodes: int):
    """hier: attributes as page-locked CPU tensors, boxes and topology as CUDA tensors."""
    h = h3dgs_hierarchy()
    h.n_nodes = hier.n
    for k in ("mean", "scale", "rot", "opacity", "sh", "box_min", "box_max", "parent", "child_start",
              "child_count"):
        setattr(h, k, _ptr(getattr(hier, k)))
    _check(ctx, lib().h3dgs_upload_hierarchy_streamed(ctx, C.byref(h), cache_nodes))


def h3dgs_stream_update(ctx, n_cams: int, cut_ids, cut_t, cut_offsets, frame: int, want_count: bool = True):
    n = C.c_int64(0)
    _check(ctx, lib().h3dgs_stream_update(ctx, n_cams, _ptr(cut_ids), _ptr(cut_t), _ptr(cut_offsets), frame,
                                          C.byref(n) if want_count else None))
    return n.value if want_count else None


def h3dgs_stream_cleanup(ctx, frame: int, max_age: int, want_count: bool = True):
    n = C.c_int64(0)
    _check(ctx, lib().h3dgs_stream_cleanup(ctx, frame, max_age, C.byref(n) if want_count else None))
    return n.value if want_count else None


def h3dgs_build_hierarchy_chunked(ctx, leaves: dict, chunk_offsets, out: "DeviceHierarchy"):
    """Consolidated hierarchy over chunks; chunk_offsets: n_chunks + 1 ascending leaf offsets from 0."""
    a = h3dgs_node_arrays()
    for k in ("mean", "scale", "rot", "opacity", "sh", "box_min", "box_max", "parent", "child_start",
              "child_count"):
        setattr(a, k, _ptr(getattr(out, k)))
    off = np.ascontiguousarray(chunk_offsets, np.int64)
    _check(ctx, lib().h3dgs_build_hierarchy_chunked(ctx, len(off) - 1, off.ctypes.data_as(C.POINTER(C.c_int64)),
                                                    *[_ptr(leaves[k]) for k in ("mean", "scale", "rot", "opacity",
                                                                                 "sh")], C.byref(a)))


def h3dgs_select_cut(ctx, cams, cut_ids, cut_t, cut_offsets, capacity: int, want_total: bool = True):
    arr = camera_array(cams)
    tot = C.c_int64(-1)
    st = lib().h3dgs_select_cut(ctx, arr, len(cams), _ptr(cut_ids), _ptr(cut_t), _ptr(cut_offsets), capacity,
                                C.byref(tot) if want_total else None)
    _check(ctx, st)
    return int(tot.value) if want_total else None


def h3dgs_select_cut_noalloc(hier: "DeviceHierarchy", cam, cut_ids, cut_t, cut_offsets, capacity: int,
                             stream: int | None = None, want_total: bool = True, n_nodes: int | None = None):
    """One camera's cut with no allocation anywhere (scratch in a fixed device array of the library).

    For callers that cannot allocate device memory; see include/h3dgs.h.  Returns the cut size
    (synchronising) when want_total, else None.  n_nodes overrides the node count (tests only).
    """
    h = h3dgs_hierarchy()
    h.n_nodes = hier.n if n_nodes is None else n_nodes
    for k in ("mean", "scale", "rot", "opacity", "sh", "box_min", "box_max", "parent", "child_start",
              "child_count"):
        setattr(h, k, _ptr(getattr(hier, k)))
    tot = C.c_int64(-1)
    st = lib().h3dgs_select_cut_noalloc(C.byref(h), C.byref(camera_struct(cam)), _ptr(cut_ids), _ptr(cut_t),
                                        _ptr(cut_offsets), capacity, C.byref(tot) if want_total else None, stream)
    if st != H3DGS_OK:
        raise H3dgsError(st, "h3dgs_select_cut_noalloc failed",
                         int(tot.value) if want_total and tot.value >= 0 else None)
    return int(tot.value) if want_total else None


def h3dgs_interpolate(ctx, cams, cut_ids, cut_t, cut_offsets, interpolate: int, out, m_total: int):
    arr = camera_array(cams)
    _check(ctx, lib().h3dgs_interpolate(ctx, arr, len(cams), _ptr(cut_ids), _ptr(cut_t), _ptr(cut_offsets),
                                        interpolate, _ptr(out), m_total))


def h3dgs_render(ctx, cams, cut_ids, cut_t, cut_offsets, opts: h3dgs_render_opts, images, save_for_backward: int = 0,
                 cam_array=None):
    arr = cam_array if cam_array is not None else camera_array(cams)
    _check(ctx, lib().h3dgs_render(ctx, arr, len(cams), _ptr(cut_ids), _ptr(cut_t), _ptr(cut_offsets),
                                   C.byref(opts), _ptr(images), save_for_backward))


def h3dgs_render_backward(ctx, dL_dimages, grads: dict, freeze_leaves: int = 0):
    g = h3dgs_grads()
    for k in ("mean", "scale", "rot", "opacity", "sh"):
        setattr(g, k, _ptr(grads[k]))
    _check(ctx, lib().h3dgs_render_backward(ctx, _ptr(dL_dimages), C.byref(g), freeze_leaves))


def h3dgs_render_ex(ctx, cams, cut_ids, cut_t, cut_offsets, opts: h3dgs_render_opts, images, depth=None,
                    exposure=None, save_for_backward: int = 0, cam_array=None):
    """depth: device [sum H_k W_k] or None; exposure: device [n_cams, 3, 4] or None."""
    arr = cam_array if cam_array is not None else camera_array(cams)
    _check(ctx, lib().h3dgs_render_ex(ctx, arr, len(cams), _ptr(cut_ids), _ptr(cut_t), _ptr(cut_offsets),
                                      C.byref(opts), _ptr(images), _ptr(depth), _ptr(exposure), save_for_backward))


def h3dgs_render_backward_ex(ctx, dL_dimages, dL_ddepth, grads: dict, freeze_leaves: int = 0):
    g = h3dgs_grads()
    for k in ("mean", "scale", "rot", "opacity", "sh"):
        setattr(g, k, _ptr(grads[k]))
    _check(ctx, lib().h3dgs_render_backward_ex(ctx, _ptr(dL_dimages), _ptr(dL_ddepth), C.byref(g), freeze_leaves))


def h3dgs_get_stats(ctx) -> dict:
    s = h3dgs_stats()
    _check(ctx, lib().h3dgs_get_stats(ctx, C.byref(s)))
    return {k: getattr(s, k) for k, _ in h3dgs_stats._fields_}


def h3dgs_measure_peaks(ctx) -> dict:
    """Measured fp32 (paired FFMA) TFLOP/s and exp2 Gop/s of this GPU."""
    f, x = C.c_float(0), C.c_float(0)
    _check(ctx, lib().h3dgs_measure_peaks(ctx, C.byref(f), C.byref(x)))
    return {"fp32_tflops": f.value, "ex2_gops": x.value}


def h3dgs_debug_wait_timeout(ctx, polls: int):
    _check(ctx, lib().h3dgs_debug_wait_timeout(ctx, polls))


def h3dgs_set_profiling(ctx, enable: int):
    _check(ctx, lib().h3dgs_set_profiling(ctx, enable))


def h3dgs_get_stage_times(ctx) -> dict:
    ms = np.zeros(len(STAGES), np.float32)
    _check(ctx, lib().h3dgs_get_stage_times(ctx, ms.ctypes.data))
    return dict(zip(STAGES, ms.tolist()))


def h3dgs_debug_tile_lists(ctx, cam: int, n_tiles: int):
    ranges = np.zeros((n_tiles, 2), np.int32)
    n = C.c_int64(0)
    st = lib().h3dgs_debug_tile_lists(ctx, cam, ranges.ctypes.data, None, 0, C.byref(n))
    if st not in (H3DGS_OK, 4):
        _check(ctx, st)
    ids = np.zeros(max(1, n.value), np.int32)
    _check(ctx, lib().h3dgs_debug_tile_lists(ctx, cam, ranges.ctypes.data, ids.ctypes.data, ids.size, C.byref(n)))
    return ranges, ids[:n.value]


def h3dgs_debug_splats(ctx, m: int):
    rec = np.zeros((m, 10), np.float32)
    rect = np.zeros((m, 4), np.int32)
    rgb = np.zeros((m, 3), np.float32)
    _check(ctx, lib().h3dgs_debug_splats(ctx, rec.ctypes.data, rect.ctypes.data, rgb.ctypes.data, m))
    return rec, rect, rgb


def h3dgs_debug_pixel_state(ctx, n_pixels: int):
    T = np.zeros(n_pixels, np.float32)
    nc = np.zeros(n_pixels, np.int32)
    _check(ctx, lib().h3dgs_debug_pixel_state(ctx, T.ctypes.data, nc.ctypes.data, n_pixels))
    return T, nc


# ----------------------------------------------------------------------------- torch-side helpers

@dataclass
class DeviceHierarchy:
    """Node arrays as torch CUDA tensors (the layouts of h3dgs_hierarchy)."""
    mean: object
    scale: object
    rot: object
    opacity: object
    sh: object
    box_min: object
    box_max: object
    parent: object
    child_start: object
    child_count: object

    @property
    def n(self) -> int:
        return int(self.mean.shape[0])

    @staticmethod
    def from_arrays(h, device="cuda") -> "DeviceHierarchy":
        import torch
        f = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(device)
        i = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.int32)).to(device)
        return DeviceHierarchy(f(h.mean), f(h.scale), f(h.rot), f(h.opacity), f(h.sh), f(h.box_min),
                               f(h.box_max), i(h.parent), i(h.child_start), i(h.child_count))


class Context:
    """One library context on the current torch device and stream."""

    def __init__(self, device: int | None = None, stream=None):
        import torch
        self.device = torch.cuda.current_device() if device is None else device
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.ctx = h3dgs_create(self.device, self.stream.cuda_stream)
        self.hier = None

    def close(self):
        if self.ctx:
            h3dgs_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build(self, leaves) -> DeviceHierarchy:
        """Build a hierarchy on the device from leaf Gaussians (synth.Leaves or dict of tensors)."""
        import torch
        if not isinstance(leaves, dict):
            leaves = {k: torch.from_numpy(np.ascontiguousarray(getattr(leaves, k), np.float32)).to(self.device)
                      for k in ("mean", "scale", "rot", "opacity", "sh")}
        L = int(leaves["mean"].shape[0])
        N = 2 * L - 1
        f = lambda *shape: torch.empty(shape, dtype=torch.float32, device=self.device)
        i = lambda n: torch.empty(n, dtype=torch.int32, device=self.device)
        out = DeviceHierarchy(f(N, 3), f(N, 3), f(N, 4), f(N), f(N, 48), f(N, 3), f(N, 3), i(N), i(N), i(N))
        h3dgs_build_hierarchy(self.ctx, leaves, out)
        return out

    def build_chunked(self, leaves: dict, chunk_offsets) -> DeviceHierarchy:
        """Consolidated hierarchy over chunks (leaves: dict of device tensors, chunks contiguous)."""
        import torch
        L = int(leaves["mean"].shape[0])
        N = 2 * L - 1
        f = lambda *shape: torch.empty(shape, dtype=torch.float32, device=self.device)
        i = lambda n: torch.empty(n, dtype=torch.int32, device=self.device)
        out = DeviceHierarchy(f(N, 3), f(N, 3), f(N, 4), f(N), f(N, 48), f(N, 3), f(N, 3), i(N), i(N), i(N))
        h3dgs_build_hierarchy_chunked(self.ctx, leaves, chunk_offsets, out)
        return out

    def compact(self, cams, tau_min: float, tau_max: float):
        """Compacted copy of the resident hierarchy (Sec. 5.2) for the training cameras `cams`.
        Returns (DeviceHierarchy, old index of every new node)."""
        import torch
        N = self.hier.n
        f = lambda *shape: torch.empty(shape, dtype=torch.float32, device=self.device)
        i = lambda n: torch.empty(n, dtype=torch.int32, device=self.device)
        out = DeviceHierarchy(f(N, 3), f(N, 3), f(N, 4), f(N), f(N, 48), f(N, 3), f(N, 3), i(N), i(N), i(N))
        old = i(N)
        m = h3dgs_compact_hierarchy(self.ctx, cams, tau_min, tau_max, out, old)
        trim = DeviceHierarchy(*[getattr(out, k)[:m] for k in ("mean", "scale", "rot", "opacity", "sh", "box_min",
                                                             "box_max", "parent", "child_start", "child_count")])
        return trim, old[:m]

    def upload_streamed(self, hier: DeviceHierarchy, cache_nodes: int) -> DeviceHierarchy:
        """Streamed hierarchy: `hier`'s attributes are moved to page-locked host memory (the boxes and
        topology stay on the device); returns the hierarchy as the library now borrows it."""
        import torch
        host = lambda t: t.detach().to("cpu").contiguous().pin_memory()
        h = DeviceHierarchy(host(hier.mean), host(hier.scale), host(hier.rot), host(hier.opacity), host(hier.sh),
                            hier.box_min, hier.box_max, hier.parent, hier.child_start, hier.child_count)
        torch.cuda.synchronize()
        h3dgs_upload_hierarchy_streamed(self.ctx, h, cache_nodes)
        self.hier = h
        return h

    def upload(self, hier: DeviceHierarchy):
        h3dgs_upload_hierarchy(self.ctx, hier)
        self.hier = hier

    def select_cut(self, cams, capacity: int | None = None):
        """Returns (cut_ids int32, cut_t f32, cut_offsets int64) device tensors, trimmed."""
        import torch
        cap = capacity if capacity is not None else self.hier.n * len(cams)
        ids = torch.empty(max(cap, 1), dtype=torch.int32, device=self.device)
        t = torch.empty(max(cap, 1), dtype=torch.float32, device=self.device)
        offs = torch.empty(len(cams) + 1, dtype=torch.int64, device=self.device)
        tot = h3dgs_select_cut(self.ctx, cams, ids, t, offs, cap)
        return ids[:tot], t[:tot], offs

    def render(self, cams, cut, opts=None, save_for_backward=0, images=None, depth=False, exposure=None):
        """Packed images; with depth=True (or a depth tensor) returns (images, depth).  exposure: device
        tensor [n_cams, 3, 4] of per-camera affines applied to the colour."""
        import torch
        opts = opts or default_opts()
        npix = sum(3 * c.width * c.height for c in cams)
        if images is None:
            images = torch.empty(npix, dtype=torch.float32, device=self.device)
        ids, t, offs = cut
        if depth is False and exposure is None:
            h3dgs_render(self.ctx, cams, ids, t, offs, opts, images, save_for_backward)
            return images
        d = depth if depth is not False and depth is not True else None
        if depth is True:
            d = torch.empty(npix // 3, dtype=torch.float32, device=self.device)
        h3dgs_render_ex(self.ctx, cams, ids, t, offs, opts, images, d, exposure, save_for_backward)
        return (images, d) if depth is not False else images

    def split_images(self, images, cams):
        out, o = [], 0
        for c in cams:
            n = 3 * c.width * c.height
            out.append(images[o:o + n].view(3, c.height, c.width))
            o += n
        return out
