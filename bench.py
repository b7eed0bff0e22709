#!/usr/bin/env python3
"""Benchmark of the hierarchical 3D Gaussian render path on one B300 per rank.

Workload: the street corridor (1M leaf Gaussians, ~2M hierarchy nodes) seen by one 1920x1080
camera at tau = 6 px.  One step = one frame of the hot path through the C ABI: cut selection with
interpolation weights, then interpolate + project + SH, depth sort, binning, tile sort, ranges and
blend.  The hierarchy is built on the device by the library and stays resident (like the paper's
GPU-resident nodes).  The frame is captured once in a CUDA graph and replayed; L2 is flushed
(256 MB write) between timed steps, outside the timed events.

Also reported in the same JSON line: fwd+bwd views/s (frame + adjoint), the end-to-end rate with
the image read back to pinned host memory every step, per-stage times, the roofline fraction of
the dominant kernel, the SM clocks during the timed region, and the CPU oracle timed on the host
cores (cpu_baseline).  `--impl reference` times the CPU oracle alone (the deliberately slow
reference program of this repository).

Multi-GPU: `torchrun --nproc-per-node N bench.py --gpus N`: every rank renders its own replica of
the workload (views are independent, no collective on the data path); value = frames of all
ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "1080p frames/s (cut+render) & fwd+bwd views/s; % of HBM/FP32 roofline"
L2_FLUSH_BYTES = 256 << 20
REF_BUDGET_S = 120.0
# Algorithmic work of the blend and its adjoint: the op lists of the oracle's blend_pixel / alpha_f
# and of its reverse walk in or_backward (Sec. 3.1 Eq. alpha; Eq. alphap), in their step order, counting
# every fp32 add, subtract, multiply and divide as one flop and a fused multiply-add as two; compares,
# min/max and selects are not flops, exp2 / log2 / sqrt / reciprocal are XU results.
#   per evaluated (pixel, splat) pair: dx, dy (2); h = ca dx + cb dy (3); g = (cc dy) dy (2);
#     p2 = dx h + g (2); o_n G (1)                                         -> 10 flops, 1 XU (exp2)
#   + t != 0: o_p G (1); 1 - alpha_p, (.)^(1/K) as exp2(log2(.) / K), 1 - (.) (3); 1 - t, (1 - t) alpha_n,
#     t alpha' + (.) (4)                                                   -> +8 flops, +2 XU
#   + per contribution (the pair's colour is accumulated): T (1 - alpha) (2), alpha T (1), 3 colour FMAs (6)
#                                                                          -> +9 flops
BLEND_FLOPS_EVAL, BLEND_FLOPS_INTERP, BLEND_FLOPS_CONTRIB = 10, 8, 9
BLEND_XU_EVAL, BLEND_XU_INTERP = 1, 2
#   adjoint, per contributing pair (reverse walk, colour only): colour gradients a T g_c (9); alpha adjoint
#     sum_c g_c (T c_c - S_c / (1 - alpha)) (18); colour behind S_c += c_c a T (9); dx, dy and the exponent
#     (11); o_n G and its adjoint terms (5); exponent adjoint dG G and the conic and centre terms (22)
#                                                                          -> 74 flops, 1 XU
#     + t != 0: (1 - t) alpha adjoint (2); o_p G, d alpha'/d alpha_p = (1/K)(1 - alpha_p)^(1/K - 1), its
#     product with t and the adjoint, o_p and G terms (12)                  -> +14 flops, +2 XU
#   plus the recomputation of the pair's alpha (the adjoint keeps no per-pair state): the evaluation
#   op list above, counted for contributing pairs only
ADJ_FLOPS_CONTRIB, ADJ_FLOPS_CONTRIB_INTERP = 74 + BLEND_FLOPS_EVAL, 14 + BLEND_FLOPS_INTERP
# DRAM bytes (read + write) of one launch of the blend's main kernel at the 1080p corridor frame
# (16x16 tiles, the automatic chunk: 320 at this frame), from an ncu capture of the current kernel; None once
# the kernel changes
BLEND_TRAFFIC_BYTES = 30.91e6 + 6.05e6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n-leaves", type=int, default=1_000_000)
    ap.add_argument("--tau", type=float, default=6.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--chunk", type=int, default=0, help="blend chunk (list entries per CTA; 0: automatic)")
    ap.add_argument("--tile", default="16x16", help="screen tile WxH")
    ap.add_argument("--batch-views", type=int, default=32, help="cameras of the batched multi-view section (0: skip)")
    ap.add_argument("--opt-leaves", type=int, default=2_000_000,
                    help="leaves of the hierarchy-optimisation section (0: skip)")
    ap.add_argument("--opt-steps", type=int, default=20)
    ap.add_argument("--compact-views", type=int, default=256,
                    help="training views of the hierarchy-compaction section (0: skip)")
    ap.add_argument("--stream-frames", type=int, default=256,
                    help="frames of the streamed (out-of-core) camera path section (0: skip)")
    ap.add_argument("--workload", choices=["corridor", "city"], default="corridor",
                    help="corridor: 1M-leaf street corridor, one 1080p view; city: 50M-leaf chunked city, "
                         "256-pose loop (and the batched views on it)")
    ap.add_argument("--city-leaves", type=int, default=50_000_000)
    ap.add_argument("--city-grid", type=int, default=20, help="chunks per side (50 m each)")
    ap.add_argument("--city-poses", type=int, default=256)
    return ap.parse_args()


def rank_max(x, world, dev):
    """The largest value of x over the ranks (x itself on one rank): a timing of the whole job."""
    if world == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def rank_barrier(world):
    if world > 1:
        import torch
        torch.distributed.barrier()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ----------------------------------------------------------------------------------- clocks

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        # the sampled clock log (kept beside the run's other outputs when H3DGS_BENCH_LOG_DIR names a
        # directory, else in the system's temporary directory)
        import tempfile
        log_dir = os.environ.get("H3DGS_BENCH_LOG_DIR") or tempfile.gettempdir()
        self.path = os.path.join(log_dir, f"h3dgs_clocks_gpu{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            if os.path.exists(self.path):
                os.remove(self.path)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.send_signal(2)
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines()]
        except Exception:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ----------------------------------------------------------------------------------- CPU oracle

def cpu_oracle_time(scene, n_frames: int, budget_s: float = 25.0):
    """Time the CPU oracle (cut + render of the full frame) on the host cores."""
    import oracle
    h = oracle.build_tree(scene.leaves)   # offline build, not timed
    cam = scene.cameras[0]
    times = []
    t_start = time.perf_counter()
    amb = None
    for _ in range(max(1, n_frames)):
        t0 = time.perf_counter()
        fr = oracle.render(cam, h, oracle.Opts())
        times.append(time.perf_counter() - t0)
        amb = float(fr.ambiguous.mean())
        if time.perf_counter() - t_start > budget_s:
            break
    return {"value": len(times) / float(np.sum(times)), "unit": "frames/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{len(times)} full 1920x1080 frames (cut + interpolate/project/SH + tile lists + blend), "
                      f"fp64 values with fp32 decisions, OpenMP",
            "ambiguous_pixel_fraction": amb,
            "ambiguous_note": "pixels of this frame whose fp32 alpha-floor or stop decision lies within 1e-5 "
                              "(relative) of its threshold: excluded from the image parity bar (allowed: 2e-4)"}


# ----------------------------------------------------------------------------------- our path

def launches_per_frame(n_tiles: int) -> int:
    """Kernels of one frame, from the pipeline's launch sites (used when the graph cannot be read)."""
    tile_bits = max(1, int(np.ceil(np.log2(max(n_tiles, 2)))))
    cut = 1                           # one-camera cut (single pass, camera derived in the kernel)
    render = (1 + 1                   # camera set-up, preprocess (also counts the depth-key digits)
              + 4                     # depth sort: 4 onesweep passes
              + 1 + 1                 # pair-offset scan, duplicate (also counts the tile-key digits)
              + (tile_bits + 7) // 8  # tile sort passes
              + 1                     # ranges
              + 3)                    # blend: plan, queue, combine
    return cut + render


def graph_kernel_count(fn, stream):
    """Number of kernel nodes in a CUDA graph captured from fn() (the launches of one step)."""
    import torch
    from cuda.bindings import runtime as rt
    g = torch.cuda.CUDAGraph(keep_graph=True)
    with torch.cuda.graph(g, stream=stream):
        fn()
    raw = rt.cudaGraph_t(init_value=g.raw_cuda_graph())
    err, _, n = rt.cudaGraphGetNodes(raw, 0)
    assert err == rt.cudaError_t.cudaSuccess, err
    err, nodes, n = rt.cudaGraphGetNodes(raw, n)
    assert err == rt.cudaError_t.cudaSuccess, err
    kern = 0
    for nd in nodes[:n]:
        err, ty = rt.cudaGraphNodeGetType(nd)
        assert err == rt.cudaError_t.cudaSuccess, err
        kern += int(ty == rt.cudaGraphNodeType.cudaGraphNodeTypeKernel)
    del g
    return kern


def run_ours(args, rank, world, local):
    import torch
    from paper_2406_12080_b300 import build, h3dgs, synth
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.Stream(dev)
    scene = synth.corridor_scene(n_leaves=args.n_leaves, tau=args.tau)
    cam = scene.cameras[0]
    cams = [cam]
    ctx = h3dgs.Context(local, stream)
    with torch.cuda.stream(stream):
        hier = ctx.build(scene.leaves)
        ctx.upload(hier)
        N = hier.n
        cap = N
        ids = torch.empty(cap, dtype=torch.int32, device=dev)
        tt = torch.empty(cap, dtype=torch.float32, device=dev)
        offs = torch.empty(2, dtype=torch.int64, device=dev)
        npix = 3 * cam.width * cam.height
        images = torch.empty(npix, dtype=torch.float32, device=dev)
        tw, th = (int(x) for x in args.tile.split("x"))
        opts = h3dgs.default_opts(blend_chunk=args.chunk, tile_w=tw, tile_h=th)
        carr = h3dgs.camera_array(cams)
        calib = h3dgs.h3dgs_measure_peaks(ctx.ctx)   # roofline denominators measured on this GPU
        # first frame in the growing mode, to size the fixed workspace
        m = h3dgs.h3dgs_select_cut(ctx.ctx, cams, ids, tt, offs, cap)
        h3dgs.h3dgs_render(ctx.ctx, cams, ids, tt, offs, opts, images, 0)
        st = h3dgs.h3dgs_get_stats(ctx.ctx)
        h3dgs.h3dgs_reserve(ctx.ctx, int(m * 1.25) + 1024, int(st["n_pairs"] * 1.25) + 4096)

        def frame():
            h3dgs.h3dgs_select_cut(ctx.ctx, cams, ids, tt, offs, cap, want_total=False)
            h3dgs.h3dgs_render(ctx.ctx, cams, ids, tt, offs, opts, images, 0, cam_array=carr)

        frame()
        ref_img = images.clone()
        graph = None
        if not args.no_graph:
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=stream):
                frame()
            graph.replay()
            stream.synchronize()
            assert torch.equal(images, ref_img), "graph replay differs from the direct frame"
        run = graph.replay if graph is not None else frame
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        with ClockSampler(local) as clk:
            for _ in range(args.warmup):
                run()
                flush.fill_(1.0)
            stream.synchronize()
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()
            for e0, e1 in evs:
                e0.record(stream)
                run()
                e1.record(stream)
                flush.fill_(1.0)
            torch.cuda.synchronize()
        step_ms = [a.elapsed_time(b) for a, b in evs]
        total_ms = float(np.sum(step_ms))
        if world > 1:
            t = torch.tensor([total_ms], device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            total_ms = float(t.item())
            torch.distributed.barrier()
        st = h3dgs.h3dgs_get_stats(ctx.ctx)
        assert st["device_flags"] == 0, f"device flags {st['device_flags']}"
        M_cut = int(st["n_cut"])
        value = world * args.steps / (total_ms / 1e3)
        try:
            launches = graph_kernel_count(frame, stream)
            launch_src = "kernel nodes of the captured frame graph"
        except Exception as e:   # noqa: BLE001 - fall back to the launch-site count
            launches = launches_per_frame(int(st["n_tiles"]))
            launch_src = f"launch sites ({type(e).__name__})"

        # ---- evaluation counts (profiling level 2), then per-stage times (level 1: events inside the
        # library around the same ABI calls, not graphed)
        h3dgs.h3dgs_set_profiling(ctx.ctx, 2)
        frame()
        st_counts = h3dgs.h3dgs_get_stats(ctx.ctx)
        h3dgs.h3dgs_set_profiling(ctx.ctx, 1)
        stage_acc = {}
        n_prof = max(3, min(args.steps, 20))
        for _ in range(n_prof):
            frame()
            times = h3dgs.h3dgs_get_stage_times(ctx.ctx)
            for k, v in times.items():
                stage_acc[k] = stage_acc.get(k, 0.0) + v
            flush.fill_(1.0)
        fwd_stages = {k: v / n_prof for k, v in stage_acc.items() if v > 0}
        st = dict(h3dgs.h3dgs_get_stats(ctx.ctx))
        st["n_evals"], st["n_evals_tpass"] = st_counts["n_evals"], st_counts["n_evals_tpass"]
        for k in ("n_evals_interp", "n_contrib", "n_contrib_interp"):
            st[k] = st_counts[k]
        # the root-down traversal of the same frame: the records it reads and its time (the frame uses the scan)
        h3dgs.h3dgs_set_cut_mode(ctx.ctx, 2)
        h3dgs.h3dgs_select_cut(ctx.ctx, cams, ids, tt, offs, cap)   # sizes its buffers
        trav_acc = []
        for _ in range(n_prof):
            h3dgs.h3dgs_select_cut(ctx.ctx, cams, ids, tt, offs, cap, want_total=False)
            trav_acc.append(h3dgs.h3dgs_get_stage_times(ctx.ctx)["cut"])
            flush.fill_(1.0)
        st_counts["n_cut_visited_traversal"] = int(h3dgs.h3dgs_get_stats(ctx.ctx)["n_cut_visited"])
        st_counts["traversal_ms"] = float(np.mean(trav_acc))
        h3dgs.h3dgs_set_cut_mode(ctx.ctx, 0)
        # visible splats with an interpolated parent (the adjoint's splat stage reads the parent's row too)
        rec_dbg, rect_dbg, _ = h3dgs.h3dgs_debug_splats(ctx.ctx, int(st["n_cut"]))
        st_counts["n_interp_visible"] = int(np.sum((rect_dbg[:, 0] >= 0) & (rec_dbg[:, 7] != 0)))
        # the frame's entries and the distinct parents the interpolation reads (of all entries with
        # t != 0 for the geometry, of the visible ones for opacity, K and SH)
        m_cut = int(st["n_cut"])
        vis_m = rect_dbg[:m_cut, 0] >= 0
        cut_np = ids[:m_cut].cpu().numpy()
        par_np = hier.parent.cpu().numpy()[cut_np]
        interp_m = (tt[:m_cut].cpu().numpy() != 0) & (par_np >= 0)
        st_counts["n_parents_geom"] = int(np.unique(par_np[interp_m]).size)
        st_counts["n_parents_vis"] = int(np.unique(par_np[interp_m & vis_m]).size)
        del rec_dbg, rect_dbg, cut_np, par_np

        # ---- fwd + bwd views/s
        grads = {k: torch.zeros_like(getattr(hier, k)) for k in ("mean", "scale", "rot", "opacity", "sh")}
        dl = torch.randn(npix, generator=torch.Generator(device=dev).manual_seed(0), device=dev)

        def fwd_bwd():
            h3dgs.h3dgs_select_cut(ctx.ctx, cams, ids, tt, offs, cap, want_total=False)
            h3dgs.h3dgs_render(ctx.ctx, cams, ids, tt, offs, opts, images, 1, cam_array=carr)
            h3dgs.h3dgs_render_backward(ctx.ctx, dl, grads, 1)

        stage_acc = {}
        for _ in range(3):
            fwd_bwd()
            flush.fill_(1.0)
        for _ in range(n_prof):
            fwd_bwd()
            times = h3dgs.h3dgs_get_stage_times(ctx.ctx)
            for k, v in times.items():
                stage_acc[k] = stage_acc.get(k, 0.0) + v
            flush.fill_(1.0)
        bwd_stages = {k: v / n_prof for k, v in stage_acc.items() if k.startswith("backward")}
        h3dgs.h3dgs_set_profiling(ctx.ctx, 0)
        fb_graph = None
        if not args.no_graph:
            fb_graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(fb_graph, stream=stream):
                fwd_bwd()
        fb_run = fb_graph.replay if fb_graph is not None else fwd_bwd
        for _ in range(args.warmup):
            fb_run()
            flush.fill_(1.0)
        torch.cuda.synchronize()
        rank_barrier(world)
        fb_ms = 0.0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(args.steps):
            e0.record(stream)
            fb_run()
            e1.record(stream)
            flush.fill_(1.0)
            e1.synchronize()
            fb_ms += e0.elapsed_time(e1)
        fb_ms = rank_max(fb_ms, world, dev)
        fb_value = world * args.steps / (fb_ms / 1e3)

        # ---- expected-depth output and exposure affine (appendix): forward frame, and forward + adjoint
        # with a depth gradient, both graph-captured like the frames above
        depth_buf = torch.empty(npix // 3, dtype=torch.float32, device=dev)
        expo = torch.tensor([[1.05, 0.02, 0.0, 0.01], [0.0, 0.97, 0.03, 0.0], [0.01, 0.0, 1.02, -0.01]],
                            dtype=torch.float32, device=dev).reshape(1, 3, 4).contiguous()
        ddep = torch.randn(npix // 3, generator=torch.Generator(device=dev).manual_seed(1), device=dev)

        def frame_de():
            h3dgs.h3dgs_select_cut(ctx.ctx, cams, ids, tt, offs, cap, want_total=False)
            h3dgs.h3dgs_render_ex(ctx.ctx, cams, ids, tt, offs, opts, images, depth_buf, expo, 0, cam_array=carr)

        def fwd_bwd_de():
            h3dgs.h3dgs_select_cut(ctx.ctx, cams, ids, tt, offs, cap, want_total=False)
            h3dgs.h3dgs_render_ex(ctx.ctx, cams, ids, tt, offs, opts, images, depth_buf, expo, 1, cam_array=carr)
            h3dgs.h3dgs_render_backward_ex(ctx.ctx, dl, ddep, grads, 1)

        def time_steps(fn):
            fn()
            g = None
            if not args.no_graph:
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=stream):
                    fn()
            r = g.replay if g is not None else fn
            for _ in range(args.warmup):
                r()
                flush.fill_(1.0)
            torch.cuda.synchronize()
            acc = 0.0
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            for _ in range(args.steps):
                a0.record(stream)
                r()
                a1.record(stream)
                flush.fill_(1.0)
                a1.synchronize()
                acc += a0.elapsed_time(a1)
            return acc / args.steps

        de_frame_ms = time_steps(frame_de)
        de_fb_ms = time_steps(fwd_bwd_de)
        assert h3dgs.h3dgs_get_stats(ctx.ctx)["device_flags"] == 0
        depth_exposure = {"frame_ms": de_frame_ms, "frames_per_s": 1e3 / de_frame_ms,
                          "fwd_bwd_ms": de_fb_ms, "fwd_bwd_views_per_s": 1e3 / de_fb_ms,
                          "note": "cut + render with the expected-depth output and a 3x4 exposure affine; the "
                                  "adjoint also takes a depth gradient"}

        # ---- end to end through the public API: every step's image is read back to pinned host memory.
        # Serial: render, then copy.  Pipelined (the headline): two image buffers, the read-back of step k
        # on a copy stream overlaps the cut and render of step k + 1 (what a viewer does).
        host_img = torch.empty(npix, dtype=torch.float32, pin_memory=True)
        for _ in range(args.warmup):
            frame()
            host_img.copy_(images, non_blocking=True)
        stream.synchronize()
        rank_barrier(world)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            frame()
            host_img.copy_(images, non_blocking=True)
        stream.synchronize()
        e2e_serial_value = world * args.steps / rank_max(time.perf_counter() - t0, world, dev)

        dev_imgs = [images, torch.empty_like(images)]
        host_imgs = [host_img, torch.empty(npix, dtype=torch.float32, pin_memory=True)]
        copy_stream = torch.cuda.Stream(dev)
        ev_done = [torch.cuda.Event(), torch.cuda.Event()]
        ev_copied = [torch.cuda.Event(), torch.cuda.Event()]

        def pipelined(k):
            b = k & 1
            if k >= 2:
                stream.wait_event(ev_copied[b])          # buffer b's previous read-back has finished
            h3dgs.h3dgs_select_cut(ctx.ctx, cams, ids, tt, offs, cap, want_total=False)
            h3dgs.h3dgs_render(ctx.ctx, cams, ids, tt, offs, opts, dev_imgs[b], 0, cam_array=carr)
            ev_done[b].record(stream)
            copy_stream.wait_event(ev_done[b])
            with torch.cuda.stream(copy_stream):
                host_imgs[b].copy_(dev_imgs[b], non_blocking=True)
            ev_copied[b].record(copy_stream)

        for k in range(args.warmup):
            pipelined(k)
        copy_stream.synchronize()
        stream.synchronize()
        rank_barrier(world)
        t0 = time.perf_counter()
        for k in range(args.steps):
            pipelined(k)
        copy_stream.synchronize()
        stream.synchronize()
        e2e_s = rank_max(time.perf_counter() - t0, world, dev)
        e2e_value = world * args.steps / e2e_s
        assert torch.equal(host_imgs[(args.steps - 1) & 1].to(dev), ref_img), "read-back differs from the frame"

        # ---- quality of the tau = 6 frame against the leaves-only (tau = 0) render of the same view
        # (after every use of the captured graphs: the leaves-only cut needs larger buffers)
        h3dgs.h3dgs_reserve(ctx.ctx, 0, 0)
        frame()
        img_tau = images.clone()
        leaf_cam = [synth.with_tau(cam, 0.0)]
        m0 = h3dgs.h3dgs_select_cut(ctx.ctx, leaf_cam, ids, tt, offs, cap)
        h3dgs.h3dgs_render(ctx.ctx, leaf_cam, ids, tt, offs, opts, images, 0)
        mse = float(((img_tau - images) ** 2).mean().item())
        quality = {"psnr_vs_leaves_db": 10.0 * np.log10(1.0 / max(mse, 1e-20)), "cut_tau": M_cut,
                   "cut_leaves": int(m0), "note": "image range ~[0, 1]; leaves = the tau = 0 render"}
        batched = run_batched(args, ctx, hier, flush, dev, stream) if args.batch_views > 0 else None
        optimisation = run_optimisation(args, dev, stream) if args.opt_leaves > 0 else None
        compaction = run_compaction(args, ctx, hier, stream) if args.compact_views > 0 else None
        streamed = run_streamed(args, hier, dev, stream) if args.stream_frames > 0 else None

    # ---- roofline of the dominant kernel: the blend's main kernel (FP32 issue-bound)
    peaks = measured_peaks()
    queue_ms = fwd_stages.get("blend_queue", 0.0)   # events around that kernel alone, on its stream
    n_evals, n_evals_i = int(st["n_evals"]), int(st["n_evals_interp"])
    n_contrib, n_contrib_i = int(st["n_contrib"]), int(st["n_contrib_interp"])
    flops = n_evals * BLEND_FLOPS_EVAL + n_evals_i * BLEND_FLOPS_INTERP + n_contrib * BLEND_FLOPS_CONTRIB
    xu_ops = n_evals * BLEND_XU_EVAL + n_evals_i * BLEND_XU_INTERP
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    fp32_peak_tflops = 148 * 128 * 2 * sm_max * 1e6 / 1e12
    achieved = flops / (queue_ms * 1e-3) / 1e12 if queue_ms > 0 else None
    roofline = {"kernel": "blend_queue_kernel<16,16>", "bound": "alu", "achieved": achieved, "peak": fp32_peak_tflops,
                "unit": "TFLOP/s", "frac": (achieved / fp32_peak_tflops) if achieved else None,
                "traffic": BLEND_TRAFFIC_BYTES if (args.tile == "16x16" and args.chunk in (0, 320)) else None,
                "kernel_ms": queue_ms,
                "peak_note": "148 SMs x 128 FP32 lanes x 2 (FFMA) x max SM clock from MEASURED_PEAKS.json",
                "work_note": f"the oracle's op list: {BLEND_FLOPS_EVAL} flops per main-pass (pixel, splat) evaluation "
                             f"x {n_evals}, +{BLEND_FLOPS_INTERP} for the {n_evals_i} on splats with an interpolated "
                             f"parent (Eq. alphap), +{BLEND_FLOPS_CONTRIB} per accumulated contribution x {n_contrib}; "
                             f"the {int(st['n_evals_tpass'])} evaluations of the middle chunks' producer walks (extra work "
                             f"of split tiles) are not counted; compares, min and selects are not flops",
                "traffic_note": "DRAM read + write of one launch from an ncu capture of this kernel at this workload"}
    if calib:
        roofline["peak_calibrated"] = calib["fp32_tflops"]
        roofline["frac_calibrated"] = (achieved / calib["fp32_tflops"]) if achieved else None
        roofline["ex2_gops_calibrated"] = calib["ex2_gops"]
        roofline["xu_frac_calibrated"] = (xu_ops / (queue_ms * 1e-3) / 1e9 / calib["ex2_gops"]) if queue_ms > 0 else None
        roofline["calibration_note"] = ("fp32 paired-FMA and exp2 chain kernels filling every SM, run by "
                                        "h3dgs_measure_peaks on this GPU before the timed region")
    # ---- adjoint (a8): the per-pixel stage against the FP32 peak with the oracle's op list, the per-splat
    # stage against HBM (node and parent rows read, gradient rows reduced)
    bb_ms, bs_ms = bwd_stages.get("backward_blend", 0.0), bwd_stages.get("backward_splat", 0.0)
    adj_flops = n_contrib * ADJ_FLOPS_CONTRIB + n_contrib_i * ADJ_FLOPS_CONTRIB_INTERP
    adj_achieved = adj_flops / (bb_ms * 1e-3) / 1e12 if bb_ms > 0 else None
    n_vis, n_parent_rows = int(st["n_visible"]), int(st_counts.get("n_interp_visible", 0))
    splat_bytes = n_vis * (236 + 59 * 4) + n_parent_rows * (236 + 59 * 4)
    hbm_peak = float(peaks.get("hbm_gbs", 6442.9))
    roofline_backward = {
        "backward_blend": {"bound": "alu", "achieved": adj_achieved, "peak": fp32_peak_tflops, "unit": "TFLOP/s",
                           "frac": (adj_achieved / fp32_peak_tflops) if adj_achieved else None,
                           "frac_calibrated": (adj_achieved / calib["fp32_tflops"]) if (adj_achieved and calib) else None,
                           "kernel_ms": bb_ms,
                           "work_note": f"the oracle's adjoint op list: {ADJ_FLOPS_CONTRIB} flops per contributing "
                                        f"(pixel, splat) pair x {n_contrib} (alpha recomputed + reverse step), "
                                        f"+{ADJ_FLOPS_CONTRIB_INTERP} for the {n_contrib_i} with t != 0"},
        "backward_splat": {"bound": "hbm", "achieved": splat_bytes / (bs_ms * 1e-3) / 1e9 if bs_ms > 0 else None,
                           "peak": hbm_peak, "unit": "GB/s",
                           "frac": (splat_bytes / (bs_ms * 1e-3) / 1e9 / hbm_peak) if bs_ms > 0 else None,
                           "kernel_ms": bs_ms,
                           "work_note": f"236 B attribute row read + 59 x 4 B gradient row reduced per visible cut "
                                        f"entry ({n_vis}) and again for the parent of each of the {n_parent_rows} "
                                        f"with t != 0"},
    }
    hbm = float(peaks.get("hbm_gbs", 6442.9))
    stage_bw = {}
    M, V, Pn = int(st["n_cut"]), int(st["n_visible"]), int(st["n_pairs"])
    visited = int(st_counts.get("n_cut_visited_traversal", 0)) or N
    Ug, Uv = int(st_counts.get("n_parents_geom", 0)), int(st_counts.get("n_parents_vis", 0))
    # algorithmic bytes per stage (the least the method moves):
    #   cut         the records of the visited nodes (the cut and its ancestors), 32 B each, + 8 B (id, t)
    #               out per cut entry
    #   preprocess  per entry its id, t, parent id and geometry (mean, scale, rot: 52 B) and per distinct
    #               interpolated parent the geometry (40 B); per visible entry opacity + SH (196 B) and per
    #               distinct parent of a visible interpolated entry opacity, K and SH (200 B); out 80 B
    #               (record 64, rect, key, tile count) per visible entry and 16 B per culled one
    #   sorts       one read and one write of each 8 B key/value pair (the LSD passes move that per pass:
    #               `pass_bytes`)
    #   duplicate   16 B read per visible splat, 8 B written per pair
    algo_bytes = {"cut": visited * 32 + M * 8,
                  "preprocess": M * 52 + Ug * 40 + V * 196 + Uv * 200 + V * 80 + (M - V) * 16,
                  "depth_sort": V * 16,
                  "duplicate": V * 16 + Pn * 8,
                  "tile_sort": Pn * 16}
    # bytes the implementation moves (the kernel's own efficiency): the scan reads the records of the
    # tiles its bound test keeps
    scan_read = int(st.get("n_cut_visited", N))
    impl_bytes = {**algo_bytes, "cut": scan_read * 32 + M * 8, "depth_sort": 4 * V * 16, "tile_sort": 2 * Pn * 16}
    for k, b in algo_bytes.items():
        if fwd_stages.get(k):
            sec = fwd_stages[k] * 1e-3
            stage_bw[k] = {"algorithmic_bytes": b, "algorithmic_GB/s": b / sec / 1e9,
                           "frac_hbm": b / sec / 1e9 / hbm}
            if impl_bytes[k] != b:
                stage_bw[k].update({"pass_bytes": impl_bytes[k], "pass_GB/s": impl_bytes[k] / sec / 1e9,
                                    "pass_frac_hbm": impl_bytes[k] / sec / 1e9 / hbm})
    if "preprocess" in stage_bw:
        stage_bw["preprocess"].update({"distinct_parents_geometry": Ug, "distinct_parents_visible": Uv})
    if "cut" in stage_bw:   # the frame's cut is the scan (all N records); the traversal is timed beside it
        vis_n = int(st_counts.get("n_cut_visited_traversal", 0))
        trav_bytes = vis_n * (32 + 16) + M * 16
        stage_bw["cut"].update({
            "mode": "scan", "visited_nodes": vis_n, "scan_read_nodes": scan_read,
            "traversal_visited_bytes": trav_bytes,
            "traversal_ms": st_counts.get("traversal_ms"),
            "traversal_GB/s": trav_bytes / (st_counts["traversal_ms"] * 1e-3) / 1e9 if st_counts.get("traversal_ms") else None,
            "note": "algorithmic: the visited nodes' records + 8 B per cut entry; pass (the scan): the "
                    "records of the tiles kept by its bound test + 8 B per cut entry; traversal: the visited "
                    "records + 16 B of frontier per visited node + 16 B per cut entry (marks, weights, ids)"})
    # frame-level roofline: the time every stage would take at its binding peak (HBM stages at the
    # measured copy bandwidth with their algorithmic bytes, the blend at the unit-count FP32 peak),
    # summed, over the frame time
    ideal_ms = sum(b / (hbm * 1e9) * 1e3 for b in algo_bytes.values())
    ideal_ms += flops / (fp32_peak_tflops * 1e12) * 1e3
    frame_ms = total_ms / args.steps
    frame_roofline = {"frac": ideal_ms / frame_ms, "ideal_ms": ideal_ms, "frame_ms": frame_ms,
                      "frac_with_pass_bytes": (ideal_ms + sum((impl_bytes[k] - algo_bytes[k]) / (hbm * 1e9) * 1e3
                                                              for k in algo_bytes)) / frame_ms,
                      "note": "sum over cut, preprocess, sorts, duplication (algorithmic bytes at the measured HBM "
                              "copy rate) and blend (main-pass flops at the FP32 peak), divided by the frame time; "
                              "frac_with_pass_bytes counts the scan's and the LSD passes' bytes instead"}
    clocks = clk.summary()
    out = {
        "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"street corridor, {args.n_leaves} leaves ({N} nodes), 1920x1080, tau={args.tau:g} px",
                   "n_leaves": args.n_leaves, "n_nodes": N, "width": cam.width, "height": cam.height, "tau": args.tau,
                   "cut_size": M, "visible_splats": V, "pairs": Pn, "evals": n_evals,
                   "l2": "flushed between timed steps (256 MB write, outside the events)",
                   "cuda_graph": graph is not None, "parallelism": f"{world} independent replicas"},
        "gaussians_per_s": M * value,
        "fwd_bwd": {"value": fb_value, "unit": "views/s", "ms_per_view": fb_ms / args.steps},
        "blend": {"items": int(st["n_items"]), "tile_chunk": int(opts.blend_chunk), "evals_main": n_evals,
                  "evals_main_interpolated": n_evals_i, "evals_tpass": int(st["n_evals_tpass"]),
                  "contributions": n_contrib, "contributions_interpolated": n_contrib_i,
                  "flops": flops, "xu_ops": xu_ops},
        "e2e": {"value": e2e_value, "unit": "frames/s", "h2d_bytes_per_step": 76 * len(cams),
                "d2h_bytes_per_step": npix * 4, "serial_value": e2e_serial_value,
                "note": "C-ABI calls from Python (not graph-captured), host clock; camera struct in, the whole "
                        "image read back to pinned host memory every step; value: read-back of step k on a "
                        "copy stream overlapping step k + 1 (two image buffers); serial_value: render then copy"},
        "stages_ms": {**fwd_stages, **bwd_stages}, "stage_bandwidth": stage_bw,
        "roofline": roofline,
        "roofline_backward": roofline_backward,
        "frame_roofline": frame_roofline,
        "tile": args.tile,
        "gpu_launches": args.steps * launches,
        "gpu_launches_per_step": launches, "gpu_launches_source": launch_src,
        "clocks": clocks,
    }
    out["quality"] = quality
    if batched is not None:
        out["batched"] = batched
    if optimisation is not None:
        out["optimisation"] = optimisation
    if compaction is not None:
        out["compaction"] = compaction
    if streamed is not None:
        out["streamed"] = streamed
    out["depth_exposure"] = depth_exposure
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_oracle_time(scene, 4)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return out if rank == 0 else None


def run_batched(args, ctx, hier, flush, dev, stream, cams=None, scene="street corridor 1M leaves"):
    """Many cameras of mixed resolution and tau in one launch per stage vs one frame per view."""
    import torch
    from paper_2406_12080_b300 import autotune, h3dgs, synth
    cams = cams if cams is not None else synth.corridor_views(n_views=args.batch_views)
    n = len(cams)
    N = hier.n
    h3dgs.h3dgs_reserve(ctx.ctx, 0, 0)
    ids = torch.empty(N, dtype=torch.int32, device=dev)
    tt = torch.empty(N, dtype=torch.float32, device=dev)
    offs = torch.empty(2, dtype=torch.int64, device=dev)
    sizes = [h3dgs.h3dgs_select_cut(ctx.ctx, [c], ids, tt, offs, N) for c in cams]
    cap = int(sum(sizes) * 1.02) + 1024
    del ids, tt
    ids = torch.empty(cap, dtype=torch.int32, device=dev)
    tt = torch.empty(cap, dtype=torch.float32, device=dev)
    offs = torch.empty(n + 1, dtype=torch.int64, device=dev)
    npix = sum(3 * c.width * c.height for c in cams)
    img_b = torch.empty(npix, dtype=torch.float32, device=dev)
    img_v = torch.empty(npix, dtype=torch.float32, device=dev)
    m = h3dgs.h3dgs_select_cut(ctx.ctx, cams, ids, tt, offs, cap)
    opts0 = h3dgs.default_opts()
    h3dgs.h3dgs_render(ctx.ctx, cams, ids, tt, offs, opts0, img_b, 0)
    st = h3dgs.h3dgs_get_stats(ctx.ctx)
    opts, table = autotune.tune(ctx, cams, (ids, tt, offs), img_b, use_cache=False)
    h3dgs.h3dgs_render(ctx.ctx, cams, ids, tt, offs, opts, img_b, 0)
    st = h3dgs.h3dgs_get_stats(ctx.ctx)
    h3dgs.h3dgs_reserve(ctx.ctx, int(m * 1.25) + 1024, int(st["n_pairs"] * 1.5) + 4096)
    carr = h3dgs.camera_array(cams)
    single = [h3dgs.camera_array([c]) for c in cams]
    offs1 = [torch.empty(2, dtype=torch.int64, device=dev) for _ in cams]
    img_off = np.cumsum([0] + [3 * c.width * c.height for c in cams])

    def batched():
        h3dgs.h3dgs_select_cut(ctx.ctx, cams, ids, tt, offs, cap, want_total=False)
        h3dgs.h3dgs_render(ctx.ctx, cams, ids, tt, offs, opts, img_b, 0, cam_array=carr)

    def per_view():
        for k, c in enumerate(cams):
            h3dgs.h3dgs_select_cut(ctx.ctx, [c], ids, tt, offs1[k], N, want_total=False)
            h3dgs.h3dgs_render(ctx.ctx, [c], ids, tt, offs1[k], opts, img_v[img_off[k]:img_off[k + 1]], 0,
                               cam_array=single[k])

    graphs = {}
    for name, fn in (("batched", batched), ("per_view", per_view)):
        fn()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            fn()
        graphs[name] = g
    times = {}
    reps = max(5, min(args.steps // 10, 30))
    for name, g in graphs.items():
        for _ in range(3):
            g.replay()
            flush.fill_(1.0)
        tot = 0.0
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.replay()
            e1.record(stream)
            flush.fill_(1.0)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        times[name] = tot / reps
    graphs["batched"].replay()   # stats of the batched frame (the per-view loop ran last)
    st = h3dgs.h3dgs_get_stats(ctx.ctx)
    max_diff = float((img_b - img_v).abs().max().item())
    # batched forward + backward (hierarchy optimisation over many views)
    grads = {k: torch.zeros_like(getattr(hier, k)) for k in ("mean", "scale", "rot", "opacity", "sh")}
    dl = torch.randn(npix, generator=torch.Generator(device=dev).manual_seed(1), device=dev)

    def fwd_bwd():
        h3dgs.h3dgs_select_cut(ctx.ctx, cams, ids, tt, offs, cap, want_total=False)
        h3dgs.h3dgs_render(ctx.ctx, cams, ids, tt, offs, opts, img_b, 1, cam_array=carr)
        h3dgs.h3dgs_render_backward(ctx.ctx, dl, grads, 1)

    fwd_bwd()
    gfb = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gfb, stream=stream):
        fwd_bwd()
    for _ in range(2):
        gfb.replay()
    tot = 0.0
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gfb.replay()
        e1.record(stream)
        flush.fill_(1.0)
        e1.synchronize()
        tot += e0.elapsed_time(e1)
    fb_ms = tot / reps
    res = sorted({f"{c.width}x{c.height}" for c in cams})
    return {"workload": f"{n} cameras ({', '.join(res)}), tau in (3, 6, 15), {scene}",
            "views": n, "pixels": npix // 3, "cut_total": int(st["n_cut"]), "pairs": int(st["n_pairs"]),
            "batched_ms": times["batched"], "per_view_ms": times["per_view"],
            "batched_views_per_s": n / (times["batched"] * 1e-3),
            "per_view_views_per_s": n / (times["per_view"] * 1e-3),
            "speedup": times["per_view"] / times["batched"], "max_abs_image_diff": max_diff,
            "fwd_bwd_views_per_s": n / (fb_ms * 1e-3),
            "autotune": {"tile": f"{opts.tile_w}x{opts.tile_h}", "chunk": int(opts.blend_chunk),
                         "table_ms": table}}


def run_optimisation(args, dev, stream):
    """Hierarchy optimisation: L1 against leaf renders, 8 views at 1280x720, autograd + Adam per step."""
    import torch
    from paper_2406_12080_b300 import autograd, h3dgs, synth
    scene = synth.corridor_scene(seed=3, n_leaves=args.opt_leaves)
    _, views = synth.optimisation_views(seed=3)
    ctx = h3dgs.Context(dev.index, stream)
    hier = ctx.build(scene.leaves)
    ctx.upload(hier)
    leaf_views = [synth.with_tau(c, 0.0) for c in views]
    targets = ctx.render(leaf_views, ctx.select_cut(leaf_views)).clone()
    params = autograd.HierarchyParams(hier)
    opt = torch.optim.Adam(params.parameters(), lr=1e-3)
    for _ in range(2):
        autograd.l1_step(params, ctx, hier, views, targets, opt)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    losses = []
    e0.record(stream)
    for _ in range(args.opt_steps):
        losses.append(autograd.l1_step(params, ctx, hier, views, targets, opt))
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / args.opt_steps
    st = h3dgs.h3dgs_get_stats(ctx.ctx)
    losses = [float(x) for x in losses]
    out = {"workload": f"street corridor {args.opt_leaves} leaves ({hier.n} nodes), {len(views)} views "
                       f"1280x720, tau log-uniform in [3, 640) px, L1 vs leaf renders, Adam",
           "ms_per_step": ms, "steps_per_s": 1e3 / ms, "views_per_s": len(views) * 1e3 / ms,
           "loss_first": losses[0], "loss_last": losses[-1], "cut_total": int(st["n_cut"]),
           "note": "each step: activations, upload, cut, render (save), adjoint, Adam; host syncs for "
                   "the cut size and pair count (not graph-captured)"}
    ctx.close()
    return out


def run_compaction(args, ctx, hier, stream, reps: int = 7):
    """Hierarchy compaction (Sec. 5.2) of the resident hierarchy for training views along the street.

    The call is synchronous (one host read per level of the new tree) and allocates its scratch, so
    it is timed on the host clock around the whole call."""
    import time
    import torch
    from paper_2406_12080_b300 import h3dgs, synth
    views = synth.corridor_views(seed=1, n_views=args.compact_views, resolutions=((1920, 1080),))
    tau_min, tau_max = 3.0, 960.0
    N = hier.n
    f = lambda *shape: torch.empty(shape, dtype=torch.float32, device=hier.mean.device)
    i = lambda n: torch.empty(n, dtype=torch.int32, device=hier.mean.device)
    out = h3dgs.DeviceHierarchy(f(N, 3), f(N, 3), f(N, 4), f(N), f(N, 48), f(N, 3), f(N, 3), i(N), i(N), i(N))
    old = i(N)
    m = h3dgs.h3dgs_compact_hierarchy(ctx.ctx, views, tau_min, tau_max, out, old)
    times = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m = h3dgs.h3dgs_compact_hierarchy(ctx.ctx, views, tau_min, tau_max, out, old)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    ms = 1e3 * min(times)
    cc = out.child_count[:m]
    return {"workload": f"street corridor hierarchy ({N} nodes), {len(views)} training views 1920x1080 along the "
                        f"street, tau levels {tau_min:g} x 2^k <= {tau_max:g} px",
            "ms": ms, "nodes_per_s": N / (ms * 1e-3), "view_node_tests_per_s": N * len(views) / (ms * 1e-3),
            "n_in": N, "n_out": int(m), "max_children": int(cc.max().item()),
            "wide_nodes": int((cc > 2).sum().item()),
            "note": "host clock around the synchronous call (best of 7), including its scratch allocation"}


def run_streamed(args, hier, dev, stream, update_every: int = 2, cleanup_every: int = 100, max_age: int = 100):
    """Out-of-core rendering along a drive down the street (Sec. 6.3): node attributes in page-locked
    host memory, a device cache of rows; the cut is updated every 2 frames (transferring the nodes it
    needs) and a cleanup runs every 100 frames.  Reported like the paper's per-path table: cut size
    (#Render) and transferred nodes (#Trans) per frame, and frames/s, next to the same path with the
    hierarchy resident."""
    import torch
    from paper_2406_12080_b300 import h3dgs, synth
    line = synth.corridor_polyline(1)
    F = args.stream_frames
    cams = [synth.corridor_camera(line, 150.0 + 0.5 * f, 1920, 1080, args.tau) for f in range(F)]
    cache = hier.n // 2
    stm = h3dgs.Context(dev.index, stream)
    res = h3dgs.Context(dev.index, stream)
    N = hier.n
    ids = torch.empty(N, dtype=torch.int32, device=dev)
    tt = torch.empty(N, dtype=torch.float32, device=dev)
    offs = torch.empty(2, dtype=torch.int64, device=dev)
    images = torch.empty(3 * 1920 * 1080, dtype=torch.float32, device=dev)
    opts = h3dgs.default_opts()
    with torch.cuda.stream(stream):
        host_h = stm.upload_streamed(hier, cache)
        res.upload(hier)
        # pass 1: counts (synchronising reads of the transfer and residency counters)
        cut_sizes, trans, resident, pairs = [], [], [], []
        for f, cam in enumerate(cams):
            if f % update_every == 0:
                cut_sizes.append(h3dgs.h3dgs_select_cut(stm.ctx, [cam], ids, tt, offs, N))
                trans.append(h3dgs.h3dgs_stream_update(stm.ctx, 1, ids, tt, offs, f))
            h3dgs.h3dgs_render(stm.ctx, [cam], ids, tt, offs, opts, images, 0)
            pairs.append(h3dgs.h3dgs_get_stats(stm.ctx)["n_pairs"])
            if (f + 1) % cleanup_every == 0:
                resident.append(h3dgs.h3dgs_stream_cleanup(stm.ctx, f, max_age))
        assert h3dgs.h3dgs_get_stats(stm.ctx)["device_flags"] == 0

        def path(ctx, streamed):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for f, cam in enumerate(cams):
                if f % update_every == 0:
                    h3dgs.h3dgs_select_cut(ctx.ctx, [cam], ids, tt, offs, N, want_total=False)
                    if streamed:
                        h3dgs.h3dgs_stream_update(ctx.ctx, 1, ids, tt, offs, f, want_count=False)
                h3dgs.h3dgs_render(ctx.ctx, [cam], ids, tt, offs, opts, images, 0)
                if streamed and (f + 1) % cleanup_every == 0:
                    h3dgs.h3dgs_stream_cleanup(ctx.ctx, f, max_age, want_count=False)
            e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1)

        # pass 2: timed, from a cold cache again (same host arrays), fixed capacities (no host reads)
        for c in (stm, res):
            h3dgs.h3dgs_reserve(c.ctx, int(max(cut_sizes) * 1.3) + 1024, int(max(pairs) * 1.3) + 4096)
        h3dgs.h3dgs_upload_hierarchy_streamed(stm.ctx, host_h, cache)
        ms_s = path(stm, True)
        assert h3dgs.h3dgs_get_stats(stm.ctx)["device_flags"] == 0
        path(res, False)
        ms_r = path(res, False)
    stm.close()
    res.close()
    return {"workload": f"drive of {F} frames (0.5 m apart) down the street corridor at 1920x1080, tau={args.tau:g}, "
                        f"cut every {update_every} frames, cleanup every {cleanup_every} frames (max age {max_age})",
            "n_nodes": N, "cache_rows": cache, "render_per_frame": float(np.mean(cut_sizes)),
            "trans_per_frame": float(np.sum(trans)) / F, "trans_first_update": trans[0],
            "resident_after_cleanups": resident, "fps_streamed": F / (ms_s * 1e-3), "fps_resident": F / (ms_r * 1e-3),
            "note": "host-side loop of ABI calls (not graph-captured), no L2 flush; each update gathers the missing "
                    "rows from page-locked host memory on the device"}


def _city_chunk(a):
    """One chunk of the city (worker of the generation pool)."""
    from paper_2406_12080_b300 import synth
    seed, c, grid, per = a
    lv = synth.city_chunk_leaves(seed, c % grid, c // grid, per)
    return c, lv


def build_city(args, ctx, dev):
    """The chunked city on the device: leaves generated chunk by chunk on the host cores, then the
    consolidated hierarchy (per-chunk trees joined by a top tree) built by the library."""
    import multiprocessing as mp
    import torch
    K = args.city_grid * args.city_grid
    per = args.city_leaves // K
    L = K * per
    f = lambda *shape: torch.empty(shape, dtype=torch.float32, device=dev)
    leaves = {"mean": f(L, 3), "scale": f(L, 3), "rot": f(L, 4), "opacity": f(L), "sh": f(L, 48)}
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1))) as pool:
        for c, lv in pool.imap(_city_chunk, [(2, c, args.city_grid, per) for c in range(K)], chunksize=4):
            sl = slice(c * per, (c + 1) * per)
            for k in leaves:
                leaves[k][sl].copy_(torch.from_numpy(getattr(lv, k)))
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    hier = ctx.build_chunked(leaves, np.arange(K + 1, dtype=np.int64) * per)
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t0
    del leaves
    torch.cuda.empty_cache()
    return hier, L, t_gen, t_build


def run_city(args, rank, world, local):
    import torch
    from paper_2406_12080_b300 import build, h3dgs, synth
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.Stream(dev)
    ctx = h3dgs.Context(local, stream)
    with torch.cuda.stream(stream):
        hier, L, t_gen, t_build = build_city(args, ctx, dev)
        ctx.upload(hier)
        N = hier.n
        poses = synth.city_path(2, args.city_poses)
        ids = torch.empty(N, dtype=torch.int32, device=dev)
        tt = torch.empty(N, dtype=torch.float32, device=dev)
        offs = torch.empty(2, dtype=torch.int64, device=dev)
        npix = 3 * poses[0].width * poses[0].height
        images = torch.empty(npix, dtype=torch.float32, device=dev)
        opts = h3dgs.default_opts(blend_chunk=args.chunk)
        # size the fixed workspace from 32 poses spread over the loop (every pose of a short loop), then
        # time every pose with events
        h3dgs.h3dgs_reserve(ctx.ctx, 0, 0)
        mmax = pmax = 0
        for c in poses[::max(1, len(poses) // 32)]:
            mmax = max(mmax, h3dgs.h3dgs_select_cut(ctx.ctx, [c], ids, tt, offs, N))
            h3dgs.h3dgs_render(ctx.ctx, [c], ids, tt, offs, opts, images, 0)
            pmax = max(pmax, h3dgs.h3dgs_get_stats(ctx.ctx)["n_pairs"])
        h3dgs.h3dgs_reserve(ctx.ctx, int(mmax * 1.3) + 4096, int(pmax * 1.3) + 65536)
        arrs = [h3dgs.camera_array([c]) for c in poses]
        for c, a in zip(poses[:args.warmup], arrs):
            h3dgs.h3dgs_select_cut(ctx.ctx, [c], ids, tt, offs, N, want_total=False)
            h3dgs.h3dgs_render(ctx.ctx, [c], ids, tt, offs, opts, images, 0, cam_array=a)
        torch.cuda.synchronize()
        rank_barrier(world)
        cut_ms, render_ms, sizes, pairs, scan_read = [], [], [], [], []
        with ClockSampler(local) as clk:
            for c, a in zip(poses, arrs):
                e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                e[0].record(stream)
                h3dgs.h3dgs_select_cut(ctx.ctx, [c], ids, tt, offs, N, want_total=False)
                e[1].record(stream)
                h3dgs.h3dgs_render(ctx.ctx, [c], ids, tt, offs, opts, images, 0, cam_array=a)
                e[2].record(stream)
                st = h3dgs.h3dgs_get_stats(ctx.ctx)   # synchronises
                assert st["device_flags"] == 0, f"device flags {st['device_flags']}"
                cut_ms.append(e[0].elapsed_time(e[1]))
                render_ms.append(e[1].elapsed_time(e[2]))
                sizes.append(int(st["n_cut"]))
                pairs.append(int(st["n_pairs"]))
                scan_read.append(int(st["n_cut_visited"]))
        frame_ms = np.array(cut_ms) + np.array(render_ms)
        # per-stage device times (profiling events) on every 16th pose, outside the timed loop
        h3dgs.h3dgs_set_profiling(ctx.ctx, 1)
        stage_acc, n_st = {}, 0
        for c, a in list(zip(poses, arrs))[::16]:
            h3dgs.h3dgs_select_cut(ctx.ctx, [c], ids, tt, offs, N, want_total=False)
            h3dgs.h3dgs_render(ctx.ctx, [c], ids, tt, offs, opts, images, 0, cam_array=a)
            for k, v in h3dgs.h3dgs_get_stage_times(ctx.ctx).items():
                stage_acc[k] = stage_acc.get(k, 0.0) + v
            n_st += 1
        h3dgs.h3dgs_set_profiling(ctx.ctx, 0)
        city_stages = {k: v / n_st for k, v in stage_acc.items() if v > 0}
        # the root-down traversal on the same poses (every 8th): the records it reads and its time
        h3dgs.h3dgs_set_cut_mode(ctx.ctx, 2)
        h3dgs.h3dgs_select_cut(ctx.ctx, [poses[0]], ids, tt, offs, N)   # sizes the traversal's buffers
        trav_ms, visited = [], []
        for c in poses[::8]:
            e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            e[0].record(stream)
            h3dgs.h3dgs_select_cut(ctx.ctx, [c], ids, tt, offs, N, want_total=False)
            e[1].record(stream)
            e[1].synchronize()
            trav_ms.append(e[0].elapsed_time(e[1]))
            visited.append(int(h3dgs.h3dgs_get_stats(ctx.ctx)["n_cut_visited"]))
        h3dgs.h3dgs_set_cut_mode(ctx.ctx, 0)
        scan_ms = cut_ms
        hbm = float(measured_peaks().get("hbm_gbs", 6442.9))
        v_mean = float(np.mean(visited))
        # algorithmic bytes: the 32 B record of every visited node (the cut and its ancestors), + 8 B per
        # cut entry written; the scan reads the records of the tiles its bound test keeps, the descent
        # also reads and writes 8 B of frontier per visited node and 4 B of weight per cut node
        algo_bytes = v_mean * 32 + float(np.mean(sizes)) * 8
        trav_bytes = v_mean * (32 + 16) + float(np.mean(sizes)) * (8 + 8)
        scan_bytes = float(np.mean(scan_read)) * 32 + float(np.mean(sizes)) * 8
        cut_bw = {"visited_nodes_mean": v_mean, "algorithmic_bytes": algo_bytes,
                  "algorithmic_GB/s": algo_bytes / (np.mean(scan_ms) * 1e-3) / 1e9,
                  "algorithmic_frac_hbm": algo_bytes / (np.mean(scan_ms) * 1e-3) / 1e9 / hbm,
                  "scan_read_nodes_mean": float(np.mean(scan_read)), "scan_bytes": scan_bytes,
                  "full_scan_bytes": N * 32 + float(np.mean(sizes)) * 8, "traversal_bytes": trav_bytes,
                  "mode": "scan", "scan_ms_mean": float(np.mean(scan_ms)),
                  "scan_GB/s": scan_bytes / (np.mean(scan_ms) * 1e-3) / 1e9,
                  "scan_frac_hbm": scan_bytes / (np.mean(scan_ms) * 1e-3) / 1e9 / hbm,
                  "traversal_ms_mean": float(np.mean(trav_ms)),
                  "traversal_GB/s": trav_bytes / (np.mean(trav_ms) * 1e-3) / 1e9,
                  "traversal_frac_hbm": trav_bytes / (np.mean(trav_ms) * 1e-3) / 1e9 / hbm,
                  "note": "one camera per frame; the frames use the scan (every record of the 256-node rows "
                          "whose parents' granularity bound reaches tau; algorithmic_GB/s is the visited nodes' "
                          "records over the scan's time); the root-down traversal (cut and ancestors + "
                          "frontier traffic) is timed on every 8th pose"}
        loop_ms = rank_max(frame_ms.sum(), world, dev)   # the slowest rank's loop
        value = world * len(poses) / (loop_ms * 1e-3)
        batched = None
        if args.batch_views > 0:
            flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
            batched = run_batched(args, ctx, hier, flush, dev, stream, cams=synth.city_views(2, args.batch_views),
                                  scene=f"chunked city {L} leaves")
    out = {
        "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": len(poses),
        "warmup": args.warmup, "ms_per_step": float(frame_ms.mean()), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"chunked city, {L} leaves ({N} nodes) in {args.city_grid}x{args.city_grid} chunks of "
                               f"50 m, {len(poses)}-pose loop at 1920x1080, tau=6 px",
                   "n_leaves": L, "n_nodes": N, "l2": "working set (3.2 GB of node records) far above L2"},
        "per_frame": {"cut_size_mean": float(np.mean(sizes)), "cut_size_max": int(np.max(sizes)),
                      "pairs_mean": float(np.mean(pairs)), "cut_ms_mean": float(np.mean(cut_ms)),
                      "cut_ms_max": float(np.max(cut_ms)), "render_ms_mean": float(np.mean(render_ms)),
                      "render_ms_max": float(np.max(render_ms)), "frame_ms_p50": float(np.median(frame_ms)),
                      "frame_ms_max": float(frame_ms.max())},
        "gaussians_per_s": float(world * np.sum(sizes) / (loop_ms * 1e-3)),
        "stage_bandwidth": {"cut": cut_bw},
        "stages_ms": city_stages,
        "build": {"host_generation_s": t_gen, "device_build_s": t_build},
        "clocks": clk.summary(),
    }
    if batched is not None:
        out["batched"] = batched
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return out if rank == 0 else None


# ----------------------------------------------------------------------------------- reference arm

def run_reference(args, rank, world):
    if rank != 0:
        return None
    from paper_2406_12080_b300 import synth
    import oracle
    scene = synth.corridor_scene(n_leaves=args.n_leaves, tau=args.tau)
    h = oracle.build_tree(scene.leaves)
    cam = scene.cameras[0]
    # each step is one full frame; the run stops early once REF_BUDGET_S of timed work is done so that
    # the default --steps finishes within a few minutes (the steps actually timed are reported)
    for _ in range(args.warmup):
        oracle.render(cam, h, oracle.Opts())
    t0 = time.perf_counter()
    done = 0
    while done < args.steps:
        oracle.render(cam, h, oracle.Opts())
        done += 1
        if time.perf_counter() - t0 > REF_BUDGET_S:
            break
    dt = time.perf_counter() - t0
    v = done / dt
    cores = oracle.num_threads()
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "frames/s", "n_gpus": world,
            "steps": done, "steps_requested": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / done,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"street corridor, {args.n_leaves} leaves, 1920x1080, tau={args.tau:g} px"},
            "cpu_baseline": {"value": v, "unit": "frames/s", "cores": cores, "kind": "oracle",
                             "sample": f"{done} full frames (cut + render) of the benchmark workload, "
                                       f"at most ~{REF_BUDGET_S:.0f} s of timed work"},
            "e2e": {"value": v, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    elif args.workload == "city":
        out = run_city(args, rank, world, local)
    else:
        out = run_ours(args, rank, world, local)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
