"""Parity of the expected-depth output and the exposure affine (h3dgs_render_ex) and of their
adjoint (h3dgs_render_backward_ex) with the oracle.

Bars: images at the forward bar (2e-3 on unambiguous pixels); depth within 2e-3 of the frame's
largest splat depth (the depth is a weighted mean of splat depths whose weights carry the colour's
error); gradients at the per-element backward bar of tests/test_parity_backward.py."""
import numpy as np
import pytest

import oracle
from paper_2406_12080_b300 import h3dgs, synth
from tests import gpu_path, scenes
from tests.test_parity_backward import _check, loss_weight

pytestmark = pytest.mark.gpu
IMG_TOL = 2e-3


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_12080_b300 import build
    build.build()


def _exposures(n, seed):
    rng = np.random.default_rng(seed)
    base = np.hstack([np.eye(3), np.zeros((3, 1))])[None]
    return (base + rng.normal(0, 0.15, size=(n, 3, 4))).astype(np.float32)


def _render(cams, opts, E, chunk=None, save=0):
    import torch
    ctx = gpu_path.context()
    cut = ctx.select_cut(cams)
    Ed = torch.from_numpy(E).cuda()
    images, depth = ctx.render(cams, cut, gpu_path.opts_from(opts, chunk), save_for_backward=save, depth=True,
                               exposure=Ed)
    torch.cuda.synchronize()
    st = h3dgs.h3dgs_get_stats(ctx.ctx)
    assert st["device_flags"] == 0
    return cut, Ed, images, depth


def _split(x, cams, ch):
    out, o = [], 0
    for c in cams:
        n = ch * c.width * c.height
        out.append(x[o:o + n].reshape(ch, c.height, c.width) if ch > 1 else x[o:o + n].reshape(c.height, c.width))
        o += n
    return out


@pytest.mark.parametrize("chunk", [None, 64])
def test_forward_batch_with_exposure_and_depth(chunk):
    sc, h = scenes.tiny()
    gpu_path.upload(h)
    cams = [synth.with_tau(sc.cameras[0], 6.0),
            synth.look_camera([5, 5, -12.0], [0.1, 0, 1], [0, -1, 0], 200, 150, 60.0, 3.0),
            synth.look_camera([-8, 5, 5.0], [1, 0, 0.05], [0, -1, 0], 96, 128, 75.0, 15.0)]
    opts = oracle.Opts(bg=(0.1, 0.3, 0.2))
    E = _exposures(len(cams), 1)
    cut, Ed, images, depth = _render(cams, opts, E, chunk)
    imgs = _split(images.cpu().numpy(), cams, 3)
    deps = _split(depth.cpu().numpy(), cams, 1)
    for k, cam in enumerate(cams):
        ofr = oracle.render(cam, h, opts, exposure=E[k])
        amb = ofr.ambiguous
        assert amb.mean() < 2e-4
        err = np.abs(imgs[k] - ofr.image).max(axis=0)
        assert err[~amb].max() <= IMG_TOL, err[~amb].max()
        zmax = ofr.val64[ofr.rect[:, 0] >= 0, 12].max()
        derr = np.abs(deps[k] - ofr.depth)
        assert derr[~amb].max() <= IMG_TOL * zmax, (derr[~amb].max(), zmax)
        assert ofr.depth.max() > 0.5 * zmax * 0.1



@pytest.mark.parametrize("seed", range(10))
def test_depth_and_exposure_on_random_scenes_and_cameras(seed):
    """The expected depth and an exposure affine on the forward path's seeded random scenes and
    cameras (one of them sees nothing: background only, depth zero)."""
    h, cam = scenes.random_case(seed)
    gpu_path.upload(h)
    opts = oracle.Opts(bg=(0.1, 0.3, 0.2))
    E = _exposures(1, 20 + seed)
    cut, Ed, images, depth = _render([cam], opts, E)
    img = _split(images.cpu().numpy(), [cam], 3)[0]
    dep = _split(depth.cpu().numpy(), [cam], 1)[0]
    ofr = oracle.render(cam, h, opts, exposure=E[0])
    amb = ofr.ambiguous
    assert amb.mean() < 2e-4
    err = np.abs(img - ofr.image).max(axis=0)
    assert err[~amb].max() <= IMG_TOL, err[~amb].max()
    vis = ofr.rect[:, 0] >= 0
    zmax = float(ofr.val64[vis, 12].max()) if vis.any() else 0.0
    derr = np.abs(dep - ofr.depth)
    assert derr[~amb].max() <= IMG_TOL * max(zmax, 1e-6), (derr[~amb].max(), zmax)

def test_plain_render_is_unchanged_by_the_extended_entry_point():
    import torch
    sc, h = scenes.tiny()
    gpu_path.upload(h)
    cam = sc.cameras[0]
    ctx = gpu_path.context()
    cut = ctx.select_cut([cam])
    a = ctx.render([cam], cut).clone()
    ident = torch.from_numpy(np.hstack([np.eye(3), np.zeros((3, 1))]).astype(np.float32)[None]).cuda()
    b, d = ctx.render([cam], cut, depth=True, exposure=ident)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


@pytest.mark.parametrize("tau,chunk", [(6.0, None), (15.0, None), (6.0, 64)])
def test_backward_with_depth_and_exposure(tau, chunk):
    import torch
    sc, h = scenes.tiny()
    dh = gpu_path.upload(h)
    cam = synth.with_tau(sc.cameras[0], tau)
    opts = oracle.Opts()
    E = _exposures(1, 2)
    fr = oracle.render(cam, h, opts, exposure=E[0])
    w = loss_weight(fr, 3)
    wd = np.random.default_rng(4).normal(size=fr.depth.shape) * 0.05
    wd[fr.ambiguous] = 0.0
    og = oracle.backward(cam, h, fr, w, opts, dL_ddepth=wd, exposure=E[0])
    cut, Ed, images, depth = _render([cam], opts, E, chunk, save=1)
    grads = {k: torch.zeros_like(getattr(dh, k)) for k in ("mean", "scale", "rot", "opacity", "sh")}
    dl = torch.from_numpy(np.ascontiguousarray(w, np.float32).reshape(-1)).cuda()
    dd = torch.from_numpy(np.ascontiguousarray(wd, np.float32).reshape(-1)).cuda()
    h3dgs.h3dgs_render_backward_ex(gpu_path.context().ctx, dl, dd, grads, 0)
    torch.cuda.synchronize()
    gg = np.concatenate([grads[k].cpu().numpy().reshape(dh.n, -1) for k in ("mean", "scale", "rot", "opacity", "sh")],
                        axis=1)
    _check(gg, og)


def test_depth_gradient_needs_a_depth_forward():
    import torch
    sc, h = scenes.tiny()
    dh = gpu_path.upload(h)
    cam = sc.cameras[0]
    ctx = gpu_path.context()
    cut = ctx.select_cut([cam])
    img = ctx.render([cam], cut, save_for_backward=1)
    grads = {k: torch.zeros_like(getattr(dh, k)) for k in ("mean", "scale", "rot", "opacity", "sh")}
    dd = torch.zeros(cam.width * cam.height, device="cuda")
    with pytest.raises(h3dgs.H3dgsError) as e:
        h3dgs.h3dgs_render_backward_ex(ctx.ctx, torch.zeros_like(img), dd, grads, 0)
    assert e.value.status == 6


def test_autograd_depth_loss_reaches_interior_means():
    import torch
    from paper_2406_12080_b300 import autograd
    sc, h = scenes.tiny()
    gpu_path.upload(h)
    dh = h3dgs.DeviceHierarchy.from_arrays(h)
    ctx = gpu_path.context()
    cam = synth.with_tau(sc.cameras[0], 15.0)
    mean = dh.mean.clone().requires_grad_(True)
    E = torch.from_numpy(_exposures(1, 4)).cuda()
    img, dep = autograd.render_depth(ctx, dh, mean, dh.scale, dh.rot, dh.opacity, dh.sh, [cam], exposure=E)
    loss = dep.sum() + 0.5 * img.sum()
    loss.backward()
    g = mean.grad.cpu().numpy()
    interior = h.child_count > 0
    assert np.abs(g[interior]).max() > 0
    assert np.all(g[~interior] == 0)   # leaves frozen by default
