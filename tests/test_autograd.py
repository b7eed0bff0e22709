"""The torch.autograd.Function over the render: its gradients, through the torch-side activations,
against the oracle's fp64 adjoint, and a few hierarchy-optimisation steps (Sec. 5.1)."""
import numpy as np
import pytest

import oracle
from paper_2406_12080_b300 import autograd, h3dgs, synth
from tests import gpu_path, scenes

pytestmark = pytest.mark.gpu
GROUPS = [("mean", 0, 3), ("scale", 3, 6), ("rot", 6, 10), ("opacity", 10, 11), ("sh", 11, 59)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_12080_b300 import build
    build.build()


def _scene():
    lv, cam = scenes.small_random_scene(n_leaves=40, res=(40, 32), seed=9, log_scale=-2.2)
    h = oracle.build_tree(lv)
    eps = oracle.granularity(cam, h)
    tau = float(np.quantile(eps[h.child_count > 0], 0.5))
    return h, synth.with_tau(cam, tau)


@pytest.mark.parametrize("freeze", [False, True])
def test_autograd_gradients_match_the_oracle_through_the_activations(freeze):
    import torch
    h, cam = _scene()
    dh = gpu_path.upload(h)
    params = autograd.HierarchyParams(dh)
    ctx = gpu_path.context()
    images = autograd.render(ctx, dh, *params.activated(), [cam], freeze_leaves=freeze)
    opts = oracle.Opts()
    fr = oracle.render(cam, h, opts)
    w = np.random.default_rng(3).normal(size=fr.image.shape)
    w[:, fr.ambiguous] = 0.0
    (images * torch.from_numpy(w.reshape(-1).astype(np.float32)).cuda()).sum().backward()
    og = oracle.backward(cam, h, fr, w, opts, freeze_leaves=int(freeze))
    leaf = h.child_count == 0
    op = h.opacity.astype(np.float64)
    # chain rule of the activations: scale = exp(log_scale); leaf opacity = sigmoid(raw); interior = |raw|
    dscale = og[:, 3:6] * h.scale.astype(np.float64)
    dop = og[:, 10] * np.where(leaf, op * (1 - op), 1.0)
    want = {"mean": og[:, 0:3], "log_scale": dscale, "rot": og[:, 6:10], "opacity_raw": dop, "sh": og[:, 11:59]}
    for name, o in want.items():
        g = getattr(params, name).grad.cpu().numpy().astype(np.float64).reshape(o.shape)
        scale = np.abs(o).max()
        assert scale > 0 or np.abs(g).max() == 0, name
        if scale > 0:   # per element: the backward bar, the activations' chain rule in torch fp32 on top
            excess = (np.abs(g - o) - 2e-3 * np.abs(o)) / scale
            assert excess.max() <= 1e-5, (name, float(excess.max()))
    if freeze:
        for name in want:
            g = getattr(params, name).grad.cpu().numpy().reshape(h.n, -1)
            assert np.all(g[leaf] == 0), name


def test_optimisation_steps_lower_the_l1_loss_and_keep_frozen_leaves():
    import torch
    sc, h = scenes.tiny()
    dh = gpu_path.upload(h)
    ctx = gpu_path.context()
    base = sc.cameras[0]
    views = [synth.with_tau(base, t) for t in (4.0, 8.0)]
    # targets: the leaves-only render (tau = 0) of the same views
    leaf_cams = [synth.with_tau(c, 0.0) for c in views]
    targets = ctx.render(leaf_cams, ctx.select_cut(leaf_cams)).clone()
    params = autograd.HierarchyParams(dh)
    leaf = (dh.child_count == 0)
    before = {k: v.detach().clone() for k, v in params.named_parameters()}
    opt = torch.optim.Adam(params.parameters(), lr=2e-3)
    losses = [float(autograd.l1_step(params, ctx, dh, views, targets, opt)) for _ in range(12)]
    assert losses[-1] < losses[0] * 0.995, losses
    for k, v in params.named_parameters():
        assert torch.equal(v.detach()[leaf], before[k][leaf]), k
        assert not torch.equal(v.detach()[~leaf], before[k][~leaf]), k
