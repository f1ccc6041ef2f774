"""Inverse rendering through the autograd wrapper: recover a dielectric height field from
the caustic it casts, with gradients from light tracing only (the paper's geometric inverse
problem, on a small synthetic slab)."""
import numpy as np
import pytest
import torch

from paper_2609_32920_gb300 import inputs as I
from paper_2609_32920_gb300 import lt
from paper_2609_32920_gb300.autograd import render

pytestmark = pytest.mark.gpu


def test_autograd_gradient_equals_direct_backward():
    sc = I.box_scene(32, heightmap=6, hm_std=0.03)
    S = lt.Scene(sc)
    albedo = S.albedo.clone().requires_grad_(True)
    Le = S.Le.clone().requires_grad_(True)
    h = S.heights.clone().requires_grad_(True)
    img = render(S, albedo, Le, h, method="lrb3", seed=3, n_paths=1 << 13, max_depth=5)
    dI = torch.tensor(I.smooth_adjoint(sc.W, sc.H, 5), dtype=torch.float32, device="cuda")
    (img * dI).sum().backward()
    o = S.opts(seed=3, n_paths=1 << 13, max_depth=5, attached=1)
    gA, gL, gH = S.backward_lrb3(o, dI)
    torch.cuda.synchronize()
    assert torch.allclose(albedo.grad, gA[: albedo.numel()], rtol=1e-5, atol=1e-12)
    assert torch.allclose(Le.grad, gL, rtol=1e-5)
    assert torch.allclose(h.grad, gH[: h.numel()], rtol=1e-4, atol=1e-9)


@pytest.mark.parametrize("method", ["lrb3", "naive"])
def test_autograd_gradient_matches_central_differences(method):
    """Detached albedo and emitted-radiance gradients through the autograd wrapper against
    central differences of the GPU image at the same seed (the light-traced image of a
    fixed seed is a polynomial in the albedos and linear in Le; no discrete decision
    depends on either).  Differences are taken in FP64 from FP32 images."""
    sc = I.box_scene(32)
    S = lt.Scene(sc)
    kw = dict(method=method, seed=9, n_paths=1 << 15, max_depth=4, attached=False)
    dI = torch.tensor(I.smooth_adjoint(sc.W, sc.H, 6), dtype=torch.float32, device="cuda")
    h0 = S.heights.clone()
    albedo = S.albedo.clone().requires_grad_(True)
    Le = S.Le.clone().requires_grad_(True)
    (render(S, albedo, Le, h0, **kw) * dI).sum().backward()
    torch.cuda.synchronize()

    def loss(a, le):
        with torch.no_grad():
            img = render(S, a, le, h0, **kw)
        return float((img.double() * dI.double()).sum())

    rng = np.random.default_rng(0)
    va = torch.tensor(rng.normal(size=albedo.numel()), dtype=torch.float32, device="cuda")
    step = 5e-3
    a0 = albedo.detach()
    fd = (loss(a0 + step * va, Le.detach()) - loss(a0 - step * va, Le.detach())) / (2 * step)
    ad = float((albedo.grad.double() * va.double()).sum())
    assert abs(fd - ad) <= 1e-3 * abs(ad), (fd, ad)
    for c in range(3):
        e = torch.zeros(3, device="cuda")
        e[c] = 0.05
        fd = (loss(a0, Le.detach() + e) - loss(a0, Le.detach() - e)) / 0.1
        assert abs(fd - float(Le.grad[c])) <= 1e-3 * abs(float(Le.grad[c])), (c, fd, float(Le.grad[c]))


@pytest.mark.parametrize("method", ["lrb3", "reslrb", "naive"])
def test_caustic_height_field_optimisation_reduces_loss(method):
    true_sc = I.slab_scene(48, n=12, seed=1)
    T_S = lt.Scene(true_sc)
    target = T_S.primal(T_S.opts(seed=777, n_paths=1 << 21, max_depth=4))
    sc = I.slab_scene(48, n=12, seed=0)
    S = lt.Scene(sc)
    h = S.heights.clone().requires_grad_(True)
    h_true = torch.tensor(true_sc.heights, dtype=torch.float32, device="cuda")
    opt = torch.optim.Adam([h], lr=1e-3)
    losses = []
    for step in range(40):
        opt.zero_grad()
        img = render(S, S.albedo, S.Le, h, method=method, seed=step, n_paths=1 << 17, max_depth=4)
        loss = ((img - target) ** 2).mean()
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
    S.sync_status()
    first, last = np.mean(losses[:5]), np.mean(losses[-5:])
    assert last < 0.7 * first, (first, last)
    d0 = torch.linalg.norm(torch.tensor(sc.heights, device="cuda") - h_true)
    assert torch.linalg.norm(h.detach() - h_true) < d0
