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


def test_autograd_backward_uses_the_geometry_of_its_own_forward_pass():
    """Two renders of one scene at different heights before either backward: each backward
    must replay its paths against the heights of its own forward pass."""
    sc = I.box_scene(32, heightmap=6, hm_std=0.03)
    S = lt.Scene(sc)
    dI = torch.tensor(I.smooth_adjoint(sc.W, sc.H, 8), dtype=torch.float32, device="cuda")
    h1 = S.heights.clone().requires_grad_(True)
    h2 = (S.heights * 0.5 + 0.01).requires_grad_(True)
    kw = dict(method="lrb3", seed=4, n_paths=1 << 13, max_depth=5)
    img1 = render(S, S.albedo, S.Le, h1, **kw)
    img2 = render(S, S.albedo, S.Le, h2, **kw)
    ((img1 + img2) * dI).sum().backward()
    torch.cuda.synchronize()
    o = S.opts(seed=4, n_paths=1 << 13, max_depth=5, attached=1)
    for h in (h1, h2):
        S.refit(h.detach())
        gH = S.backward_lrb3(o, dI)[2][: h.numel()]
        torch.cuda.synchronize()
        assert torch.allclose(h.grad, gH, rtol=1e-4, atol=1e-9)
    assert not torch.allclose(h1.grad, h2.grad, rtol=1e-2)


@pytest.mark.parametrize("method", ["lrb3", "naive", "lrb2"])
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


def _loss64(img, dI):
    return float((img.double() * dI.double()).sum())


def test_autograd_reslrb_matches_central_differences_in_expectation():
    """ResLRB's per-seed gradient differentiates its own reservoir estimator (weights held),
    so it is compared in expectation (Eq. 10): per seed, its detached albedo and Le
    gradients through autograd, projected on a fixed direction, minus the central
    difference of the plain light-traced image of the same seed (exact per seed: a
    polynomial in the albedos, linear in Le); the mean of these paired differences over 64
    seeds is within 3 standard errors of zero."""
    sc = I.box_scene(32)
    S = lt.Scene(sc)
    dI = torch.tensor(I.smooth_adjoint(sc.W, sc.H, 16), dtype=torch.float32, device="cuda")
    h0 = S.heights.clone()
    a0, le0 = S.albedo.clone(), S.Le.clone()
    rng = np.random.default_rng(3)
    va = torch.tensor(rng.normal(size=a0.numel()), dtype=torch.float32, device="cuda")
    vl = torch.tensor([0.3, -0.2, 0.5], dtype=torch.float32, device="cuda")
    step = 5e-3
    d = []
    for s in range(64):
        kw = dict(seed=200 + s, n_paths=1 << 13, max_depth=5, attached=False)
        a = a0.clone().requires_grad_(True)
        le = le0.clone().requires_grad_(True)
        (render(S, a, le, h0, method="reslrb", **kw) * dI).sum().backward()
        ad = float((a.grad.double() * va.double()).sum() + (le.grad.double() * vl.double()).sum())
        with torch.no_grad():
            fp = _loss64(render(S, a0 + step * va, le0 + step * vl, h0, method="lrb3", **kw), dI)
            fm = _loss64(render(S, a0 - step * va, le0 - step * vl, h0, method="lrb3", **kw), dI)
        d.append(ad - (fp - fm) / (2 * step))
    S.sync_status()
    d = np.array(d)
    z = d.mean() / (d.std(ddof=1) / np.sqrt(len(d)))
    assert abs(z) < 3.0, z


@pytest.mark.parametrize("method", ["lrb3", "reslrb"])
def test_autograd_attached_heights_match_central_differences_in_expectation(method):
    """Attached height gradients through autograd against common-random-number central
    differences of the full GPU renderer, which re-takes its discrete decisions at the
    perturbed heights: a diffuse height field under a square emitter, seen from the side,
    where no visibility boundary moves (interior derivative only).  Per seed the two
    differ (the differences re-decide paths near triangle edges); over 64 seeds the mean of
    the paired differences is within 3.5 standard errors of zero for each probed height."""
    sc = I.plane_under_light(res=16, heightmap=9, hm_std=0.05, plane_half=1.5, light_h=0.8, light_size=0.3)
    S = lt.Scene(sc)
    dI = torch.full((sc.H, sc.W, 3), 1.0 / (sc.W * sc.H), device="cuda")
    h0 = S.heights.clone()
    ks, h = [40, 31], 2e-3
    diffs = []
    for s in range(64):
        kw = dict(seed=s, n_paths=1 << 15, max_depth=1, attached=True)
        hh = h0.clone().requires_grad_(True)
        (render(S, S.albedo, S.Le, hh, method=method, **kw) * dI).sum().backward()
        fd = []
        for k in ks:
            e = torch.zeros_like(h0)
            e[k] = h
            with torch.no_grad():
                fd.append((_loss64(render(S, S.albedo, S.Le, h0 + e, method="lrb3", **kw), dI)
                           - _loss64(render(S, S.albedo, S.Le, h0 - e, method="lrb3", **kw), dI)) / (2 * h))
        diffs.append(hh.grad[ks].double().cpu().numpy() - np.array(fd))
    S.sync_status()
    d = np.array(diffs)
    z = d.mean(0) / (d.std(0, ddof=1) / np.sqrt(len(d)))
    assert np.all(np.abs(z) < 3.5), z


def test_caustic_gradient_direction_matches_central_differences():
    """The attached LRB-3 height gradient of the caustic inverse problem, with the image
    adjoint taken from an independent render (so that it is not correlated with the paths
    being differentiated), against common-random-number central differences of the full
    renderer along two smooth directions that leave the slab's border still (no silhouette
    moves): per seed the two differ (re-decided Fresnel branches and triangle hits), over 48
    seeds their paired difference is within 3.5 standard errors of zero and the gradient's
    projection has the sign of the differences."""
    sc = I.slab_scene(64, n=16, seed=0)
    S = lt.Scene(sc)
    T_S = lt.Scene(I.slab_scene(64, n=16, seed=1))
    target = T_S.primal(T_S.opts(seed=5, n_paths=1 << 22, max_depth=6))
    del T_S
    h0 = S.heights.clone()
    img = S.primal(S.opts(seed=99, n_paths=1 << 22, max_depth=6))
    dI = 2.0 * (img - target) / img.numel()
    g = np.linspace(-1, 1, 16)
    X, Z = np.meshgrid(g, g)
    window = np.clip(1.0 - np.maximum(np.abs(X), np.abs(Z)), 0, None) ** 2  # zero on the border ring
    dirs = [window * np.exp(-((X - 0.2) ** 2 + (Z + 0.1) ** 2) / 0.18),
            window * np.cos(2.0 * X) * np.sin(1.5 * Z + 0.3)]
    eps = 1e-4
    for v_np in dirs:
        v = torch.tensor((v_np / np.abs(v_np).max()).reshape(-1), dtype=torch.float32, device="cuda")
        ad, fd = [], []
        for s in range(48):
            kw = dict(seed=700 + s, n_paths=1 << 17, max_depth=6)
            S.refit(h0)
            gH = S.backward_lrb3(S.opts(attached=1, **kw), dI)[2][: h0.numel()]
            ad.append(float((gH.double() * v.double()).sum()))
            f = []
            for sgn in (1.0, -1.0):
                S.refit(h0 + sgn * eps * v)
                f.append(_loss64(S.primal(S.opts(**kw)), dI))
            fd.append((f[0] - f[1]) / (2 * eps))
        S.refit(h0)
        ad, fd = np.array(ad), np.array(fd)
        d = ad - fd
        z = d.mean() / (d.std(ddof=1) / np.sqrt(len(d)))
        assert abs(z) < 3.5, (z, ad.mean(), fd.mean())
        assert np.sign(ad.mean()) == np.sign(fd.mean()), (ad.mean(), fd.mean())
    S.sync_status()


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
