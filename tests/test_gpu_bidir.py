"""Bidirectional estimator on the GPU (light-tracer connections and camera samples with
next-event estimation, combined by the balance heuristic) against the FP64 oracle: the
image, and per seed the gradient (LRB-3-pass on the light side, path replay
backpropagation on the camera side) against naive tape AD of the same combined estimator."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2609_32920_gb300 import inputs as I
from paper_2609_32920_gb300 import lt
from tests.gpu_util import rel_l2, t32

pytestmark = pytest.mark.gpu


def _masks(S, sc, seed, n, m, D):
    """Decision-hash agreement of light paths and camera samples (GPU vs oracle)."""
    h = torch.zeros(max(1, n), dtype=torch.int32, device="cuda")
    ch = torch.zeros(max(1, m), dtype=torch.int32, device="cuda")
    S.bidir_primal(S.opts(seed=seed, n_paths=n, max_depth=D, hash_out=h), S.bidir_opts(m, cam_hash=ch))
    _, oh, och = O.render_bidir(sc, m, seed=seed, n_paths=n, max_depth=D, want_hash=True)
    a = h.cpu().numpy().view(np.uint32)[:n] == oh
    b = ch.cpu().numpy().view(np.uint32)[:m] == och
    assert a.mean() >= 0.999 if n else True
    assert b.mean() >= 0.999 if m else True
    return a.astype(np.uint8), b.astype(np.uint8)


@pytest.mark.parametrize("n,m,D,seed", [(1 << 14, 1 << 14, 5, 3), (0, 5003, 4, 4), (3001, 0, 4, 5),
                                        (4096, 1 << 15, 7, 6)])
def test_bidir_image_and_gradient_match_oracle(n, m, D, seed):
    sc = I.box_scene(64)
    S = lt.Scene(sc)
    mask, cmask = _masks(S, sc, seed, n, m, D)
    dm = torch.tensor(mask, device="cuda") if n else None
    cm = torch.tensor(cmask, device="cuda") if m else None
    o = S.opts(seed=seed, n_paths=n, max_depth=D, mask=dm)
    b = S.bidir_opts(m, cam_mask=cm)
    img = S.bidir_primal(o, b).cpu().numpy()
    ref = O.render_bidir(sc, m, seed=seed, n_paths=n, max_depth=D, mask=mask if n else None,
                         cam_mask=cmask if m else None)
    assert np.abs(img - ref).max() <= 1e-4 * np.abs(ref).max()
    assert rel_l2(img, ref) < 1e-4
    dI_np = I.smooth_adjoint(sc.W, sc.H, 40 + seed)
    gA, gL, _ = S.bidir_backward(o, b, t32(dI_np))
    r = O.gradient_bidir(sc, dI_np, m, seed=seed, n_paths=n, max_depth=D, mask=mask if n else None,
                         cam_mask=cmask if m else None)
    S.sync_status()
    assert rel_l2(gA.cpu().numpy(), r["d_albedo"]) < 1e-3
    assert rel_l2(gL.cpu().numpy(), r["d_Le"]) < 1e-3


def test_bidir_without_camera_samples_is_the_light_tracer():
    sc = I.box_scene(48, heightmap=6, hm_std=0.03)
    S = lt.Scene(sc)
    o = S.opts(seed=7, n_paths=1 << 14, max_depth=6)
    b = S.bidir_opts(0)
    a = S.bidir_primal(o, b)
    ref = S.primal(o)
    assert rel_l2(a.cpu().numpy(), ref.cpu().numpy()) < 1e-6
    dI = t32(I.smooth_adjoint(sc.W, sc.H, 9))
    g = S.bidir_backward(o, b, dI)
    gr = S.backward_lrb3(o, dI)
    for x, y in zip(g[:2], gr[:2]):
        assert rel_l2(x.cpu().numpy(), y.cpu().numpy()) < 1e-5


def test_bidir_expectation_equals_light_tracer_and_lowers_variance():
    """Over 32 seeds the bidirectional image's mean equals the light tracer's (per-pixel
    z-scores), with lower variance than the light tracer given the same number of light
    paths (the camera samples are extra work)."""
    sc = I.box_scene(32)
    S = lt.Scene(sc)
    n, D, seeds = 1 << 16, 4, 32
    lt_imgs, bi_imgs = [], []
    for s in range(seeds):
        lt_imgs.append(S.primal(S.opts(seed=100 + s, n_paths=n, max_depth=D)).cpu().numpy().astype(np.float64))
        bi_imgs.append(S.bidir_primal(S.opts(seed=500 + s, n_paths=n, max_depth=D), S.bidir_opts(n))
                       .cpu().numpy().astype(np.float64))
    A, B = np.array(lt_imgs), np.array(bi_imgs)
    se = np.sqrt(A.var(0, ddof=1) / seeds + B.var(0, ddof=1) / seeds)
    z = (B.mean(0) - A.mean(0))[se > 0] / se[se > 0]
    assert 0.8 < np.mean(z * z) < 1.3 and np.abs(z).max() < 5.0, (np.mean(z * z), np.abs(z).max())
    assert B.var(0, ddof=1).mean() < A.var(0, ddof=1).mean()


def test_bidir_rejects_unsupported_requests():
    box = lt.Scene(I.box_scene(16))
    with pytest.raises(lt.LTError) as e:
        box.bidir_primal(box.opts(n_paths=64, max_depth=3, attached=1), box.bidir_opts(64))
    assert e.value.status == lt.LT_ERR_UNSUPPORTED
    slab = lt.Scene(I.slab_scene(32, n=6))
    with pytest.raises(lt.LTError) as e:
        slab.bidir_primal(slab.opts(n_paths=64, max_depth=3), slab.bidir_opts(64))
    assert e.value.status == lt.LT_ERR_UNSUPPORTED
    with pytest.raises(lt.LTError) as e:
        box.bidir_primal(box.opts(n_paths=64, max_depth=3), box.bidir_opts(-1))
    assert e.value.status == lt.LT_ERR_INVALID_ARG
