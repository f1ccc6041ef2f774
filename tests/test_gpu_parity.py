"""GPU (liblt, CUDA) vs FP64 oracle on the same seeded inputs.

Tolerances: primal pixels |a-b| <= 1e-4 max(|b|, 1e-3 mean|b|); per-seed gradients
relative L2 <= 1e-3; discrete decisions (hashes, reservoir winners, connection counts)
bit-exact on every path whose decisions agree (paths whose FP32 and FP64 decisions
differ are counted, bounded, and masked out on both sides)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2609_32920_gb300 import inputs as I
from paper_2609_32920_gb300 import lt
from tests.gpu_util import agree_mask, primal_close, rel_l2, t32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def box64():
    sc = I.box_scene(64)
    return sc, lt.Scene(sc)


@pytest.fixture(scope="module")
def boxhm():
    sc = I.box_scene(64, heightmap=8, hm_std=0.03)
    return sc, lt.Scene(sc)


def _dev_mask(m):
    return torch.tensor(m, dtype=torch.uint8, device="cuda")


@pytest.mark.parametrize("seed,n,D", [(0, 1 << 14, 4), (3, 5000, 7)])
def test_primal_matches_oracle(box64, seed, n, D):
    sc, S = box64
    mask = agree_mask(S, sc, seed, n, D)
    img = S.primal(S.opts(seed=seed, n_paths=n, max_depth=D, mask=_dev_mask(mask))).cpu().numpy()
    ref = O.render(sc, seed=seed, n_paths=n, max_depth=D, mask=mask)
    mass = O.render(sc, seed=seed, n_paths=n, max_depth=D, mask=mask, estimator=2)
    assert np.abs(img - ref).max() <= 1e-4 * np.abs(ref).max()
    ok = primal_close(img, ref, mass=mass, W=max(sc.W, sc.H))
    assert ok.all(), f"{(~ok).sum()} pixels off; max rel {np.abs(img - ref).max() / np.abs(ref).max()}"


def test_primal_connection_counts_exact(box64):
    sc, S = box64
    n, D = 1 << 13, 6
    dbg = torch.zeros((n, 4), device="cuda")
    S.primal(S.opts(seed=5, n_paths=n, max_depth=D, dbg_out=dbg))
    ref = O.gradient(sc, I.smooth_adjoint(sc.W, sc.H, 0), seed=5, n_paths=n, max_depth=D, want_dbg=True,
                     want_hash=True)
    mask = agree_mask(S, sc, 5, n, D).astype(bool)
    assert np.array_equal(dbg.cpu().numpy()[mask, 0], ref["dbg"][mask, 3])


@pytest.mark.parametrize("seed,D,split", [(0, 4, False), (1, 12, False), (1, 12, True)])
def test_lrb3_detached_matches_naive_ad(box64, seed, D, split):
    """split: passes 2 and 3 as two kernels with the per-path state in global memory."""
    sc, S = box64
    n = 1 << 14
    dI_np = I.smooth_adjoint(sc.W, sc.H, 10 + seed)
    mask = agree_mask(S, sc, seed, n, D)
    dbg = torch.zeros((n, 4), device="cuda")
    state = S.new_lrb3_state(n) if split else None
    gA, gL, _ = S.backward_lrb3(S.opts(seed=seed, n_paths=n, max_depth=D, mask=_dev_mask(mask), dbg_out=dbg,
                                       lrb3_state=state), t32(dI_np))
    ref = O.gradient(sc, dI_np, seed=seed, n_paths=n, max_depth=D, mask=mask, want_dbg=True)
    assert rel_l2(gA.cpu().numpy(), ref["d_albedo"]) < 1e-3
    assert rel_l2(gL.cpu().numpy(), ref["d_Le"]) < 1e-3
    m = mask.astype(bool)
    d = dbg.cpu().numpy()
    assert np.array_equal(d[m, 3], ref["dbg"][m, 3])  # connection counts per path
    assert rel_l2(d[m, :3], ref["dbg"][m, :3]) < 1e-4  # delta_total per path (Eq. 14)


def test_reslrb_detached_records_and_gradient(box64):
    sc, S = box64
    n, D, seed = 1 << 14, 8, 2
    dI_np = I.smooth_adjoint(sc.W, sc.H, 21)
    mask = agree_mask(S, sc, seed, n, D)
    o = S.opts(seed=seed, n_paths=n, max_depth=D, mask=_dev_mask(mask))
    rec = torch.zeros((n, 8), device="cuda")
    img = S.primal(o, estimator=lt.EST_RESLRB, aux=rec).cpu().numpy()
    ref_img, ref_rec = O.render(sc, seed=seed, n_paths=n, max_depth=D, estimator=1, mask=mask, want_records=True)
    r = rec.cpu().numpy()
    R = r[:, 0].view(np.int32)
    m = mask.astype(bool)
    assert np.array_equal(R[m], ref_rec[m, 0].astype(np.int32)), "reservoir winners differ"
    sel = m & (R >= 0)
    assert np.allclose(r[sel, 1], ref_rec[sel, 1], rtol=1e-4)          # Omega / omega_R
    assert np.allclose(r[sel, 2:4], ref_rec[sel, 2:4], rtol=0, atol=1e-3)  # u_R (pixels)
    assert rel_l2(r[sel, 4:7], ref_rec[sel, 4:7]) < 1e-4                # S
    # primal image of the reservoir estimator: winners' splats scaled by Omega/omega_R;
    # the mass bound uses the full-estimator tap mass scaled by the largest weight
    mass = O.render(sc, seed=seed, n_paths=n, max_depth=D, mask=mask, estimator=2) * max(1.0, r[sel, 1].max())
    assert primal_close(img, ref_img, mass=mass, W=max(sc.W, sc.H)).all()
    gA, gL, _ = S.backward_reslrb(o, t32(dI_np), rec)
    refg = O.gradient(sc, dI_np, seed=seed, n_paths=n, max_depth=D, method=O.RESLRB_AD, mask=mask)
    assert rel_l2(gA.cpu().numpy(), refg["d_albedo"]) < 1e-3
    assert rel_l2(gL.cpu().numpy(), refg["d_Le"]) < 1e-3


def test_naive_detached_matches_oracle(box64):
    sc, S = box64
    n, D, seed = 1 << 14, 6, 4
    dI_np = I.smooth_adjoint(sc.W, sc.H, 31)
    mask = agree_mask(S, sc, seed, n, D)
    o = S.opts(seed=seed, n_paths=n, max_depth=D, mask=_dev_mask(mask))
    ws = torch.empty(S.naive_workspace_bytes(o), dtype=torch.uint8, device="cuda")
    S.primal(o, estimator=lt.EST_NAIVE, aux=ws)
    gA, gL, _ = S.backward_naive(o, t32(dI_np), ws)
    ref = O.gradient(sc, dI_np, seed=seed, n_paths=n, max_depth=D, mask=mask)
    assert rel_l2(gA.cpu().numpy(), ref["d_albedo"]) < 1e-3
    assert rel_l2(gL.cpu().numpy(), ref["d_Le"]) < 1e-3


@pytest.mark.parametrize("fixture_name,attached", [("box64", 0), ("boxhm", 1), ("slab", 1)])
def test_lrb3_reuses_primal_validity_masks(request, fixture_name, attached):
    """A plain primal given the LRB-3 state stores each path's connection-validity mask;
    pass 2 then traces no visibility rays and the gradient is the one of the full passes."""
    sc, S = request.getfixturevalue(fixture_name)
    n, D, seed = 1 << 13, 8, 31
    dI = t32(I.smooth_adjoint(sc.W, sc.H, 33))
    state = S.new_lrb3_state(n)
    h = torch.zeros(n, dtype=torch.int32, device="cuda")
    o = S.opts(seed=seed, n_paths=n, max_depth=D, attached=attached, lrb3_state=state, hash_out=h)
    img = S.primal(o)
    h_ref = torch.zeros(n, dtype=torch.int32, device="cuda")
    ref_img = S.primal(S.opts(seed=seed, n_paths=n, max_depth=D, hash_out=h_ref))
    assert rel_l2(img.cpu().numpy(), ref_img.cpu().numpy()) < 1e-6
    # the primal given the state visits its paths in its own order: every path once, with the
    # decisions of the index-ordered run
    assert torch.equal(h, h_ref)
    om = S.opts(seed=seed, n_paths=n, max_depth=D, attached=attached, lrb3_state=state, lrb3_mask_ready=1)
    g = S.backward_lrb3(om, dI)
    ref = S.backward_lrb3(S.opts(seed=seed, n_paths=n, max_depth=D, attached=attached), dI)
    S.sync_status()
    for x, y in zip(g, ref):
        assert rel_l2(x.cpu().numpy(), y.cpu().numpy()) < 1e-5


@pytest.mark.parametrize("fixture_name,attached,D", [("boxhm", 1, 8), ("slab", 1, 8), ("boxhm", 0, 40)])
def test_single_connection_paths_take_delta_total_from_the_primal_record(request, fixture_name, attached, D):
    """With the primal's masks, pass 2 forms delta_total of a path with one valid connection
    from the primal's record of that connection (film position and contribution) instead of
    replaying it: per path, the same delta_total and connection count as the replay of the
    fused form, on every path with a connection (depth 40: validity bits beyond 32 too)."""
    sc, S = request.getfixturevalue(fixture_name)
    n, seed = 1 << 13, 37
    dI = t32(I.smooth_adjoint(sc.W, sc.H, 39))
    state = S.new_lrb3_state(n)
    S.primal(S.opts(seed=seed, n_paths=n, max_depth=D, attached=attached, lrb3_state=state))
    dbg = torch.zeros((n, 4), device="cuda")
    S.backward_lrb3(S.opts(seed=seed, n_paths=n, max_depth=D, attached=attached, lrb3_state=state,
                           lrb3_mask_ready=1, dbg_out=dbg), dI)
    ref = torch.zeros((n, 4), device="cuda")
    S.backward_lrb3(S.opts(seed=seed, n_paths=n, max_depth=D, attached=attached, dbg_out=ref), dI)
    S.sync_status()
    a, b = dbg.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)
    lit = b[:, 3] > 0
    one = b[:, 3] == 1
    assert one.sum() > 100 and one.sum() <= lit.sum()
    assert np.array_equal(a[lit, 3], b[lit, 3])
    scale = np.abs(b[lit, :3]).max()
    assert np.abs(a[lit, :3] - b[lit, :3]).max() <= 1e-6 * scale
    assert np.all(a[~lit] == 0)


def _lrb2(S, o, dI, **kw):
    """Buffered two-pass: primal with splat records, then the backward from them."""
    buf = torch.empty(S.lrb2_buffer_bytes(o), dtype=torch.uint8, device="cuda")
    img = S.primal(o, estimator=lt.EST_BUFFERED, aux=buf)
    return img, S.backward_lrb2(o, dI, buf, **kw)


def test_lrb2_detached_matches_naive_ad_and_lrb3(box64):
    sc, S = box64
    n, D, seed = 1 << 14, 9, 8
    dI_np = I.smooth_adjoint(sc.W, sc.H, 18)
    mask = agree_mask(S, sc, seed, n, D)
    dbg = torch.zeros((n, 4), device="cuda")
    o = S.opts(seed=seed, n_paths=n, max_depth=D, mask=_dev_mask(mask), dbg_out=dbg)
    img, (gA, gL, _) = _lrb2(S, o, t32(dI_np))
    ref = O.gradient(sc, dI_np, seed=seed, n_paths=n, max_depth=D, mask=mask, want_dbg=True)
    assert rel_l2(gA.cpu().numpy(), ref["d_albedo"]) < 1e-3
    assert rel_l2(gL.cpu().numpy(), ref["d_Le"]) < 1e-3
    m = mask.astype(bool)
    d = dbg.cpu().numpy()
    assert np.array_equal(d[m, 3], ref["dbg"][m, 3])
    assert rel_l2(d[m, :3], ref["dbg"][m, :3]) < 1e-4
    # the same gradient as LRB-3 per seed, and the same image as the plain primal
    g3 = S.backward_lrb3(S.opts(seed=seed, n_paths=n, max_depth=D, mask=_dev_mask(mask)), t32(dI_np))
    assert rel_l2(gA.cpu().numpy(), g3[0].cpu().numpy()) < 1e-5
    plain = S.primal(S.opts(seed=seed, n_paths=n, max_depth=D, mask=_dev_mask(mask)))
    assert rel_l2(img.cpu().numpy(), plain.cpu().numpy()) < 1e-6
    small = torch.empty(S.lrb2_buffer_bytes(o) - 1, dtype=torch.uint8, device="cuda")
    with pytest.raises(lt.LTError) as e:
        S.primal(o, estimator=lt.EST_BUFFERED, aux=small)
    assert e.value.status == lt.LT_ERR_OOM
    with pytest.raises(lt.LTError) as e:
        S.backward_lrb2(o, t32(dI_np), small)
    assert e.value.status == lt.LT_ERR_OOM


@pytest.mark.parametrize("method", ["lrb3", "lrb3_split", "lrb2", "reslrb", "naive"])
def test_attached_height_field_matches_oracle(boxhm, method):
    sc, S = boxhm
    n, D, seed = 1 << 14, 6, 6
    dI_np = I.smooth_adjoint(sc.W, sc.H, 41)
    mask = agree_mask(S, sc, seed, n, D)
    state = S.new_lrb3_state(n) if method == "lrb3_split" else None
    o = S.opts(seed=seed, n_paths=n, max_depth=D, attached=1, mask=_dev_mask(mask), lrb3_state=state)
    dI = t32(dI_np)
    if method.startswith("lrb3"):
        gA, gL, gH = S.backward_lrb3(o, dI)
        ref = O.gradient(sc, dI_np, seed=seed, n_paths=n, max_depth=D, attached=1, mask=mask)
    elif method == "lrb2":
        _, (gA, gL, gH) = _lrb2(S, o, dI)
        ref = O.gradient(sc, dI_np, seed=seed, n_paths=n, max_depth=D, attached=1, mask=mask)
    elif method == "reslrb":
        rec = torch.zeros((n, 8), device="cuda")
        S.primal(o, estimator=lt.EST_RESLRB, aux=rec)
        gA, gL, gH = S.backward_reslrb(o, dI, rec)
        ref = O.gradient(sc, dI_np, seed=seed, n_paths=n, max_depth=D, attached=1, method=O.RESLRB_AD, mask=mask)
    else:
        ws = torch.empty(S.naive_workspace_bytes(o), dtype=torch.uint8, device="cuda")
        S.primal(o, estimator=lt.EST_NAIVE, aux=ws)
        gA, gL, gH = S.backward_naive(o, dI, ws)
        ref = O.gradient(sc, dI_np, seed=seed, n_paths=n, max_depth=D, attached=1, mask=mask)
    assert rel_l2(gH.cpu().numpy(), ref["d_heights"]) < 1e-3
    assert rel_l2(gL.cpu().numpy(), ref["d_Le"]) < 1e-3
    assert rel_l2(gA.cpu().numpy(), ref["d_albedo"]) < 1e-3


def test_ragged_offset_and_depth_limits(box64):
    sc, S = box64
    dI_np = I.smooth_adjoint(sc.W, sc.H, 51)
    for n, off, D in [(1, 0, 1), (1000, 12345, 5), (777, (1 << 33) + 5, 64)]:
        mask = agree_mask(S, sc, 9, n, D, path_offset=off, n_norm=1 << 20)
        o = S.opts(seed=9, n_paths=n, max_depth=D, path_offset=off, n_norm=1 << 20, mask=_dev_mask(mask))
        img = S.primal(o).cpu().numpy()
        ref = O.render(sc, seed=9, n_paths=n, max_depth=D, path_begin=off, n_norm=1 << 20, mask=mask)
        mass = O.render(sc, seed=9, n_paths=n, max_depth=D, path_begin=off, n_norm=1 << 20, mask=mask, estimator=2)
        assert primal_close(img, ref, mass=mass, W=max(sc.W, sc.H)).all()
        gA, gL, _ = S.backward_lrb3(o, t32(dI_np))
        r = O.gradient(sc, dI_np, seed=9, n_paths=n, max_depth=D, path_begin=off, n_norm=1 << 20, mask=mask)
        assert rel_l2(gA.cpu().numpy(), r["d_albedo"]) < 1e-3


def test_empty_and_degenerate_inputs(box64):
    sc, S = box64
    o = S.opts(seed=0, n_paths=0, max_depth=4)
    img = S.primal(o)
    assert float(img.abs().sum()) == 0.0
    gA, gL, _ = S.backward_lrb3(o, torch.ones((sc.H, sc.W, 3), device="cuda"))
    assert float(gA.abs().sum()) == 0 and float(gL.abs().sum()) == 0
    # camera facing away: no connection is ever valid, so image and gradients vanish
    away = I.box_scene(16)
    away.cam_look = np.array([0.5, 0.5, -3.0])
    S2 = lt.Scene(away)
    o = S2.opts(seed=1, n_paths=4096, max_depth=4)
    assert float(S2.primal(o).abs().sum()) == 0.0
    gA, gL, _ = S2.backward_lrb3(o, torch.ones((16, 16, 3), device="cuda"))
    assert float(gA.abs().sum()) == 0.0
    # zero adjoint: zero gradient
    gA, gL, _ = S.backward_lrb3(S.opts(seed=0, n_paths=4096, max_depth=4), torch.zeros((sc.H, sc.W, 3), device="cuda"))
    assert float(gA.abs().sum()) == 0.0


def test_invalid_arguments_raise(box64):
    sc, S = box64
    with pytest.raises(lt.LTError) as e:
        S.primal(S.opts(n_paths=16, max_depth=0))
    assert e.value.status == lt.LT_ERR_INVALID_ARG
    with pytest.raises(lt.LTError):
        S.primal(S.opts(n_paths=16, max_depth=65))
    o = S.opts(n_paths=1024, max_depth=8)
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(lt.LTError) as e:
        S.primal(o, estimator=lt.EST_NAIVE, aux=small)
    assert e.value.status == lt.LT_ERR_OOM
    with pytest.raises(lt.LTError) as e:
        S.primal(o, estimator=lt.EST_RESLRB, aux=None)
    assert e.value.status == lt.LT_ERR_INVALID_ARG
    short = torch.empty(S.lrb3_state_bytes(1024) - 1, dtype=torch.uint8, device="cuda")
    with pytest.raises(lt.LTError) as e:
        S.backward_lrb3(S.opts(n_paths=1024, max_depth=8, lrb3_state=short), torch.zeros((sc.H, sc.W, 3), device="cuda"))
    assert e.value.status == lt.LT_ERR_INVALID_ARG
    S.sync_status()


def test_film_l2_kernel():
    torch.manual_seed(0)
    I_ = torch.rand(64, 64, 3, device="cuda")
    T = torch.rand(64, 64, 3, device="cuda")
    loss, d = lt.film_l2(I_, T)
    n = I_.numel()
    ref_loss = float(((I_.double() - T.double()) ** 2).sum() / n)
    assert float(loss) == pytest.approx(ref_loss, rel=1e-5)
    assert torch.allclose(d, 2 * (I_ - T) / n, rtol=1e-6, atol=1e-12)


@pytest.fixture(scope="module")
def slab():
    sc = I.slab_scene(48, n=12)
    return sc, lt.Scene(sc)


@pytest.mark.parametrize("method,D", [("lrb3", 4), ("lrb3", 8), ("reslrb", 8), ("naive", 8), ("lrb3", 12),
                                      ("lrb3_split", 12), ("lrb2", 12)])
def test_attached_caustic_slab_matches_oracle(slab, method, D):
    """Dielectric height field: attached gradients through specular chains (first- and
    later-generation chains, anchors that are themselves chain ends)."""
    sc, S = slab
    n, seed = 1 << 13, 11
    dI_np = I.smooth_adjoint(sc.W, sc.H, 61)
    mask = agree_mask(S, sc, seed, n, D, max_divergent=2e-3)
    state = S.new_lrb3_state(n) if method == "lrb3_split" else None
    o = S.opts(seed=seed, n_paths=n, max_depth=D, attached=1, mask=_dev_mask(mask), lrb3_state=state)
    dI = t32(dI_np)
    if method.startswith("lrb3"):
        gA, gL, gH = S.backward_lrb3(o, dI)
        ref = O.gradient(sc, dI_np, seed=seed, n_paths=n, max_depth=D, attached=1, mask=mask)
    elif method == "lrb2":
        _, (gA, gL, gH) = _lrb2(S, o, dI)
        ref = O.gradient(sc, dI_np, seed=seed, n_paths=n, max_depth=D, attached=1, mask=mask)
    elif method == "reslrb":
        rec = torch.zeros((n, 8), device="cuda")
        S.primal(o, estimator=lt.EST_RESLRB, aux=rec)
        gA, gL, gH = S.backward_reslrb(o, dI, rec)
        ref = O.gradient(sc, dI_np, seed=seed, n_paths=n, max_depth=D, attached=1, method=O.RESLRB_AD, mask=mask)
    else:
        ws = torch.empty(S.naive_workspace_bytes(o), dtype=torch.uint8, device="cuda")
        S.primal(o, estimator=lt.EST_NAIVE, aux=ws)
        gA, gL, gH = S.backward_naive(o, dI, ws)
        ref = O.gradient(sc, dI_np, seed=seed, n_paths=n, max_depth=D, attached=1, mask=mask)
    S.sync_status()
    assert rel_l2(gH.cpu().numpy(), ref["d_heights"]) < 1e-3
    assert rel_l2(gL.cpu().numpy(), ref["d_Le"]) < 1e-3


def test_detached_caustic_slab_matches_oracle(slab):
    sc, S = slab
    n, seed, D = 1 << 13, 12, 8
    mask = agree_mask(S, sc, seed, n, D, max_divergent=2e-3)
    o = S.opts(seed=seed, n_paths=n, max_depth=D, mask=_dev_mask(mask))
    img = S.primal(o).cpu().numpy()
    ref = O.render(sc, seed=seed, n_paths=n, max_depth=D, mask=mask)
    mass = O.render(sc, seed=seed, n_paths=n, max_depth=D, mask=mask, estimator=2)
    assert primal_close(img, ref, mass=mass, W=max(sc.W, sc.H)).all()
    dI_np = I.smooth_adjoint(sc.W, sc.H, 62)
    gA, gL, _ = S.backward_lrb3(o, t32(dI_np))
    r = O.gradient(sc, dI_np, seed=seed, n_paths=n, max_depth=D, mask=mask)
    assert rel_l2(gL.cpu().numpy(), r["d_Le"]) < 1e-3
    assert rel_l2(gA.cpu().numpy(), r["d_albedo"]) < 1e-3


@pytest.mark.parametrize("width", [2, 4, 8])
def test_bvh_widths_match_oracle(boxhm, slab, width):
    """Every BVH width (threaded binary, 4- and 8-wide ordered traversal) gives the
    oracle's decisions, image and attached gradients."""
    for (sc, S), D, seed in ((boxhm, 6, 71), (slab, 8, 72)):
        n = 1 << 13
        h = torch.zeros(n, dtype=torch.int32, device="cuda")
        S.primal(S.opts(seed=seed, n_paths=n, max_depth=D, hash_out=h, bvh_width=width))
        g = h.cpu().numpy().view(np.uint32)
        _, oh = O.render(sc, seed=seed, n_paths=n, max_depth=D, want_hash=True)
        assert (g != oh).mean() <= 2e-3
        mask = (g == oh).astype(np.uint8)
        dI_np = I.smooth_adjoint(sc.W, sc.H, seed)
        o = S.opts(seed=seed, n_paths=n, max_depth=D, attached=1, mask=_dev_mask(mask), bvh_width=width)
        img = S.primal(o).cpu().numpy()
        ref = O.render(sc, seed=seed, n_paths=n, max_depth=D, mask=mask)
        mass = O.render(sc, seed=seed, n_paths=n, max_depth=D, mask=mask, estimator=2)
        assert primal_close(img, ref, mass=mass, W=max(sc.W, sc.H)).all()
        gA, gL, gH = S.backward_lrb3(o, t32(dI_np))
        r = O.gradient(sc, dI_np, seed=seed, n_paths=n, max_depth=D, attached=1, mask=mask)
        S.sync_status()
        assert rel_l2(gH.cpu().numpy(), r["d_heights"]) < 1e-3
        assert rel_l2(gL.cpu().numpy(), r["d_Le"]) < 1e-3


def test_bvh_width_rejected_when_unsupported(box64):
    sc, S = box64
    with pytest.raises(lt.LTError) as e:
        S.primal(S.opts(n_paths=16, max_depth=4, bvh_width=3))
    assert e.value.status == lt.LT_ERR_INVALID_ARG


def test_device_check_reports_a_corrupt_buffer(box64):
    """Device-side checks return an error status instead of faulting: a buffered two-pass
    buffer whose per-path vertex counts exceed max_depth (as after a primal with other
    options) makes the reduction set the scene's error word, which lt_sync_status reports
    as LT_ERR_DEVICE_CHECK and clears."""
    sc, S = box64
    n, D = 256, 4
    o = S.opts(seed=1, n_paths=n, max_depth=D)
    buf = torch.zeros(S.lrb2_buffer_bytes(o), dtype=torch.uint8, device="cuda")
    # the buffer begins with the LRB-3 delta_total/mask words (16 + 4 B per path, each
    # array 256-B aligned), then the per-path vertex counts
    a256 = lambda x: (x + 255) // 256 * 256  # noqa: E731
    head = a256(16 * n) + a256(4 * n)
    buf[head: head + 4 * n].view(torch.int32).fill_(D + 5)  # impossible vertex counts
    S.backward_lrb2(o, torch.zeros((sc.H, sc.W, 3), device="cuda"), buf)
    with pytest.raises(lt.LTError) as e:
        S.sync_status()
    assert e.value.status == lt.LT_ERR_DEVICE_CHECK
    S.sync_status()  # cleared


@pytest.mark.parametrize("method", ["lrb3", "lrb2", "reslrb", "naive"])
def test_russian_roulette_matches_oracle(boxhm, slab, method):
    """Russian roulette (continue with probability 0.7 after depth 2) gives the oracle's
    decisions, image and attached gradients in every method: each replay ends a path at
    the vertex the primal ended it."""
    rr = dict(rr_depth=2, rr_prob=0.7)
    for (sc, S), seed in ((boxhm, 81), (slab, 82)):
        n, D = 1 << 13, 10
        h = torch.zeros(n, dtype=torch.int32, device="cuda")
        S.primal(S.opts(seed=seed, n_paths=n, max_depth=D, hash_out=h, **rr))
        g = h.cpu().numpy().view(np.uint32)
        _, oh = O.render(sc, seed=seed, n_paths=n, max_depth=D, want_hash=True, **rr)
        assert (g != oh).mean() <= 2e-3
        mask = (g == oh).astype(np.uint8)
        dI_np = I.smooth_adjoint(sc.W, sc.H, seed)
        dI = t32(dI_np)
        state = S.new_lrb3_state(n)
        o = S.opts(seed=seed, n_paths=n, max_depth=D, attached=1, mask=_dev_mask(mask), lrb3_state=state, **rr)
        if method == "lrb3":
            img = S.primal(o)
            om = S.opts(seed=seed, n_paths=n, max_depth=D, attached=1, mask=_dev_mask(mask), lrb3_state=state,
                        lrb3_mask_ready=1, **rr)
            gA, gL, gH = S.backward_lrb3(om, dI)
            ref = O.gradient(sc, dI_np, seed=seed, n_paths=n, max_depth=D, attached=1, mask=mask, **rr)
            oimg = O.render(sc, seed=seed, n_paths=n, max_depth=D, mask=mask, **rr)
            mass = O.render(sc, seed=seed, n_paths=n, max_depth=D, mask=mask, estimator=2, **rr)
            assert primal_close(img.cpu().numpy(), oimg, mass=mass, W=max(sc.W, sc.H)).all()
        elif method == "lrb2":
            _, (gA, gL, gH) = _lrb2(S, o, dI)
            ref = O.gradient(sc, dI_np, seed=seed, n_paths=n, max_depth=D, attached=1, mask=mask, **rr)
        elif method == "reslrb":
            rec = torch.zeros((n, 8), device="cuda")
            S.primal(o, estimator=lt.EST_RESLRB, aux=rec)
            gA, gL, gH = S.backward_reslrb(o, dI, rec)
            ref = O.gradient(sc, dI_np, seed=seed, n_paths=n, max_depth=D, attached=1, method=O.RESLRB_AD,
                             mask=mask, **rr)
        else:
            ws = torch.empty(S.naive_workspace_bytes(o), dtype=torch.uint8, device="cuda")
            S.primal(o, estimator=lt.EST_NAIVE, aux=ws)
            gA, gL, gH = S.backward_naive(o, dI, ws)
            ref = O.gradient(sc, dI_np, seed=seed, n_paths=n, max_depth=D, attached=1, mask=mask, **rr)
        S.sync_status()
        assert rel_l2(gH.cpu().numpy(), ref["d_heights"]) < 1e-3
        assert rel_l2(gL.cpu().numpy(), ref["d_Le"]) < 1e-3


@pytest.mark.parametrize("method", ["lrb3", "reslrb"])
def test_gaussian_filter_matches_oracle(boxhm, slab, method):
    """The wider (Gaussian) reconstruction filter in splat and adjoint read, including the
    splat-position derivative of the attached gradients, agrees with the oracle."""
    for (sc, S), seed in ((boxhm, 91), (slab, 92)):
        n, D = 1 << 13, 6
        mask = agree_mask(S, sc, seed, n, D, max_divergent=2e-3)
        dI_np = I.smooth_adjoint(sc.W, sc.H, seed)
        dI = t32(dI_np)
        o = S.opts(seed=seed, n_paths=n, max_depth=D, attached=1, mask=_dev_mask(mask), filter=1)
        if method == "lrb3":
            img = S.primal(o).cpu().numpy()
            ref_img = O.render(sc, seed=seed, n_paths=n, max_depth=D, mask=mask, filter=1)
            mass = O.render(sc, seed=seed, n_paths=n, max_depth=D, mask=mask, estimator=2, filter=1)
            assert primal_close(img, ref_img, mass=mass, W=max(sc.W, sc.H)).all()
            gA, gL, gH = S.backward_lrb3(o, dI)
            ref = O.gradient(sc, dI_np, seed=seed, n_paths=n, max_depth=D, attached=1, mask=mask, filter=1)
        else:
            rec = torch.zeros((n, 8), device="cuda")
            S.primal(o, estimator=lt.EST_RESLRB, aux=rec)
            gA, gL, gH = S.backward_reslrb(o, dI, rec)
            ref = O.gradient(sc, dI_np, seed=seed, n_paths=n, max_depth=D, attached=1, method=O.RESLRB_AD,
                             mask=mask, filter=1)
        S.sync_status()
        assert rel_l2(gH.cpu().numpy(), ref["d_heights"]) < 1e-3
        assert rel_l2(gL.cpu().numpy(), ref["d_Le"]) < 1e-3


KINK_PX = 5e-3  # above the largest FP32 film-position drift measured at these sizes (2.7e-3 px)


def _sampled_full_size_check(sc, N, D, seed, blk, dI_seed):
    """Launch every path index of the full range; a path mask keeps the paths of nine
    blocks spread over the range (the last one ends at the last path), which the oracle
    computes one by one with the full-size normalisation 1/N.  Paths whose FP32 and FP64
    decisions differ, or that have a connection within the FP32 drift of a pixel centre
    (where the tent filter's derivative jumps), are masked out on both sides.

    Along deep paths the FP32 vertex positions drift from the FP64 ones (each vertex is
    found from its predecessor, and grazing intersections and refraction amplify the
    rounding: film positions differ by up to a few 1e-3 pixels, splat values by about 1e-4
    relative through the texture lookups), beyond what a per-pixel bound linear in the path
    length covers.  A film-position error only moves a splat's weight between the pixels
    of its 2x2 tap square, so the image is held to: its flux (sum) within 1e-5 relative;
    its relative L2 within 1e-4, and within 1e-4 after summing each pixel's 3x3 neighbourhood
    (which contains every tap square touching the pixel, so that a film-position error
    cancels there); every unlit pixel exactly zero.  (Measured: box 3.6e-5 and 1.4e-5,
    caustic 6.1e-5 and 2.8e-5; the per-pixel bound of the small cases, with its
    film-position term linear in the path length, holds on all but about 3 in 100 000 lit
    pixels of the box at depth 16.)  The reservoir
    weights are held to 1e-3 and the gradients to the 1e-3 relative L2 of the small cases."""
    S = lt.Scene(sc)
    rng = np.random.default_rng(11)
    offs = sorted(int(x) for x in rng.choice(N - blk, 8, replace=False)) + [N - blk]
    dI_np = I.smooth_adjoint(sc.W, sc.H, dI_seed)
    dI = t32(dI_np)
    # decision hashes over the full launch, compared on the sampled blocks
    h = torch.zeros(N, dtype=torch.int32, device="cuda")
    S.primal(S.opts(seed=seed, n_paths=N, max_depth=D, hash_out=h))
    g_hash = h.cpu().numpy().view(np.uint32)
    mask = np.zeros(N, dtype=np.uint8)
    agree = {}
    for o in offs:
        _, oh = O.render(sc, seed=seed, n_paths=blk, max_depth=D, path_begin=o, n_norm=N, want_hash=True)
        agree[o] = (g_hash[o:o + blk] == oh).astype(np.uint8)
    assert sum(a.sum() for a in agree.values()) >= 0.998 * blk * len(offs), \
        "too many paths took different discrete decisions"
    # The tent filter's derivative jumps at pixel centres (Eq. 21): a path with a connection
    # within the FP32 film-position drift of one may take the other one-sided derivative
    # than the FP64 oracle, so it is left out like a path with different decisions.
    for o in offs:
        _, kr = O.render(sc, seed=seed, n_paths=blk, max_depth=D, path_begin=o, n_norm=N, estimator=3,
                         want_records=True)
        agree[o] &= (kr[:, 0] >= KINK_PX).astype(np.uint8)
        mask[o:o + blk] = agree[o]
    m_dev = _dev_mask(mask)

    # primal (plain estimator, storing the LRB-3 validity masks) and LRB-3 backward
    state = S.new_lrb3_state(N)
    o_p = S.opts(seed=seed, n_paths=N, max_depth=D, mask=m_dev, lrb3_state=state)
    img = S.primal(o_p).cpu().numpy()
    o_b = S.opts(seed=seed, n_paths=N, max_depth=D, attached=1, mask=m_dev, lrb3_state=state, lrb3_mask_ready=1)
    gA, gL, gH = S.backward_lrb3(o_b, dI)
    ref_img = np.zeros_like(img, dtype=np.float64)
    mass = np.zeros_like(ref_img)
    ref = None
    for o in offs:
        kw = dict(seed=seed, n_paths=blk, max_depth=D, path_begin=o, n_norm=N, mask=agree[o])
        ref_img += O.render(sc, **kw)
        mass += O.render(sc, estimator=2, **kw)
        r = O.gradient(sc, dI_np, attached=1, **kw)
        ref = r if ref is None else {k: ref[k] + r[k] for k in ("d_albedo", "d_Le", "d_heights")}
    def box3(a):
        p = np.pad(np.asarray(a, dtype=np.float64), ((1, 1), (1, 1), (0, 0)))
        return sum(p[i:i + a.shape[0], j:j + a.shape[1]] for i in range(3) for j in range(3))
    lit = ref_img != 0
    close = primal_close(img, ref_img, mass=mass, W=max(sc.W, sc.H), depth=D)
    print("full-size primal: rel L2 %.2e, 3x3-summed rel L2 %.2e, flux rel %.2e, per-pixel bound met on %.5f of lit "
          "pixels" % (rel_l2(img, ref_img), rel_l2(box3(img), box3(ref_img)),
                      abs(img.sum() - ref_img.sum()) / abs(ref_img.sum()), close[lit].mean()))
    assert abs(img.sum() - ref_img.sum()) <= 1e-5 * abs(ref_img.sum())
    assert rel_l2(img, ref_img) < 1e-4
    assert rel_l2(box3(img), box3(ref_img)) < 1e-4
    assert np.all(img[~lit] == 0)
    errs = [rel_l2(x.cpu().numpy(), ref[k]) for x, k in ((gH, "d_heights"), (gL, "d_Le"), (gA, "d_albedo"))]
    assert max(errs) < 1e-3, f"LRB-3 gradient relative L2 (heights, Le, albedo): {errs}"

    # ResLRB: reservoir winners bit-exact on the sampled paths, then its gradient
    rec = torch.zeros((N, 8), device="cuda")
    o_r = S.opts(seed=seed, n_paths=N, max_depth=D, attached=1, mask=m_dev)
    S.primal(o_r, estimator=lt.EST_RESLRB, aux=rec)
    gA, gL, gH = S.backward_reslrb(o_r, dI, rec)
    r_all = rec.cpu().numpy()
    ref = None
    for o in offs:
        kw = dict(seed=seed, n_paths=blk, max_depth=D, path_begin=o, n_norm=N, mask=agree[o])
        _, rr = O.render(sc, estimator=1, want_records=True, **kw)
        m = agree[o].astype(bool)
        R = r_all[o:o + blk, 0].view(np.int32)
        assert np.array_equal(R[m], rr[m, 0].astype(np.int32)), "reservoir winners differ"
        sel = m & (R >= 0)
        assert np.allclose(r_all[o:o + blk][sel, 1], rr[sel, 1], rtol=1e-3)
        g = O.gradient(sc, dI_np, attached=1, method=O.RESLRB_AD, **kw)
        ref = g if ref is None else {k: ref[k] + g[k] for k in ("d_albedo", "d_Le", "d_heights")}
    errs = [rel_l2(x.cpu().numpy(), ref[k]) for x, k in ((gH, "d_heights"), (gL, "d_Le"), (gA, "d_albedo"))]
    assert max(errs) < 1e-3, f"ResLRB gradient relative L2 (heights, Le, albedo): {errs}"


def test_bench_size_sampled_paths_match_oracle():
    """The bench workload in the bench's launch configuration: box 256x256 with the 32x32
    height field, 2^22 paths, depth 16, attached; the primal stores the validity masks and
    LRB-3 runs as two kernels that reuse them; ResLRB with its 32-byte records."""
    _sampled_full_size_check(I.box_scene(256, heightmap=32), 1 << 22, 16, 1, 500, 61)


def test_caustic_full_size_sampled_paths_match_oracle():
    """The caustic workload at its full size: slab with the 128x128 height field over the
    receiver, 512x512, 2^24 paths, depth 8, attached (specular chains), as the bench's
    caustic study launches it."""
    _sampled_full_size_check(I.slab_scene(512, n=128, seed=0), 1 << 24, 8, 3, 4000, 62)


# Paths of the caustic workload (slab512_hm128, seed 3) whose first specular chain reflects
# and ends at a sliding diffuse vertex that anchors a second chain ending in a connection:
# found by scanning the FP64 oracle's paths.
SECOND_GENERATION_PATHS = [3369, 10344, 13028, 13605, 16623, 20825, 24369, 29502, 29615, 43839, 44944, 49760,
                           49840, 54435, 54953, 58738, 63040, 70633, 74762, 78854]


def test_chain_cache_matches_replay_on_second_generation_chains():
    """The attached LRB-3 pass 3 reads chain vertex states from the forward walk's cache; the
    naive baseline replays them.  On paths whose second chain's anchor adjoint continues
    through an earlier, reflecting chain (geometry only: that chain's Fresnel factors are
    counted once) both must give the same per-path height gradient, and the oracle's."""
    sc = I.slab_scene(512, n=128, seed=0)
    S = lt.Scene(sc)
    N, D, seed = 1 << 24, 8, 3
    dI_np = I.smooth_adjoint(sc.W, sc.H, 62)
    dI = t32(dI_np)
    for p in SECOND_GENERATION_PATHS:
        kw = dict(seed=seed, n_paths=1, path_offset=p, n_norm=N, max_depth=D, attached=1)
        g = S.backward_lrb3(S.opts(lrb3_state=S.new_lrb3_state(1), **kw), dI)[2].cpu().numpy()
        o = S.opts(**kw)
        ws = torch.empty(S.naive_workspace_bytes(o), dtype=torch.uint8, device="cuda")
        S.primal(o, estimator=lt.EST_NAIVE, aux=ws)
        gn = S.backward_naive(o, dI, ws)[2].cpu().numpy()
        ref = O.gradient(sc, dI_np, seed=seed, n_paths=1, max_depth=D, attached=1, path_begin=p, n_norm=N)
        assert rel_l2(g, gn) < 1e-5, f"path {p}: cached and replayed chains differ"
        assert rel_l2(g, ref["d_heights"]) < 1e-3, f"path {p}: differs from the oracle"


def _expectation_z(d, seeds):
    """Per-parameter z-scores of the mean of paired differences d [seeds, params] (only the
    parameters that receive a gradient) and the z-scores of three seeded random projections
    of the whole mean."""
    sd = d.std(axis=0, ddof=1)
    ok = sd > 0
    z = d.mean(axis=0)[ok] / (sd[ok] / np.sqrt(seeds))
    zp = []
    for k in range(3):
        p = d @ (np.random.default_rng(7 + k).normal(size=d.shape[1]) * ok)
        zp.append(p.mean() / (p.std(ddof=1) / np.sqrt(seeds)))
    return z, np.array(zp)


@pytest.mark.parametrize("attached", [0, 1])
def test_reslrb_matches_naive_in_expectation_over_256_seeds(boxhm, attached):
    """Eq. 10: ResLRB is unbiased for the gradient.  Over 256 seeds its mean matches the
    oracle's naive tape AD of the full estimator (every connection), paired per seed on the
    same paths to cancel path noise (paths whose FP32 and FP64 decisions differ are masked
    on both sides).  Criteria: each of three random projections of the mean difference
    within 3 standard errors; per parameter, at least 99 % of the z-scores within 3 and
    their mean square in [0.7, 1.4] (for independent parameters the chi-square 0.1-99.9 %
    band of a mean of ~1000 squares is [0.86, 1.15]; neighbouring texels and heights share
    paths, which widens it; a bias of half a standard deviation would put it near 64)."""
    sc, S = boxhm
    n, D, seeds = 1 << 12, 6, 256
    dI_np = I.smooth_adjoint(sc.W, sc.H, 91)
    dI = t32(dI_np)
    gi, key = (2, "d_heights") if attached else (0, "d_albedo")
    diffs = []
    for s in range(seeds):
        seed = 5000 + s
        mask = agree_mask(S, sc, seed, n, D)
        o = S.opts(seed=seed, n_paths=n, max_depth=D, attached=attached, mask=_dev_mask(mask))
        rec = torch.zeros((n, 8), device="cuda")
        S.primal(o, estimator=lt.EST_RESLRB, aux=rec)
        res = S.backward_reslrb(o, dI, rec)
        ref = O.gradient(sc, dI_np, seed=seed, n_paths=n, max_depth=D, attached=attached, mask=mask)
        diffs.append(np.concatenate([res[gi].cpu().numpy()[: ref[key].size] - ref[key],
                                     res[1].cpu().numpy() - ref["d_Le"]]))
    S.sync_status()
    d = np.array(diffs, dtype=np.float64)
    z, zp = _expectation_z(d, seeds)
    assert z.size >= 10
    assert np.mean(np.abs(z) <= 3.0) >= 0.99, np.sort(np.abs(z))[-5:]
    assert 0.7 < np.mean(z * z) < 1.4, np.mean(z * z)
    assert np.all(np.abs(zp) < 3.0), zp


@pytest.mark.parametrize("which", ["slab128", "boxhm"])
def test_scatter_modes_agree(which):
    """Every way of bringing gradients and splats to memory (opts.scatter: per-block
    shared-memory arrays within 46 KB or within the opt-in limit, plain global atomics,
    warp-aggregated global atomics for gradients and splats) gives the same image and
    gradients up to the order of float additions; the 128x128 height field (64 KB) goes
    to global memory by default and to shared memory under the opt-in limit."""
    sc = I.slab_scene(96, n=128, seed=0) if which == "slab128" else I.box_scene(64, heightmap=8, hm_std=0.03)
    S = lt.Scene(sc)
    n, D, seed = 1 << 16, 6, 3
    dI = t32(I.smooth_adjoint(sc.W, sc.H, 77))
    out = {}
    for mode in (0, 1, 2, 3):
        state = S.new_lrb3_state(n)
        op = S.opts(seed=seed, n_paths=n, max_depth=D, lrb3_state=state, scatter=mode)
        img = S.primal(op).cpu().numpy()
        om = S.opts(seed=seed, n_paths=n, max_depth=D, attached=1, lrb3_state=state, lrb3_mask_ready=1,
                    scatter=mode)
        g = [x.cpu().numpy() for x in S.backward_lrb3(om, dI)]
        rec = torch.zeros((n, 8), device="cuda")
        o = S.opts(seed=seed, n_paths=n, max_depth=D, attached=1, scatter=mode)
        S.primal(o, estimator=lt.EST_RESLRB, aux=rec)
        gr = [x.cpu().numpy() for x in S.backward_reslrb(o, dI, rec)]
        out[mode] = (img, g, gr)
    S.sync_status()
    ref = out[2]
    assert np.abs(ref[1][2]).sum() > 0
    for mode in (0, 1, 3):
        img, g, gr = out[mode]
        assert rel_l2(img, ref[0]) < 1e-6, mode
        for a, b in zip(g + gr, ref[1] + ref[2]):
            assert rel_l2(a, b) < 1e-5, mode
