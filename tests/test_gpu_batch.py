"""Batched passes (lt_batch_*): many scenes of uneven size in one persistent launch per
pass, replayed from a CUDA graph, must give every item the result of the single-scene
call with the same options (up to the summation order of float atomics)."""
import numpy as np
import pytest
import torch

from paper_2609_32920_gb300 import inputs as I
from paper_2609_32920_gb300 import lt
from tests.gpu_util import rel_l2, t32

pytestmark = pytest.mark.gpu


def _close(a, b, rtol=2e-5):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return np.abs(a - b) <= rtol * np.abs(b) + 1e-6 * max(np.abs(b).max(), 1e-30)


@pytest.fixture(scope="module")
def batch_items():
    """Six items: detached and attached box scenes, caustic slabs (chains), an empty item,
    a one-path item; ragged path counts that are not multiples of any chunk size."""
    specs = [
        (I.box_scene(32), dict(n_paths=3000, max_depth=5, seed=1)),
        (I.box_scene(48, heightmap=8, hm_std=0.03), dict(n_paths=5001, max_depth=7, seed=2, attached=1)),
        (I.slab_scene(64, n=12, seed=2), dict(n_paths=20011, max_depth=6, seed=3, attached=1)),
        (I.box_scene(16), dict(n_paths=0, max_depth=4, seed=4)),
        (I.box_scene(32, tex_seed=3), dict(n_paths=1, max_depth=3, seed=5)),
        (I.slab_scene(32, n=8, seed=5), dict(n_paths=7777, max_depth=4, seed=6)),
    ]
    items = []
    for k, (sc, kw) in enumerate(specs):
        S = lt.Scene(sc)
        it = dict(scene=S, reslrb=True, **kw)
        if S.n_heights:
            it["heights"] = S.heights.clone()
        it["d_image"] = t32(I.smooth_adjoint(sc.W, sc.H, 100 + k))
        items.append(it)
    return items


def _single_opts(it):
    return it["scene"].opts(seed=it.get("seed", 0), n_paths=it["n_paths"], max_depth=it["max_depth"],
                            attached=it.get("attached", 0))


def _check_all(B):
    torch.cuda.synchronize()
    for it in B.items:
        S = it["scene"]
        o = _single_opts(it)
        if S.n_heights:
            S.refit(it["heights"])
        img = S.primal(o)
        assert _close(it["image"].cpu(), img.cpu()).all()
        g = S.backward_lrb3(o, it["d_image"])
        for x, y in zip(it["grads"], g):
            assert rel_l2(x.cpu().numpy(), y.cpu().numpy()) < 1e-4


def test_batch_primal_and_lrb3_match_single_scene_calls(batch_items):
    B = lt.Batch(batch_items)
    B.run(lt.PASS_PRIMAL)
    B.run(lt.PASS_LRB3)
    _check_all(B)
    assert np.abs(B.items[1]["grads"][2].cpu().numpy()).sum() > 0  # attached heights gradient
    assert np.abs(B.items[2]["grads"][2].cpu().numpy()).sum() > 0  # caustic chain heights gradient
    assert float(B.items[3]["image"].abs().sum()) == 0.0  # the empty item


def test_batch_two_kernel_lrb3_matches_single_scene_calls(batch_items):
    """Items with an LRB-3 state: pass 2 over all items (reusing the primal pass's
    validity masks), then pass 3 per kernel group."""
    items = [dict(it, lrb3_state=True) for it in batch_items]
    B = lt.Batch(items)
    B.run(lt.PASS_PRIMAL)
    B.run(lt.PASS_LRB3)
    _check_all(B)
    B.run(lt.PASS_PRIMAL)
    B.run(lt.PASS_LRB3)  # replayed graphs
    _check_all(B)


def test_batch_reslrb_matches_single_scene_calls(batch_items):
    B = lt.Batch(batch_items)
    B.run(lt.PASS_PRIMAL_RESLRB)
    B.run(lt.PASS_RESLRB)
    torch.cuda.synchronize()
    for it in B.items:
        S = it["scene"]
        if it["n_paths"] == 0:
            continue
        o = _single_opts(it)
        if S.n_heights:
            S.refit(it["heights"])
        rec = torch.empty_like(it["records"])
        img = S.primal(o, estimator=lt.EST_RESLRB, aux=rec)
        a, b = it["records"].cpu().numpy(), rec.cpu().numpy()
        Ra, Rb = a[:, 0].view(np.int32), b[:, 0].view(np.int32)
        same = Ra == Rb
        assert same.mean() >= 0.999
        assert _close(a[same][:, 1:7], b[same][:, 1:7], rtol=1e-5).all()
        assert _close(it["image"].cpu(), img.cpu(), rtol=1e-4).mean() > 0.999
        g = S.backward_reslrb(o, it["d_image"], it["records"])
        for x, y in zip(it["grads"], g):
            assert rel_l2(x.cpu().numpy(), y.cpu().numpy()) < 1e-4


def test_batch_graph_replay_sees_new_parameters(batch_items):
    """Buffers are fixed at creation, their contents are read at every replay: new heights
    and a new emitted radiance reach the replayed primal and backward passes."""
    B = lt.Batch(batch_items)
    B.run(lt.PASS_PRIMAL)
    B.run(lt.PASS_LRB3)
    first = [it["image"].clone() for it in B.items]
    it1 = B.items[1]
    it1["heights"].add_(torch.linspace(-0.01, 0.01, it1["heights"].numel(), device="cuda"))
    it1["Le"].mul_(1.5)
    B.run(lt.PASS_PRIMAL)
    B.run(lt.PASS_LRB3)
    torch.cuda.synchronize()
    assert _close(B.items[0]["image"].cpu(), first[0].cpu()).all()  # unchanged item, replayed
    assert not _close(it1["image"].cpu(), first[1].cpu()).all()
    _check_all(B)


def test_batch_tune_picks_a_candidate_and_keeps_results(batch_items):
    B = lt.Batch(batch_items)
    B.run(lt.PASS_PRIMAL)
    cfg, ms = B.tune(lt.PASS_LRB3, reps=1)
    assert cfg["block_size"] in (64, 128, 256) and cfg["paths_per_thread"] in (1, 2, 4, 8)
    assert cfg["bvh_width"] in (2, 4, 8)
    assert ms > 0 and B.config() == cfg
    _check_all(B)
    for w in (2, 8):
        B.set_config(block_size=64, paths_per_thread=1, blocks_per_sm=2, bvh_width=w)
        B.run(lt.PASS_PRIMAL)
        B.run(lt.PASS_LRB3)
        _check_all(B)


def test_batch_rejects_bad_requests(batch_items):
    it = dict(batch_items[0])
    it.pop("reslrb", None)
    B = lt.Batch([it])
    with pytest.raises(lt.LTError) as e:
        B.run(lt.PASS_RESLRB)
    assert e.value.status == lt.LT_ERR_INVALID_ARG
    with pytest.raises(lt.LTError):
        B.run(7)
    with pytest.raises(lt.LTError):
        B.set_config(block_size=96)
    two = [dict(batch_items[1]), dict(batch_items[1])]
    with pytest.raises(lt.LTError) as e:
        lt.Batch(two)
    assert e.value.status == lt.LT_ERR_INVALID_ARG


def test_batch_items_match_oracle():
    """The batched kernels against the FP64 oracle directly (not only against the
    single-scene calls): a box with a diffuse height field, a caustic slab (specular chains)
    and a detached textured box, attached where they have heights, with ragged path counts.
    LRB-3 runs in its two-kernel form (batched pass 2 over all items, pass 3 by spans with
    shared-memory gradient sinks) and in its fused form, ResLRB through its batched primal
    and backward; the rare paths whose FP32 and FP64 decisions differ are masked on both
    sides (decision hashes)."""
    from oracle import oracle as O
    from tests.gpu_util import agree_mask, primal_close
    specs = [(I.box_scene(48, heightmap=8, hm_std=0.03), dict(n_paths=4001, max_depth=6, seed=21, attached=1)),
             (I.slab_scene(48, n=10, seed=2), dict(n_paths=6007, max_depth=6, seed=22, attached=1)),
             (I.box_scene(32, tex_seed=2), dict(n_paths=3001, max_depth=5, seed=23, attached=0))]
    items, refs = [], []
    for k, (sc, kw) in enumerate(specs):
        S = lt.Scene(sc)
        mask = agree_mask(S, sc, kw["seed"], kw["n_paths"], kw["max_depth"], max_divergent=2e-3)
        dI_np = I.smooth_adjoint(sc.W, sc.H, 300 + k)
        it = dict(scene=S, reslrb=True, mask=torch.tensor(mask, device="cuda"), d_image=t32(dI_np), **kw)
        if S.n_heights:
            it["heights"] = S.heights.clone()
        items.append(it)
        common = dict(seed=kw["seed"], n_paths=kw["n_paths"], max_depth=kw["max_depth"], mask=mask)
        refs.append(dict(
            img=O.render(sc, **common),
            mass=O.render(sc, estimator=2, **common),
            naive=O.gradient(sc, dI_np, attached=kw["attached"], **common),
            reslrb=O.gradient(sc, dI_np, attached=kw["attached"], method=O.RESLRB_AD, **common),
            sc=sc))

    def check_grads(B, key):
        torch.cuda.synchronize()
        for it, r in zip(B.items, refs):
            gA, gL, gH = (g.cpu().numpy() for g in it["grads"])
            ref = r[key]
            assert rel_l2(gL, ref["d_Le"]) < 1e-3, (key, it["n_paths"])
            if r["sc"].albedo.size:
                assert rel_l2(gA[: r["sc"].albedo.size], ref["d_albedo"]) < 1e-3, (key, it["n_paths"])
            if it["attached"] and r["sc"].heights.size:
                assert rel_l2(gH[: r["sc"].heights.size], ref["d_heights"]) < 1e-3, (key, it["n_paths"])

    for two_kernel in (True, False):
        B = lt.Batch([dict(it, lrb3_state=two_kernel) for it in items])
        B.run(lt.PASS_PRIMAL)
        B.run(lt.PASS_LRB3)
        torch.cuda.synchronize()
        for it, r in zip(B.items, refs):
            sc = r["sc"]
            ok = primal_close(it["image"].cpu().numpy(), r["img"], mass=r["mass"], W=max(sc.W, sc.H))
            assert ok.all(), (~ok).sum()
        check_grads(B, "naive")
    B = lt.Batch(items)
    B.run(lt.PASS_PRIMAL_RESLRB)
    B.run(lt.PASS_RESLRB)
    check_grads(B, "reslrb")
    for it in items:
        it["scene"].sync_status()
