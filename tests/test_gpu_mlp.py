"""Learned reservoir target on the GPU: tensor-core MLP forward/backward against the FP64
oracle network (BFloat16 roundings emulated), training, pair collection, and the
unbiasedness and variance of ResLRB with the learned target."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2609_32920_gb300 import inputs as I
from paper_2609_32920_gb300 import lt
from tests.gpu_util import agree_mask, rel_l2, t32

pytestmark = pytest.mark.gpu


def _params(seed):
    P = lt.mlp_init(seed).cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(seed)
    P[1024:1088] = rng.normal(size=64) * 0.1
    P[5184:5248] = rng.normal(size=64) * 0.1
    P[5312] = 0.2
    P[5313:5329] = rng.normal(size=16) * 0.2
    P[5329:5345] = rng.uniform(0.5, 2.0, size=16)
    P[5345], P[5346] = 1.3, -0.5
    return P


@pytest.mark.parametrize("n", [1, 37, 4096])
def test_mlp_forward_matches_oracle(n):
    P = _params(1)
    X = np.random.default_rng(2).normal(size=(n, 16))
    y = lt.mlp_forward(t32(P), t32(X)).cpu().numpy()
    ref = O.mlp_forward(P, X, round_bf16=True)
    scale = max(np.abs(ref).mean(), 1e-3)
    assert np.max(np.abs(y - ref)) / scale < 5e-3


def test_mlp_gradient_matches_oracle():
    P = _params(3)
    rng = np.random.default_rng(4)
    X = rng.normal(size=(1000, 16))
    T = rng.normal(size=1000) * 1.3 - 0.5
    g = torch.zeros(lt.MLP_WEIGHTS, device="cuda")
    loss = torch.zeros(1, device="cuda")
    lt.mlp_grad(t32(P), t32(X), t32(T), g, loss)
    ref, ref_loss = O.mlp_grad(P, X, T, round_bf16=True)
    gg = g.cpu().numpy()
    assert float(loss) == pytest.approx(ref_loss, rel=2e-3)
    # per parameter group (the GEMM operands are BFloat16-rounded on the GPU)
    for a, b in [(0, 1024), (1024, 1088), (1088, 5184), (5184, 5248), (5248, 5312), (5312, 5313)]:
        assert rel_l2(gg[a:b], ref[a:b]) < 2e-2, (a, b)


def test_mlp_training_reduces_loss():
    rng = np.random.default_rng(5)
    X = rng.normal(size=(16384, 16))
    T = np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2] + 0.3 * np.abs(X[:, 5])
    P = lt.mlp_init(0)
    losses = lt.mlp_train(P, t32(X), t32(T), epochs=8, batch=1024, lr=2e-3)
    assert losses[-1] < 0.25 * losses[0], losses
    # the trained network predicts unseen samples of the same function
    Xt = rng.normal(size=(2048, 16))
    Tt = np.sin(Xt[:, 0]) + 0.5 * Xt[:, 1] * Xt[:, 2] + 0.3 * np.abs(Xt[:, 5])
    Pn = P.cpu().numpy()
    pred = lt.mlp_forward(P, t32(Xt)).cpu().numpy() * Pn[5345] + Pn[5346]
    assert np.mean((pred - Tt) ** 2) < 0.3 * np.var(Tt)


def test_mlp_collect_counts_every_valid_connection():
    sc = I.box_scene(64)
    S = lt.Scene(sc)
    n, D = 1 << 13, 6
    dI_np = I.smooth_adjoint(sc.W, sc.H, 71)
    o = S.opts(seed=3, n_paths=n, max_depth=D)
    f, t, cnt = S.mlp_collect(o, t32(dI_np), capacity=1 << 16, target_floor=1e-12)
    ref = O.gradient(sc, dI_np, seed=3, n_paths=n, max_depth=D, want_dbg=True)
    mask = agree_mask(S, sc, 3, n, D)
    expect = ref["dbg"][:, 3].sum()
    bad = (mask == 0).sum()
    assert abs(cnt - expect) <= bad * D  # paths with disagreeing decisions may differ
    assert np.isfinite(f.cpu().numpy()).all() and np.isfinite(t.cpu().numpy()).all()
    ff = f.cpu().numpy()
    assert np.all((ff[:, 13] >= 0) & (ff[:, 13] < 1) & (ff[:, 14] >= 0) & (ff[:, 14] < 1))
    assert np.allclose(np.linalg.norm(ff[:, 3:6], axis=1), 1, atol=1e-5)


def test_learned_reservoir_target_unbiased_and_lower_variance():
    """ResLRB with the learned target stays unbiased (paired per seed against LRB-3, which
    equals naive AD per seed) and, on a high-connectivity scene, has lower gradient
    variance than ResLRB with the luminance target."""
    sc = I.box_scene(32)
    S = lt.Scene(sc)
    D, n = 8, 1 << 13
    # the image-space adjoint of an inverse problem that is wrong in one region
    dI_np = I.blob_adjoint(sc.W, sc.H, 81)
    dI = t32(dI_np)
    f, t, _ = S.mlp_collect(S.opts(seed=999, n_paths=1 << 16, max_depth=D), dI, capacity=1 << 18,
                            target_floor=0.01 * float(np.abs(dI_np).max()))
    P = lt.mlp_init(0)
    lt.mlp_train(P, f, t, epochs=6, batch=4096, lr=2e-3)
    rows = {"lrb3": [], "plain": [], "learned": []}
    for s in range(48):
        o = S.opts(seed=100 + s, n_paths=n, max_depth=D)
        rows["lrb3"].append(S.backward_lrb3(o, dI)[0].cpu().numpy().copy())
        rec = torch.zeros((n, 8), device="cuda")
        S.primal(o, estimator=lt.EST_RESLRB, aux=rec)
        rows["plain"].append(S.backward_reslrb(o, dI, rec)[0].cpu().numpy().copy())
        ol = S.opts(seed=100 + s, n_paths=n, max_depth=D, target=lt.TARGET_MLP, mlp=P)
        S.primal(ol, estimator=lt.EST_RESLRB, aux=rec)
        rows["learned"].append(S.backward_reslrb(ol, dI, rec)[0].cpu().numpy().copy())
    S.sync_status()
    L = {k: np.array(v) for k, v in rows.items()}
    proj = np.random.default_rng(0).normal(size=L["lrb3"].shape[1])
    for k in ("plain", "learned"):
        d = (L[k] - L["lrb3"]) @ proj
        z = d.mean() / (d.std(ddof=1) / np.sqrt(len(d)))
        assert abs(z) < 3.5, (k, z)
    var = {k: L[k].var(axis=0, ddof=1).mean() for k in L}
    print("mean per-parameter variance", var)
    assert var["learned"] < var["plain"]


def test_mlp_collect_pairs_match_oracle_connections():
    """Every training pair of the learned target against an FP64 computation from the
    oracle's own connections: the 16 features (position, arrival-side normal, arrival
    direction, log throughput, relative depth, film position, log connection weight) and
    the regression target log(|Lbar * L|_1 / lum(L) + floor) (Lbar: the filter-weighted
    read of dI, Eq. 21).  Rows are matched one to one by depth and nearest film position
    (rows of one depth lie far farther apart on the film than the FP32 drift of a
    position); paths whose FP32 and FP64 decisions differ are masked on both sides.  Along
    a path the FP32 vertex positions drift from the FP64 ones (each vertex is found from its
    predecessor): up to a few 1e-3 pixels on the film at depth 6, which moves the tent
    weights of the adjoint read and so the target by a few 1e-3; the bounds below allow for
    that, and 99 % of the targets must agree within 1e-3."""
    from scipy.spatial import cKDTree
    sc = I.box_scene(64, heightmap=8, hm_std=0.03)
    S = lt.Scene(sc)
    n, D, seed = 1 << 13, 6, 17
    dI_np = I.blob_adjoint(sc.W, sc.H, 5)
    floor = 0.01 * float(np.abs(dI_np).max())
    mask = agree_mask(S, sc, seed, n, D)
    o = S.opts(seed=seed, n_paths=n, max_depth=D, mask=torch.tensor(mask, device="cuda"))
    f, t, cnt = S.mlp_collect(o, t32(dI_np), capacity=1 << 17, target_floor=floor)
    rows = O.connections(sc, dI_np, seed=seed, n_paths=n, max_depth=D, mask=mask)
    L, Lb = rows[:, 17:20], rows[:, 20:23]
    lum = 0.2126 * L[:, 0] + 0.7152 * L[:, 1] + 0.0722 * L[:, 2]
    rows, L, Lb, lum = rows[lum > 0], L[lum > 0], Lb[lum > 0], lum[lum > 0]
    assert cnt == rows.shape[0]
    ref_f = np.concatenate([rows[:, 2:11], np.log(rows[:, 11:14] + 1e-30), ((rows[:, 1] + 1) / D)[:, None],
                            (rows[:, 14] / sc.W)[:, None], (rows[:, 15] / sc.H)[:, None],
                            np.log(rows[:, 16] + 1e-30)[:, None]], axis=1)
    ref_t = np.log(np.abs(Lb * L).sum(axis=1) / lum + floor)
    gf, gt = f.cpu().numpy().astype(np.float64), t.cpu().numpy().astype(np.float64)
    # key: depth (far apart) and film position in pixels
    key = lambda F: np.stack([F[:, 12] * D * 1e3, F[:, 13] * sc.W, F[:, 14] * sc.H], axis=1)  # noqa: E731
    dist, idx = cKDTree(key(ref_f)).query(key(gf))
    assert dist.max() < 1e-2 and np.unique(idx).size == idx.size  # a one-to-one matching
    ref_f, ref_t = ref_f[idx], ref_t[idx]
    assert np.array_equal(gf[:, 12], np.float32(ref_f[:, 12]).astype(np.float64))  # same depths
    assert np.abs(gf[:, 13:15] - ref_f[:, 13:15]).max() < 5e-5           # film position / size
    assert np.abs(gf[:, 0:9] - ref_f[:, 0:9]).max() < 2e-4               # position, normal, direction
    assert np.abs(gf[:, 9:12] - ref_f[:, 9:12]).max() < 5e-4             # log throughput
    assert np.abs(gf[:, 15] - ref_f[:, 15]).max() < 5e-4                 # log connection weight
    assert np.abs(gt - ref_t).max() < 5e-3                               # regression target
    assert np.quantile(np.abs(gt - ref_t), 0.99) < 1e-3
