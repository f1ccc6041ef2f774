"""The paper-literal attached transport (opts.literal: forward-accumulated two-point
Jacobians, the determinant-guarded inverse, optional Jacobian noise; Eq. 18-19, Sec. 5) on the
GPU against its FP64 oracle restatement per seed, and its bias against naive AD of the exact
model over seeds, with and without the noise."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2609_32920_gb300 import inputs as I
from paper_2609_32920_gb300 import lt
from tests.gpu_util import agree_mask, rel_l2, t32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def slab():
    sc = I.slab_scene(48, n=12)
    return sc, lt.Scene(sc)


@pytest.mark.parametrize("D,noise", [(3, False), (8, False), (8, True)])
def test_literal_transport_matches_oracle_per_seed(slab, D, noise):
    sc, S = slab
    n, seed = 1 << 13, 11
    dI_np = I.smooth_adjoint(sc.W, sc.H, 61)
    mask = agree_mask(S, sc, seed, n, D, max_divergent=2e-3)
    o = S.opts(seed=seed, n_paths=n, max_depth=D, attached=1, mask=torch.tensor(mask, device="cuda"), literal=1,
               jac_noise=int(noise), noise_seed=5)
    gA, gL, gH = S.backward_lrb3(o, t32(dI_np))
    ref = O.gradient_literal(sc, dI_np, seed=seed, n_paths=n, max_depth=D, mask=mask, jac_noise=noise,
                             noise_seed=5)
    S.sync_status()
    assert rel_l2(gH.cpu().numpy(), ref["d_heights"]) < 1e-3
    assert rel_l2(gL.cpu().numpy(), ref["d_Le"]) < 1e-3
    if D == 3:  # every chain starts at the emitter: the literal transport is the exact one
        ex = S.backward_lrb3(S.opts(seed=seed, n_paths=n, max_depth=D, attached=1,
                                    mask=torch.tensor(mask, device="cuda")), t32(dI_np))[2]
        assert rel_l2(gH.cpu().numpy(), ex.cpu().numpy()) < 1e-4


def test_literal_transport_bias_over_seeds(slab):
    """Paired per seed against naive AD of the exact model (oracle): the mean difference of a
    random projection of the height gradient over 64 seeds, in standard errors.  With the
    Jacobian noise (a new noise seed per seed) it is unbiased; with the determinant guard alone
    the transport of chains that start after a diffuse vertex is lost, a bias."""
    sc, S = slab
    n, D = 1 << 12, 8
    dI_np = I.smooth_adjoint(sc.W, sc.H, 61)
    proj = np.random.default_rng(3).normal(size=sc.heights.size)
    z, rel = {}, {}
    for noise in (True, False):
        d, r = [], []
        for s in range(64):
            seed = 900 + s
            mask = agree_mask(S, sc, seed, n, D, max_divergent=2e-3)
            o = S.opts(seed=seed, n_paths=n, max_depth=D, attached=1, mask=torch.tensor(mask, device="cuda"),
                       literal=1, jac_noise=int(noise), noise_seed=7000 + s)
            g = S.backward_lrb3(o, t32(dI_np))[2].cpu().numpy().astype(np.float64)
            ref = O.gradient(sc, dI_np, seed=seed, n_paths=n, max_depth=D, attached=1, mask=mask)["d_heights"]
            d.append((g - ref) @ proj)
            r.append(rel_l2(g, ref))
        d = np.array(d)
        z[noise] = d.mean() / (d.std(ddof=1) / np.sqrt(len(d)))
        rel[noise] = float(np.mean(r))
    S.sync_status()
    print("literal transport vs naive AD over 64 seeds: z (noise, guard only)", z[True], z[False],
          "mean per-seed relative L2", rel[True], rel[False])
    assert abs(z[True]) < 3.5, z
    assert rel[False] > 1e-2, rel  # the guard alone is not the exact gradient
