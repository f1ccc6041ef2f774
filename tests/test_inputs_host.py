"""The seeded synthetic workloads (CPU): the sizes and structure the benchmark and the
parity tests rely on, and determinism under their seeds."""
import numpy as np

from paper_2609_32920_gb300 import inputs as I


def test_caustic_slab_structure():
    """Receiver and emitter quads; an n x n height-field top (2 (n-1)^2 triangles), four side
    strips of n-1 segments (8 (n-1) triangles) and a two-triangle bottom, all dielectric
    (IOR 1.5); 512 x 512 film; n^2 heights, a sum of Gaussians, the same for the same seed."""
    n = 128
    s = I.slab_scene(512, n=n, seed=0)
    assert s.n_quads == 2 and s.n_tris == 2 * (n - 1) ** 2 + 8 * (n - 1) + 2 == 33276
    assert (s.W, s.H) == (512, 512) and s.heights.shape == (n * n,)
    mats, counts = np.unique(s.prim_mat, return_counts=True)
    dielectric = int(np.flatnonzero(s.mat_type == 1)[0])
    assert s.mat_ior[dielectric] == 1.5 and counts[list(mats).index(dielectric)] == s.n_tris
    assert np.array_equal(s.heights, I.slab_scene(512, n=n, seed=0).heights)
    other = I.slab_scene(512, n=n, seed=1).heights
    assert not np.allclose(s.heights, other)
    # a few centimetres of relief at most (8 Gaussians with N(0, 1 cm) amplitudes)
    assert 0 < np.abs(s.heights).max() < 0.06


def test_box_with_height_field_structure():
    """Five textured walls and the emitter (6 quads); a 32 x 32-vertex diffuse height field
    (1922 triangles) with N(0, 0.02) heights; 16 x 16 x 3 albedo texels per wall plus the
    height field's single texel."""
    b = I.box_scene(256, heightmap=32)
    assert b.n_quads == 6 and b.n_tris == 2 * 31 ** 2 == 1922
    assert b.heights.shape == (1024,) and abs(b.heights.std() - 0.02) < 0.002
    assert b.albedo.shape == (5 * 16 * 16 * 3 + 3,)
    assert np.all(b.albedo[:3840] >= 0.2) and np.all(b.albedo[:3840] <= 0.8)
    assert np.array_equal(b.Le, [8.0, 8.0, 8.0]) and (b.W, b.H) == (256, 256)


def test_workload_presets():
    for name, (paths, depth, W) in {"slab512_hm128": (1 << 24, 8, 512), "box256_hm32": (1 << 22, 16, 256),
                                    "box64": (1 << 14, 4, 64)}.items():
        w = I.workload(name)
        assert (w["n_paths"], w["max_depth"], w["scene"].W) == (paths, depth, W)


def test_batched_set_totals():
    """The 64-scene batched study: height-field sides in [32, 256], depths 4..32, 2^16..2^22
    paths, slab and box alternating; 62 783 488 paths and 1 781 308 triangles in all."""
    bs = I.batched_set()
    assert len(bs) == 64
    assert sum(x["n_paths"] for x in bs) == 62783488
    assert sum(x["scene"].n_tris for x in bs) == 1781308
    assert all(4 <= x["max_depth"] <= 32 and (1 << 16) <= x["n_paths"] <= (1 << 22) for x in bs)
    assert all(x["scene"].meta["kind"] == ("slab" if i % 2 == 0 else "box") for i, x in enumerate(bs))
